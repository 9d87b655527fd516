"""Adjoint (environment) contraction on the GPU vs the FP64 oracle.

env_G = sum_b cot_b d amp_b / dG for every gate tensor G, compared with the
oracle's state-vector adjoint (O3); the Euler identity <env_G, G> = sum_b cot_b
amp_b (an amplitude is linear in each tensor); sliced = unsliced; and angle
gradients through torch.autograd against central finite differences of the
FP64 state vector (h = 1e-3)."""
import math

import numpy as np
import pytest

import oracle
from circuits import (configs, circuit_to_network, param_grid_circuit, random_grid_circuit, gbs_lattice_circuit,
                      random_bitstrings, random_patterns, Circuit, Gate)
from circuits.rqc import gate_with_params
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu


def rounded(circ):
    return Circuit(n=circ.n, d=circ.d,
                   gates=[Gate(np.asarray(g.matrix, np.complex64).astype(np.complex128), g.qubits, g.params, g.kind)
                          for g in circ.gates],
                   initial=[np.asarray(v, np.complex64).astype(np.complex128) for v in circ.initial])


def _env_vs_oracle(circ, outs, prec, trials=8, sliced=None):
    tn = circuit_to_network(circ)
    rc = rounded(circ)
    amps_ref = oracle.sv_amplitudes(rc, outs)
    cot = np.conj(amps_ref)
    env_ref = oracle.sv_env(rc, outs, cot)
    net = jet.from_network(tn, precision=prec)
    net.path_greedy(seed=1, n_trials=trials)
    if sliced:
        net.slice_auto(sliced, min_n=2, max_n=16)
    ids = list(tn.gate_tensor)
    amps, envs = net.contract_grad(outs, cot, ids)
    got = np.concatenate([e.reshape(-1) for e in envs])
    ref = np.concatenate([e.reshape(-1) for e in env_ref])
    err_env = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    err_amp = float(np.linalg.norm(amps - amps_ref) / np.linalg.norm(amps_ref))
    return err_env, err_amp, net, tn, cot, amps, envs


# environments are returned as complex64 (the tensors' own type), so even the FP64
# path's environments carry ~2^-24 output rounding; its amplitudes are held to 1e-12
@pytest.mark.parametrize("prec,tol_env,tol_amp", [("fp32", 1e-5, 1e-5), ("fp64", 1e-7, 1e-12)])
def test_param20_environments_vs_statevector_adjoint(prec, tol_env, tol_amp):
    w = configs.build("param20")
    err_env, err_amp, *_ = _env_vs_oracle(w.circuit, w.outputs, prec, trials=16)
    print(f"{prec}: env err {err_env:.3e} amp err {err_amp:.3e}")
    assert err_env <= tol_env and err_amp <= tol_amp


def test_euler_identity_every_tensor():
    """sum_i env_G[i] G[i] = sum_b cot_b amp_b for every input tensor, kets included."""
    circ = random_grid_circuit(3, 3, 6, seed=14)
    tn = circuit_to_network(circ)
    outs = random_bitstrings(9, 5, 3)
    net = jet.from_network(tn, precision="fp64")
    net.path_greedy(seed=2, n_trials=4)
    amps0 = net.contract(outs)
    cot = np.conj(amps0) + 0.25j
    amps, envs = net.contract_grad(outs, cot, list(range(len(tn.data))))
    target = np.sum(cot * amps)
    for G, E in zip(tn.data, envs):
        g = np.asarray(G, np.complex64).astype(np.complex128)
        assert abs(np.sum(E.astype(np.complex128) * g) - target) <= 1e-6 * abs(target)


def test_sliced_gradient_equals_unsliced():
    circ = random_grid_circuit(3, 3, 8, seed=15)
    outs = random_bitstrings(9, 4, 5)
    e1, _, _, _, _, _, env1 = _env_vs_oracle(circ, outs, "fp64", trials=4)
    e2, _, net2, _, _, _, env2 = _env_vs_oracle(circ, outs, "fp64", trials=4, sliced=1 << 4)
    assert net2.stats()["n_slices"] >= 4
    assert e1 <= 1e-7 and e2 <= 1e-7
    for a, b in zip(env1, env2):
        assert np.allclose(a, b, rtol=1e-6, atol=1e-7)


def test_bosonic_environments_vs_statevector_adjoint():
    circ = gbs_lattice_circuit(2, 2, 4, 2, seed=19)
    outs = random_patterns(4, 16, 20, 4)
    err_env, err_amp, *_ = _env_vs_oracle(circ, outs, "fp32", trials=4)
    assert err_env <= 1e-5 and err_amp <= 1e-5


def _torch_gates(torch, circ, tn, thetas):
    """The circuit's gate tensors as differentiable functions of their angles."""
    def rzry_t(a, b):
        rz = torch.stack([torch.stack([torch.exp(-0.5j * a), torch.zeros((), dtype=torch.complex128)]),
                          torch.stack([torch.zeros((), dtype=torch.complex128), torch.exp(0.5j * a)])])
        c, s = torch.cos(0.5 * b).to(torch.complex128), torch.sin(0.5 * b).to(torch.complex128)
        ry = torch.stack([torch.stack([c, -s]), torch.stack([s, c])])
        return rz @ ry

    def fsim_t(th, ph):
        c, s = torch.cos(th).to(torch.complex128), torch.sin(th).to(torch.complex128)
        z, o = torch.zeros((), dtype=torch.complex128), torch.ones((), dtype=torch.complex128)
        return torch.stack([torch.stack([o, z, z, z]), torch.stack([z, c, -1j * s, z]),
                            torch.stack([z, -1j * s, c, z]), torch.stack([z, z, z, torch.exp(-1j * ph)])])

    return [(rzry_t(*t) if g.kind == "rzry" else fsim_t(*t)).reshape(tn.data[tn.gate_tensor[i]].shape)
            for i, (g, t) in enumerate(zip(circ.gates, thetas))]


def _fd(circ, outs, gi, pi, h=1e-3):
    """Central finite difference of sum |amp|^2 in FP64 (the oracle's state vector)."""
    g = circ.gates[gi]
    vals = []
    for sgn in (+1, -1):
        p = list(g.params)
        p[pi] += sgn * h
        ms = [gg.matrix for gg in circ.gates]
        ms[gi] = gate_with_params(g, p)
        vals.append(np.sum(np.abs(oracle.sv_amplitudes(circ, outs, gate_mats=ms)) ** 2))
    return (vals[0] - vals[1]) / (2 * h)


def _autograd_angle_grads(torch, circ, tn, outs, trials):
    from paper_2107_09793_b300.autograd import amplitudes
    net = jet.from_network(tn, precision="fp32")
    net.path_greedy_batch(outs, seed=1, n_trials=trials) if len(outs) > 8 else net.path_greedy(seed=1, n_trials=trials)
    thetas = [torch.tensor(list(g.params), dtype=torch.float64, requires_grad=True) for g in circ.gates]
    mats = _torch_gates(torch, circ, tn, thetas)
    amps = amplitudes(net, outs, tn.gate_tensor, [m.to(torch.complex64) for m in mats])
    loss = (amps.abs() ** 2).sum()
    loss.backward()
    net.close()
    return [t.grad.numpy() for t in thetas]


def test_angle_gradients_autograd_vs_finite_differences():
    torch = pytest.importorskip("torch")
    circ = param_grid_circuit(2, 3, 4, seed=33)
    tn = circuit_to_network(circ)
    outs = random_bitstrings(circ.n, 8, 34)
    grads = _autograd_angle_grads(torch, circ, tn, outs, 4)
    grad = np.concatenate(grads)
    fd = np.array([_fd(circ, outs, gi, pi) for gi, g in enumerate(circ.gates) for pi in range(len(g.params))])
    err = np.linalg.norm(grad - fd) / np.linalg.norm(fd)
    print(f"angle-gradient rel err vs central FD: {err:.3e}")
    assert err <= 1e-5


def test_param20_angle_gradients_vs_finite_differences_on_sampled_angles():
    """The full-size parameterised workload (20 qubits, 12 cycles, 64 amplitudes,
    666 angles): every angle's gradient of sum |amp|^2 from the GPU adjoint
    through torch.autograd; 12 seeded angles checked against central finite
    differences of the FP64 state vector (h = 1e-3)."""
    torch = pytest.importorskip("torch")
    from circuits import SplitMix64
    w = configs.build("param20")
    circ, tn, outs = w.circuit, w.network, w.outputs
    grads = _autograd_angle_grads(torch, circ, tn, outs, 16)
    flat = [(gi, pi) for gi, g in enumerate(circ.gates) for pi in range(len(g.params))]
    rng = SplitMix64(2020)
    pick = sorted({flat[rng.randint(len(flat))] for _ in range(12)})
    got = np.array([grads[gi][pi] for gi, pi in pick])
    fd = np.array([_fd(circ, outs, gi, pi) for gi, pi in pick])
    err = float(np.linalg.norm(got - fd) / np.linalg.norm(fd))
    print(f"param20: {len(pick)} sampled angle gradients vs central FD: rel err {err:.3e}")
    assert err <= 2e-5
