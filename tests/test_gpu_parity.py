"""CUDA path vs the FP64 oracle, element by element, on seeded inputs.

Tolerances: normwise relative error <= 1e-5 for the complex64 modes and
<= 1e-12 for the FP64 mode (normwise over the batch, Section 2.4's amplitudes;
the oracle sees the same complex64-rounded tensors upcast to complex128)."""
import math

import numpy as np
import pytest

import oracle
from circuits import (configs, random_grid_circuit, param_grid_circuit, gbs_lattice_circuit,
                      circuit_to_network, random_bitstrings, random_patterns, Circuit, Gate, SplitMix64)
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}


def rel(a, ref):
    a, ref = np.asarray(a), np.asarray(ref)
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def sv_ref(circ, outs):
    return oracle.sv_amplitudes(circ, outs)


def rounded(circ):
    """The circuit with complex64-rounded gates and initial vectors (what the GPU sees)."""
    c = Circuit(n=circ.n, d=circ.d,
                gates=[Gate(np.asarray(g.matrix, np.complex64).astype(np.complex128), g.qubits, g.params, g.kind)
                       for g in circ.gates],
                initial=[np.asarray(v, np.complex64).astype(np.complex128) for v in circ.initial])
    return c


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_grid12_batch_vs_statevector(prec):
    w = configs.build("grid12")
    net = jet.from_network(w.network, precision=prec)
    net.path_greedy(seed=1, n_trials=8)
    outs = np.concatenate([w.outputs, random_bitstrings(12, 255, 7)])
    amps = net.contract(outs)
    ref = sv_ref(rounded(w.circuit), outs)
    assert rel(amps, ref) <= TOL[prec]
    assert abs(amps[0] - ref[0]) <= TOL[prec] * abs(ref[0]) * 10


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_sliced_sum_vs_statevector(prec):
    circ = random_grid_circuit(3, 3, 8, seed=5)
    tn = circuit_to_network(circ)
    outs = random_bitstrings(9, 6, 8)
    net = jet.from_network(tn, precision=prec)
    net.path_greedy(seed=2, n_trials=4)
    sl = net.slice_auto(1 << 5, min_n=4, max_n=12)
    assert net.stats()["n_slices"] >= 16
    amps = net.contract(outs)
    assert rel(amps, sv_ref(rounded(circ), outs)) <= TOL[prec]


def test_slice_partials_vs_oracle_einsum():
    """Each slice's partial contraction equals the oracle's (Eq. sliced_sum): slice a
    single label at a time by running the GPU with all other labels unsliced."""
    circ = random_grid_circuit(2, 3, 6, seed=6)
    tn = circuit_to_network(circ)
    x = [0, 1, 1, 0, 1, 0]
    net = jet.from_network(tn, precision="fp64")
    net.path_greedy(seed=3, n_trials=4)
    sl = net.slice_auto(1 << 3, min_n=3, max_n=8)
    full = net.contract([x])[0]
    parts = oracle.sliced_partials(rounded_tn(tn), x, sl)
    assert abs(full - parts.sum()) <= 1e-12 * abs(parts.sum())


def rounded_tn(tn):
    return tn.as_complex64()


def test_reuse_on_off_bitwise_identical():
    circ = random_grid_circuit(3, 3, 8, seed=9)
    tn = circuit_to_network(circ)
    outs = random_bitstrings(9, 4, 1)
    a = jet.from_network(tn)
    a.path_greedy(seed=1, n_trials=4)
    sl = a.slice_auto(1 << 5, min_n=3, max_n=12)
    b = jet.from_network(tn, reuse=False)
    b.path_set(a.path_get())
    b.slice(sl)
    ra, rb = a.contract(outs), b.contract(outs)
    assert np.array_equal(ra, rb)
    assert b.stats()["flop_executed"] > a.stats()["flop_executed"]


def test_path_independence_on_gpu():
    w = configs.build("grid12")
    ref = sv_ref(rounded(w.circuit), w.outputs)
    vals = []
    for seed, trials in [(1, 1), (2, 16), (3, 64)]:
        net = jet.from_network(w.network)
        net.path_greedy(seed=seed, n_trials=trials)
        vals.append(net.contract(w.outputs)[0])
    for v in vals:
        assert abs(v - ref[0]) <= 1e-5 * abs(ref[0]) * 10


def test_graph_and_eager_launches_agree():
    w = configs.build("grid12")
    a = jet.from_network(w.network, use_graph=True)
    a.path_greedy(seed=1, n_trials=4)
    b = jet.from_network(w.network, use_graph=False)
    b.path_set(a.path_get())
    outs = random_bitstrings(12, 16, 3)
    r1, r2, r3 = a.contract(outs), a.contract(outs), b.contract(outs)
    assert np.array_equal(r1, r2) and np.array_equal(r1, r3)


def test_param20_batch_vs_statevector():
    w = configs.build("param20")
    net = jet.from_network(w.network)
    net.path_greedy(seed=1, n_trials=16)
    amps = net.contract(w.outputs)
    assert rel(amps, sv_ref(rounded(w.circuit), w.outputs)) <= 1e-5


def test_gbs_small_lattice_vs_statevector():
    circ = gbs_lattice_circuit(2, 3, 4, 2, seed=17)
    tn = circuit_to_network(circ)
    outs = random_patterns(6, 32, 18, 4)
    outs[0] = 0
    net = jet.from_network(tn)
    net.path_greedy(seed=1, n_trials=8)
    amps = net.contract(outs)
    ref = sv_ref(rounded(circ), outs)
    assert rel(amps, ref) <= 1e-5
    odd = outs.sum(axis=1) % 2 == 1
    assert np.all(amps[odd] == 0)
    assert abs(amps[0] - np.prod([1 / math.sqrt(math.cosh(r)) for r in circ.squeezing])) < 1e-6


def test_edge_single_tensor_and_scalar_leaf():
    v = np.array([0.5 + 1j, -2.0], np.complex64)
    net = jet.Network([[7]], [v])
    net.set_open([7])
    net.path_set([])
    amps = net.contract([[0], [1]])
    assert np.allclose(amps, v.astype(np.complex128))
    # a rank-0 factor, a matrix and a vector: outer products and a scalar
    s = np.array(2 - 1j, np.complex64).reshape(())
    m = np.array([[1, 2j], [3, 4]], np.complex64)
    net = jet.Network([[], [0, 1], [1]], [s, m, np.array([1j, 1], np.complex64)])
    net.set_open([0])
    net.path_set([(0, 1), (3, 2)])
    got = net.contract([[0], [1]])
    ref = complex(s) * (m.astype(complex) @ np.array([1j, 1]))
    assert np.allclose(got, ref, rtol=1e-6)


def test_edge_non_power_of_two_dims():
    """Qutrits (d=3): the general (div/mod) index decode."""
    rng = SplitMix64(5)
    d, n = 3, 3
    def rand_u(k):
        m = np.array([[complex(rng.uniform() - .5, rng.uniform() - .5) for _ in range(d ** k)]
                      for _ in range(d ** k)])
        q, _ = np.linalg.qr(m)
        return q
    gates = [Gate(rand_u(1), (q,)) for q in range(n)] + [Gate(rand_u(2), (0, 1)), Gate(rand_u(2), (1, 2)),
                                                         Gate(rand_u(1), (2,))]
    circ = Circuit(n=n, d=d, gates=gates, initial=[np.eye(d)[0]] * n)
    tn = circuit_to_network(circ)
    outs = np.array([[a, b, c] for a in range(3) for b in range(3) for c in range(3)], np.int32)
    net = jet.from_network(tn)
    net.path_greedy(seed=1, n_trials=2)
    net.slice_auto(9, min_n=1, max_n=6)
    amps = net.contract(outs)
    assert rel(amps, sv_ref(rounded(circ), outs)) <= 1e-5


def test_disconnected_network_outer_product():
    circ = Circuit(n=2, d=2, gates=[Gate(np.array([[0, 1], [1, 0]], complex), (0,)),
                                    Gate(np.array([[1, 1], [1, -1]], complex) / math.sqrt(2), (1,))],
                   initial=[np.eye(2)[0]] * 2)
    tn = circuit_to_network(circ)
    net = jet.from_network(tn)
    net.path_greedy(seed=1, n_trials=1)
    amps = net.contract([[1, 0], [1, 1], [0, 0]])
    assert np.allclose(amps, [1 / math.sqrt(2), 1 / math.sqrt(2), 0], atol=1e-7)


def test_user_workspace_from_torch():
    torch = pytest.importorskip("torch")
    w = configs.build("grid12")
    net = jet.from_network(w.network)
    net.path_greedy(seed=1, n_trials=4)
    nbytes = net.plan(w.outputs)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    ptr = (ws.data_ptr() + 255) // 256 * 256
    net.set_workspace(ptr, nbytes)
    stream = torch.cuda.current_stream().cuda_stream
    a1 = net.contract(w.outputs, stream=stream)
    ref = sv_ref(rounded(w.circuit), w.outputs)
    assert rel(a1, ref) <= 1e-5
    with pytest.raises(jet.JetError) as e:
        net.set_workspace(ptr, 256)
        net.contract(w.outputs, stream=stream)
    assert e.value.code == jet.JET_ENOMEM
    net.set_workspace(0, 0)


def test_contract_async_device_output():
    torch = pytest.importorskip("torch")
    w = configs.build("grid12")
    net = jet.from_network(w.network)
    net.path_greedy(seed=1, n_trials=4)
    out = torch.zeros(2, dtype=torch.complex128, device="cuda")
    s = torch.cuda.current_stream()
    net.contract_async(np.concatenate([w.outputs, w.outputs]), out.data_ptr(), s.cuda_stream)
    s.synchronize()
    ref = sv_ref(rounded(w.circuit), w.outputs)[0]
    assert abs(out[0].item() - ref) <= 1e-5 * abs(ref) * 10
    assert out[0].item() == out[1].item()
