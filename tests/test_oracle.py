"""Pins of the FP64 oracle against what the paper and the mathematics fix
(closed forms, brute force, the worked example), never against itself."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle.einsum import contract_network, greedy_path, network_flops, slice_network
from circuits import (Circuit, Gate, circuit_to_network, configs, fsim, sqrt_x, sqrt_y,
                      sqrt_w, random_grid_circuit, param_grid_circuit, gbs_lattice_circuit,
                      gbs_nd_circuit, random_bitstrings, SplitMix64)
from circuits.rqc import gate_with_params, gate_param_derivs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_c(rng, shape):
    n = int(np.prod(shape))
    v = np.array([complex(rng.uniform() - 0.5, rng.uniform() - 0.5) for _ in range(n)])
    return v.reshape(shape)


def _paper_example(D, seed):
    """Section 2.2.1 example: S on both qudits, then B; bras <a1|_c, <a2|_f."""
    rng = SplitMix64(seed)
    S1 = _rand_c(rng, (D, D))
    S2 = _rand_c(rng, (D, D))
    B = _rand_c(rng, (D, D, D, D))
    a1, a2 = rng.randint(D), rng.randint(D)
    e = lambda i: np.eye(D, dtype=np.complex128)[i]
    # a=0 b=1 c=2 d=3 e=4 f=5
    labels = [[2], [5], [2, 5, 1, 4], [1, 0], [4, 3], [0], [3]]
    data = [e(a1), e(a2), B, S1, S2, e(0), e(0)]
    return labels, data, (S1, S2, B, a1, a2)


def _read_sequence():
    rows = []
    with open(os.path.join(GOLDEN, "paper_example_sequence.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, a, b, out, p = line.split()
            rows.append((int(a), int(b), [] if out == "-" else [int(x) for x in out.split(",")], int(p)))
    return rows


@pytest.mark.parametrize("D", [2, 4])
def test_paper_example_pairwise_equals_naive(D):
    labels, data, (S1, S2, B, a1, a2) = _paper_example(D, 11 + D)
    seq = _read_sequence()
    path = [(a, b) for a, b, _, _ in seq]
    naive = oracle.naive_sum(labels, data)
    _, t = contract_network(labels, data, path)
    assert abs(complex(t) - naive) <= 1e-12 * max(1.0, abs(naive))
    # and the state-vector route on the same two-qudit circuit
    circ = Circuit(n=2, d=D, initial=[np.eye(D)[0], np.eye(D)[0]],
                   gates=[Gate(S1, (0,)), Gate(S2, (1,)), Gate(B.reshape(D * D, D * D), (0, 1))])
    psi = oracle.sv_state(circ)
    assert abs(psi[a1 * D + a2] - naive) <= 1e-12 * max(1.0, abs(naive))


@pytest.mark.parametrize("D", [2, 4])
def test_paper_example_step_labels_and_costs(D):
    """Each step of Eq. sequence yields the printed result tensor and costs O(D^p)."""
    labels, data, _ = _paper_example(D, 3)
    dims = {x: D for x in range(6)}
    live = dict(enumerate(labels))
    nxt = len(labels)
    for a, b, out, p in _read_sequence():
        la, lb = live.pop(a), live.pop(b)
        res = [x for x in la if x not in lb] + [x for x in lb if x not in la]
        assert sorted(res) == sorted(out)
        assert network_flops([la, lb], dims, [(0, 1)]) == 8 * D ** p
        live[nxt] = res
        nxt += 1


@pytest.mark.parametrize("D", [2, 3])
def test_paper_example_sliced_sum(D):
    """Eq. sliced_sum: fixing e to each value and summing the partials."""
    labels, data, _ = _paper_example(D, 5)
    full = oracle.naive_sum(labels, data)
    parts = []
    for v in range(D):
        sl, sd = slice_network(labels, data, [4], [v])
        parts.append(oracle.naive_sum(sl, sd))
        _, t = contract_network(sl, sd)
        assert abs(complex(t) - parts[-1]) <= 1e-12
    assert abs(sum(parts) - full) <= 1e-12 * max(1, abs(full))


def _product_circuit(n, seed):
    rng = SplitMix64(seed)
    gates = []
    pool = [sqrt_x(), sqrt_y(), sqrt_w()]
    for layer in range(3):
        for q in range(n):
            gates.append(Gate(pool[rng.randint(3)], (q,)))
    return Circuit(n=n, d=2, initial=[np.array([1, 0], complex)] * n, gates=gates)


def _product_amp(circ, x):
    """Closed form for a circuit of 1-qubit gates only: prod_q (U_q...|0>)[x_q]."""
    cols = [np.array([1, 0], complex) for _ in range(circ.n)]
    for g in circ.gates:
        (q,) = g.qubits
        cols[q] = g.matrix @ cols[q]
    return np.prod([cols[q][x[q]] for q in range(circ.n)])


def test_single_qubit_only_closed_form():
    circ = _product_circuit(5, 7)
    tn = circuit_to_network(circ)
    psi = oracle.sv_state(circ)
    for xi in range(32):
        x = [(xi >> (4 - q)) & 1 for q in range(5)]
        ref = _product_amp(circ, x)
        assert abs(psi[xi] - ref) < 1e-13
        assert abs(oracle.amplitude(tn, x) - ref) < 1e-13


def test_planted_mistakes_fail_pins():
    """Transposed gates or reversed qubit order break the closed-form pin."""
    circ = _product_circuit(4, 9)
    ref = np.array([_product_amp(circ, [(xi >> (3 - q)) & 1 for q in range(4)]) for xi in range(16)])
    bad_t = Circuit(n=4, d=2, initial=circ.initial,
                    gates=[Gate(g.matrix.T, g.qubits) for g in circ.gates])
    assert np.max(abs(oracle.sv_state(bad_t) - ref)) > 1e-3
    bad_q = Circuit(n=4, d=2, initial=circ.initial,
                    gates=[Gate(g.matrix, (3 - g.qubits[0],)) for g in circ.gates])
    assert np.max(abs(oracle.sv_state(bad_q) - ref)) > 1e-3


def test_fsim_textbook_cases():
    # fSim(theta, phi)|00> = |00> for any angles
    for th, ph in [(0.3, 1.1), (math.pi / 2, math.pi / 6), (2.0, 0.0)]:
        circ = Circuit(n=2, d=2, initial=[np.array([1, 0], complex)] * 2,
                       gates=[Gate(fsim(th, ph), (0, 1))])
        psi = oracle.sv_state(circ)
        assert abs(psi[0] - 1) < 1e-15 and np.max(abs(psi[1:])) < 1e-15
    # sqrt(X)^2 = -iX, so sqrt(X)^2 on qubit 1 gives -i|01>; fSim(pi/2, 0) maps
    # |01> -> -i|10>: amplitude of |10> is (-i)(-i) = -1, all others 0.
    circ = Circuit(n=2, d=2, initial=[np.array([1, 0], complex)] * 2,
                   gates=[Gate(sqrt_x(), (1,)), Gate(sqrt_x(), (1,)), Gate(fsim(math.pi / 2, 0), (0, 1))])
    tn = circuit_to_network(circ)
    psi = oracle.sv_state(circ)
    assert abs(psi[2] + 1) < 1e-15 and abs(psi[0]) + abs(psi[1]) + abs(psi[3]) < 1e-15
    assert abs(oracle.amplitude(tn, [1, 0]) + 1) < 1e-15
    assert abs(oracle.amplitude(tn, [0, 1])) < 1e-15


def test_ghz_closed_form():
    """H on qubit 0 then a CNOT chain: amplitude 1/sqrt(2) on 0..0 and 1..1."""
    n = 5
    H = np.array([[1, 1], [1, -1]], complex) / math.sqrt(2)
    CX = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], complex)
    gates = [Gate(H, (0,))] + [Gate(CX, (q, q + 1)) for q in range(n - 1)]
    circ = Circuit(n=n, d=2, initial=[np.array([1, 0], complex)] * n, gates=gates)
    psi = oracle.sv_state(circ)
    ref = np.zeros(2 ** n, complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.max(abs(psi - ref)) < 1e-15
    tn = circuit_to_network(circ)
    for xi in [0, 1, 2 ** n - 1, 5]:
        x = [(xi >> (n - 1 - q)) & 1 for q in range(n)]
        assert abs(oracle.amplitude(tn, x) - ref[xi]) < 1e-15
    # control/target swapped is a different state: the pin sees orientation
    bad = Circuit(n=n, d=2, initial=circ.initial,
                  gates=[Gate(H, (0,))] + [Gate(CX, (q + 1, q)) for q in range(n - 1)])
    assert np.max(abs(oracle.sv_state(bad) - ref)) > 0.1


def test_norm_over_all_bitstrings_grid12():
    w = configs.build("grid12")
    psi = oracle.sv_state(w.circuit)
    assert abs(np.sum(abs(psi) ** 2) - 1) < 1e-12


def test_statevector_vs_pairwise_vs_naive_tiny():
    circ = random_grid_circuit(1, 2, 3, seed=21)
    tn = circuit_to_network(circ)
    psi = oracle.sv_state(circ)
    assert len(set(sum(tn.labels, []))) <= 16
    for xi in range(4):
        x = [(xi >> 1) & 1, xi & 1]
        labels, data = oracle.attach_bras(tn.labels, tn.data, tn.open_labels, x, 2)
        nv = oracle.naive_sum(labels, data)
        assert abs(nv - psi[xi]) < 1e-13
        assert abs(oracle.amplitude(tn, x) - psi[xi]) < 1e-13


def test_all_amplitudes_2x2_pairwise_vs_statevector():
    circ = random_grid_circuit(2, 2, 6, seed=8)
    tn = circuit_to_network(circ)
    psi = oracle.sv_state(circ)
    amps = np.array([oracle.amplitude(tn, [(xi >> (3 - q)) & 1 for q in range(4)]) for xi in range(16)])
    assert np.max(abs(amps - psi)) < 1e-13
    assert abs(np.sum(abs(amps) ** 2) - 1) < 1e-12


def _random_path(n, rng):
    ids = list(range(n))
    path, nxt = [], n
    while len(ids) > 1:
        i = rng.randint(len(ids)); a = ids.pop(i)
        j = rng.randint(len(ids)); b = ids.pop(j)
        path.append((a, b)); ids.append(nxt); nxt += 1
    return path


def test_path_independence_grid12():
    """Section 2.3: any pairwise order gives the same value (greedy, random,
    circuit order)."""
    w = configs.build("grid12")
    tn = w.network
    x = w.outputs[0]
    labels, data = oracle.attach_bras(tn.labels, tn.data, tn.open_labels, x, 2)
    ref = oracle.sv_amplitudes(w.circuit, [x])[0]
    vals = [complex(contract_network(labels, data)[1])]
    rng = SplitMix64(77)
    n = len(labels)
    seq = [(0, 1)] + [(n + k, k + 2) for k in range(n - 2)]   # circuit order: absorb one by one
    vals.append(complex(contract_network(labels, data, seq)[1]))
    for _ in range(3):
        vals.append(complex(contract_network(labels, data, _random_path_connected(labels, rng))[1]))
    for v in vals:
        assert abs(v - ref) < 1e-12


def test_stepwise_contraction_ends_at_the_state_vector_amplitude():
    """The stepwise form (one tensordot per next(), used to time parts of a
    contraction) ends at the state-vector amplitude, one step per pair."""
    from oracle.einsum import contract_pairs
    w = configs.build("grid12")
    x = w.outputs[0]
    labels, data = oracle.attach_bras(w.network.labels, w.network.data, w.network.open_labels, x, 2)
    path = greedy_path(labels, {l: 2 for ls in labels for l in ls})
    steps = list(contract_pairs(labels, data, path))
    assert [s[0] for s in steps] == list(range(len(path)))
    assert steps[-1][1] == []
    assert abs(complex(steps[-1][2]) - oracle.sv_amplitudes(w.circuit, [x])[0]) < 1e-12


def _random_path_connected(labels, rng):
    """Random order that only contracts pairs sharing an index (keeps sizes small)."""
    live = {i: set(l) for i, l in enumerate(labels)}
    nxt = len(labels)
    path = []
    while len(live) > 1:
        ids = sorted(live)
        pairs = [(a, b) for ai, a in enumerate(ids) for b in ids[ai + 1:] if live[a] & live[b]]
        if not pairs:
            pairs = [(ids[0], ids[1])]
        a, b = pairs[rng.randint(len(pairs))]
        la, lb = live.pop(a), live.pop(b)
        live[nxt] = la ^ lb
        path.append((a, b)); nxt += 1
    return path


def test_slicing_sum_equals_unsliced_grid12():
    w = configs.build("grid12")
    tn = w.network
    x = w.outputs[0]
    ref = oracle.amplitude(tn, x)
    # slice three closed labels of gates in the middle of the circuit
    closed = sorted(set(sum(tn.labels, [])) - set(tn.open_labels))
    sliced = [closed[40], closed[60], closed[90]]
    parts = oracle.sliced_partials(tn, x, sliced)
    assert len(parts) == 8
    assert abs(np.sum(parts) - ref) < 1e-13
    # each partial is itself a definite contraction: check one by brute slicing + O1 order path
    assert abs(oracle.sliced_partials(tn, x, sliced, [5])[0] - parts[5]) < 1e-15


def test_adjoint_env_identities_small():
    circ = param_grid_circuit(2, 3, 4, seed=31)
    tn = circuit_to_network(circ)
    outs = random_bitstrings(circ.n, 5, 99)
    amps = oracle.sv_amplitudes(circ, outs)
    cot = np.conj(amps)
    env = oracle.sv_env(circ, outs, cot)
    target = np.sum(cot * amps)
    # Euler identity: amplitude is linear in every gate tensor
    for g, e in zip(circ.gates, env):
        assert abs(np.sum(e * g.matrix) - target) < 1e-13
    # env of a gate equals the network contracted without that gate (pairwise route)
    for gi in [0, 7, len(circ.gates) - 1]:
        tid = tn.gate_tensor[gi]
        acc = 0
        for x, c in zip(outs, cot):
            labels, data = oracle.attach_bras(tn.labels, tn.data, tn.open_labels, x, 2)
            lab = labels[:tid] + labels[tid + 1:]
            dat = data[:tid] + data[tid + 1:]
            rl, t = contract_network(lab, dat)
            order = [rl.index(l) for l in tn.labels[tid]]
            acc = acc + c * np.transpose(t, order)
        k = len(circ.gates[gi].qubits)
        assert np.max(abs(acc.reshape(2 ** k, 2 ** k) - env[gi])) < 1e-13


def test_adjoint_vs_central_fd():
    """dL/dtheta for L = sum_b |amp_b|^2: adjoint vs central differences, h=1e-3."""
    circ = param_grid_circuit(2, 3, 4, seed=32)
    outs = random_bitstrings(circ.n, 6, 98)
    amps = oracle.sv_amplitudes(circ, outs)
    env = oracle.sv_env(circ, outs, np.conj(amps))
    grad = []
    for g, e in zip(circ.gates, env):
        for dG in gate_param_derivs(g):
            grad.append(2 * np.real(np.sum(e * dG)))
    grad = np.array(grad)
    h = 1e-3
    fd = []
    for gi, g in enumerate(circ.gates):
        for pi in range(len(g.params)):
            vals = []
            for s in (+1, -1):
                p = list(g.params); p[pi] += s * h
                mats = [gg.matrix for gg in circ.gates]
                mats[gi] = gate_with_params(g, p)
                a = oracle.sv_amplitudes(circ, outs, gate_mats=mats)
                vals.append(np.sum(abs(a) ** 2))
            fd.append((vals[0] - vals[1]) / (2 * h))
    fd = np.array(fd)
    assert np.linalg.norm(grad - fd) <= 1e-5 * np.linalg.norm(fd)


def test_bosonic_vacuum_and_parity():
    circ = gbs_lattice_circuit(2, 2, 4, 2, seed=41)
    tn = circuit_to_network(circ)
    # vacuum: passive beamsplitters leave N=0 untouched, truncation included
    ref = np.prod([1 / math.sqrt(math.cosh(r)) for r in circ.squeezing])
    assert abs(oracle.amplitude(tn, [0, 0, 0, 0]) - ref) < 1e-14
    psi = oracle.sv_state(circ)
    assert abs(psi[0] - ref) < 1e-14
    # odd total photon number: exactly zero (squeezers emit pairs, BS conserve N)
    for pat in ([1, 0, 0, 0], [1, 1, 1, 0], [3, 0, 2, 2]):
        assert oracle.amplitude(tn, pat) == 0
    # state-vector route vs pairwise route on every even pattern with N <= 4
    for xi in range(256):
        pat = [(xi >> (6 - 2 * q)) & 3 for q in range(4)]
        if sum(pat) % 2 == 0 and sum(pat) <= 4:
            assert abs(oracle.amplitude(tn, pat) - psi[xi]) < 1e-14


def test_bosonic_sector_closed_form_single_bs():
    """One beamsplitter on |1,0> (sector N=1): the 2x2 block is the rotation
    exp(theta [[0, e^{i phi}], [-e^{-i phi}, 0]])."""
    from circuits.gbs import beamsplitter
    th, ph = 0.7, 1.3
    U = beamsplitter(th, ph, 4)
    # |n1,n2> -> index n1*4+n2.  exp of theta*[[0, a],[-conj(a), 0]] with |a|=1
    a = np.exp(1j * ph)
    blk = np.array([[math.cos(th), a * math.sin(th)], [-np.conj(a) * math.sin(th), math.cos(th)]])
    idx = [0 * 4 + 1, 1 * 4 + 0]   # basis (n1=0,n2=1), (n1=1,n2=0)
    got = U[np.ix_(idx, idx)]
    assert np.max(abs(got - blk)) < 1e-14


def test_sector_counting_table_closed_form():
    """Compositions of N into n parts below d: sum_j (-1)^j C(n,j) C(N - d j + n - 1, n - 1)."""
    for n, d in [(16, 4), (6, 4), (5, 3)]:
        for N in range(0, n * (d - 1) + 1):
            ref = sum((-1) ** j * math.comb(n, j) * math.comb(N - d * j + n - 1, n - 1)
                      for j in range(0, n + 1) if N - d * j >= 0)
            assert oracle.sector_dim(n, d, N) == ref


def test_sector_state_vector_equals_dense_on_every_pattern():
    """Per-sector state vector = dense state vector on all 4^6 patterns of a
    2x3 lattice (beamsplitters with random theta, phi: a transposed block, a
    wrong rank or a dropped sector member would show)."""
    from itertools import product as iproduct
    circ = gbs_lattice_circuit(2, 3, 4, 2, seed=17)
    pats = np.array(list(iproduct(range(4), repeat=6)), np.int32)
    got = oracle.sector_amplitudes(circ, pats)
    ref = oracle.sv_amplitudes(circ, pats)
    assert np.max(np.abs(got - ref)) < 1e-14
    # and against the pairwise route on a few patterns of a 3x2 lattice (other digit strides)
    circ2 = gbs_lattice_circuit(3, 2, 4, 1, seed=23)
    tn2 = circuit_to_network(circ2)
    for p in ([0, 2, 1, 1, 0, 0], [3, 1, 0, 2, 2, 0], [1, 1, 1, 1, 1, 1]):
        assert abs(oracle.sector_amplitudes(circ2, [p])[0] - oracle.amplitude(tn2, p)) < 1e-14


def test_sector_oracle_refuses_gates_that_mix_sectors():
    circ = gbs_lattice_circuit(2, 2, 4, 1, seed=29)
    mats = [g.matrix for g in circ.gates]
    bad = np.array(mats[0], np.complex128)
    bad[0, 5] = 1e-3   # (0,0) <- (1,1): photon number 2 -> 0
    mats[0] = bad
    with pytest.raises(ValueError):
        oracle.sector_amplitudes(circ, [[0, 0, 0, 0]], gate_mats=mats)


def test_sector_oracle_full_lattice_vacuum_and_parity():
    """The 16-mode, d = 4 lattice at full size: the vacuum amplitude is the
    product of the squeezers' vacuum coefficients (passive beamsplitters leave
    N = 0 alone), odd totals vanish exactly."""
    w = configs.build("gbs16")
    circ = w.circuit
    ref = np.prod([1 / math.sqrt(math.cosh(r)) for r in circ.squeezing])
    a = oracle.sector_amplitudes(circ, [[0] * 16, [1] + [0] * 15, [1, 2] + [0] * 14])
    assert abs(a[0] - ref) < 1e-14
    assert a[1] == 0 and a[2] == 0


def test_nd_lattice_generator_reduces_to_2d_and_counts_bonds():
    """Algorithm 1 in n dimensions: for a 2-D shape the n-D generator is the 2-D
    lattice draw for draw (same squeezers, bonds, angles); a w0 x w1 x w2
    lattice has sum_a (w_a - 1) * n / w_a bonds per layer, each joining modes
    whose coordinates differ by one along one axis."""
    a, b = gbs_lattice_circuit(3, 4, 4, 2, seed=7), gbs_nd_circuit((3, 4), 4, 2, seed=7)
    assert [g.qubits for g in a.gates] == [g.qubits for g in b.gates]
    assert all(np.array_equal(g.matrix, h.matrix) for g, h in zip(a.gates, b.gates))
    assert all(np.array_equal(x, y) for x, y in zip(a.initial, b.initial))
    c = gbs_nd_circuit((2, 3, 4), 3, 2, seed=9)
    n = 24
    per_layer = sum((w - 1) * n // w for w in (2, 3, 4))
    assert len(c.gates) == 2 * per_layer
    for g in c.gates:
        p, q = g.qubits
        diff = [abs(x - y) for x, y in zip(c.sites[p], c.sites[q])]
        assert sorted(diff) == [0, 0, 1]


def test_sector_oracle_on_a_3d_lattice_every_pattern():
    """The per-sector state vector equals the dense one on all 3^8 patterns of
    a 2x2x2 lattice at cutoff 3 (bonds along all three axes)."""
    from itertools import product as iproduct
    circ = gbs_nd_circuit((2, 2, 2), 3, 2, seed=31)
    pats = np.array(list(iproduct(range(3), repeat=8)), np.int32)
    got = oracle.sector_amplitudes(circ, pats)
    ref = oracle.sv_amplitudes(circ, pats)
    assert np.max(np.abs(got - ref)) < 1e-14
