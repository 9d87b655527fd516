"""Higher Fock cutoff and 3-D lattices (Algorithm 1 with dim = 3; the cutoff-8
tensors of the paper's 2-D timing runs): every index has dimension 8 or the
lattice is three-dimensional, which changes the contraction's tile shapes.

Checks against the FP64 state-vector oracles:
- 2x2x2 lattice at cutoff 8 (8 modes, 8^8 states, dense O1): seeded patterns,
  and two rows with 4 modes left free (4096 values each);
- gbs3d at full size (2x3x3, cutoff 4, 2 layers, batch planner): patterns of
  total photon number <= 6 against the per-sector oracle, odd totals exactly
  zero, the vacuum amplitude = prod 1/sqrt(cosh r);
- gbs88d8 at full size (8x8, cutoff 8, one layer, r = 0.5): patterns of total
  <= 4 against the per-sector oracle, odd totals zero, the vacuum;
both full-size workloads on the CUDA cores (FP32) and the tensor cores (FP16x3)."""
import math

import numpy as np
import pytest

import oracle
from circuits import configs, circuit_to_network, gbs_nd_circuit, random_patterns, Circuit, Gate, SplitMix64
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu


def rounded(circ):
    return Circuit(n=circ.n, d=circ.d,
                   gates=[Gate(np.asarray(g.matrix, np.complex64).astype(np.complex128), g.qubits, g.params, g.kind)
                          for g in circ.gates],
                   initial=[np.asarray(v, np.complex64).astype(np.complex128) for v in circ.initial])


def _low_totals(n, count, max_total, seed, d):
    """Seeded patterns of small even and odd totals (vacuum first)."""
    rng = SplitMix64(seed)
    pats = [[0] * n]
    while len(pats) < count:
        total = 1 + int(rng.uniform() * max_total)
        p = [0] * n
        left = total
        while left:
            k = int(rng.uniform() * n)
            if p[k] < d - 1:
                p[k] += 1
                left -= 1
        pats.append(p)
    return np.array(pats, np.int32)


def test_cutoff8_cube_vs_dense_state_vector():
    circ = gbs_nd_circuit((2, 2, 2), 8, 2, seed=41)
    psi = oracle.sv_state(rounded(circ))
    tn = circuit_to_network(circ)
    pats = random_patterns(8, 12, 43, 8)
    net = jet.from_network(tn, precision="fp32")
    net.path_greedy(seed=1, n_trials=8)
    got = net.contract(pats)
    idx = [sum(int(v) * 8 ** (7 - q) for q, v in enumerate(p)) for p in pats]
    ref = psi[idx]
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"2x2x2 cutoff 8, 12 patterns: {err:.2e}")
    assert err <= 1e-5
    # four modes left free: 8^4 values per row
    free_q = [1, 2, 5, 6]
    net.set_free([tn.open_labels[q] for q in free_q])
    net.path_greedy(seed=1, n_trials=8)
    rows = pats[:2]
    got2 = net.contract(rows)
    assert got2.shape == (2, 4096)
    ref2 = np.zeros((2, 4096), np.complex128)
    for b, row in enumerate(rows):
        for e in range(4096):
            dig = list(row)
            x = e
            for q in reversed(free_q):
                dig[q] = x % 8
                x //= 8
            ref2[b, e] = psi[sum(int(v) * 8 ** (7 - q) for q, v in enumerate(dig))]
    err2 = np.linalg.norm(got2 - ref2) / np.linalg.norm(ref2)
    print(f"2x2x2 cutoff 8, 4 free modes: {err2:.2e}")
    assert err2 <= 1e-5
    net.close()


def _check_full_size(name, pats, tol, prec):
    w = configs.build(name)
    net = jet.from_network(w.network, precision=prec)
    net.path_greedy_batch(pats, seed=1, n_trials=8, max_elems=1 << 30)   # planned for these patterns
    got = net.contract(pats)
    ref = oracle.sector_amplitudes(rounded(w.circuit), pats)
    vac = np.prod([1 / math.sqrt(math.cosh(r)) for r in w.circuit.squeezing])
    # the oracle reads the complex64-rounded squeezers: each factor within 2^-24 relative
    assert abs(ref[0] - vac) <= w.circuit.n * 2.0 ** -24 * vac
    odd = pats.sum(axis=1) % 2 == 1
    assert odd.any() and np.all(got[odd] == 0)
    even = ~odd
    err = np.linalg.norm(got[even] - ref[even]) / np.linalg.norm(ref[even])
    print(f"{name} {prec}: {even.sum()} even-total patterns, rel err {err:.2e}")
    assert err <= tol
    net.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_gbs3d_full_size_low_totals(prec):
    w = configs.build("gbs3d")
    _check_full_size("gbs3d", _low_totals(w.circuit.n, 16, 6, 51, 4), 1e-5, prec)


@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_gbs88d8_full_size_low_totals(prec):
    w = configs.build("gbs88d8")
    _check_full_size("gbs88d8", _low_totals(w.circuit.n, 8, 4, 53, 8), 1e-5, prec)
