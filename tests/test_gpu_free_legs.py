"""Open-leg batches (jet_network_set_free): output legs left without bras stay
indices of the result (Section 2.2.1), so one multi-contraction (Section 3.2)
returns every value of those legs for each row of fixed ones, the work that
does not hold a free leg done once.

Checks against the FP64 state-vector oracle (O1):
- grid12 with every open leg free: the whole 2^12 state vector from one
  contraction, in FP32, FP16x3 and FP64;
- grid12 with 4 free legs listed out of order, 3 rows: each row's 16 values;
- the same with 2 sliced labels, and per-slice partials summing to it;
- a 2x3 bosonic lattice (Fock cutoff 4) with 2 free modes: 16 values per row;
- grid30 at full size with 4 free legs (the path and slicing planned with them
  counted at dim 2; 21.7 GB of workspace), the rows being the 8 stored
  bitstrings' other 26 digits: each row's value at the stored bitstring's free
  digits against the stored 2^30 state-vector amplitude
  (tests/golden/grid30.json).
Host-side argument errors are in test_lib_cpu.py."""
import json
import os

import numpy as np
import pytest

import oracle
from circuits import configs, circuit_to_network, gbs_lattice_circuit, Circuit, Gate
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu

GOLDEN30 = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "grid30.json")))


def rounded(circ):
    """The circuit with complex64-rounded gates and states (what the library reads)."""
    return Circuit(n=circ.n, d=circ.d,
                   gates=[Gate(np.asarray(g.matrix, np.complex64).astype(np.complex128), g.qubits, g.params, g.kind)
                          for g in circ.gates],
                   initial=[np.asarray(v, np.complex64).astype(np.complex128) for v in circ.initial])


def _expected(psi, d, n, rows, free_q):
    """psi at every row x every value of the free qudits (mixed radix, first free slowest)."""
    fixed_q = [q for q in range(n) if q not in free_q]
    out = []
    for row in rows:
        vals = []
        for e in range(d ** len(free_q)):
            digits = [0] * n
            for q, v in zip(fixed_q, [row[q] for q in fixed_q]):
                digits[q] = v
            x = e
            for q in reversed(free_q):
                digits[q] = x % d
                x //= d
            vals.append(psi[sum(v * d ** (n - 1 - q) for q, v in enumerate(digits))])
        out.append(vals)
    return np.array(out)


def _net(tn, prec, free_q, trials=8):
    net = jet.from_network(tn, precision=prec)
    net.set_free([tn.open_labels[q] for q in free_q])
    net.path_greedy(seed=1, n_trials=trials)
    return net


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp16x3", 1e-5), ("fp64", 1e-12)])
def test_grid12_whole_state_vector(prec, tol):
    w = configs.build("grid12")
    psi = oracle.sv_state(rounded(w.circuit))
    net = _net(w.network, prec, list(range(12)))
    got = net.contract(np.zeros((1, 12), np.int32))
    assert got.shape == (1, 4096)
    err = np.linalg.norm(got[0] - psi) / np.linalg.norm(psi)
    print(f"grid12 whole state, {prec}: {err:.2e}")
    assert err <= tol
    net.close()


def test_grid12_free_subset_rows_and_slices():
    w = configs.build("grid12")
    psi = oracle.sv_state(rounded(w.circuit))
    free_q = [9, 2, 6, 11]   # listed out of order: value e runs over them in this order
    rows = np.array([[1, 0, 1, 1, 0, 0, 1, 0, 1, 1, 0, 1],
                     [0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0],
                     [1, 1, 1, 0, 1, 0, 0, 1, 0, 0, 1, 0]], np.int32)
    ref = _expected(psi, 2, 12, rows, free_q)
    net = _net(w.network, "fp32", free_q)
    got = net.contract(rows)
    assert got.shape == (3, 16)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    # two sliced labels: the slices summed in FP64, and the per-slice partials
    labels = net.slice_auto(1 << 30, min_n=2, max_n=2)
    assert len(labels) == 2
    got_sl = net.contract(rows)
    assert np.linalg.norm(got_sl - ref) / np.linalg.norm(ref) <= 1e-5
    part = net.contract_slices(rows, list(range(4)))
    assert part.shape == (3, 4, 16)
    assert np.allclose(part.sum(axis=1), got_sl, rtol=0, atol=1e-12 * np.abs(ref).max())
    net.close()


def test_bosonic_lattice_free_modes():
    circ = gbs_lattice_circuit(2, 3, 4, 2, seed=11)
    tn = circuit_to_network(circ)
    psi = oracle.sv_state(rounded(circ))
    free_q = [1, 4]
    rows = np.array([[0, 0, 1, 0, 0, 1], [2, 0, 0, 1, 0, 3]], np.int32)
    ref = _expected(psi, 4, 6, rows, free_q)
    net = _net(tn, "fp32", free_q)
    got = net.contract(rows)
    assert got.shape == (2, 16)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"2x3 bosonic lattice, 2 free modes: {err:.2e}")
    assert err <= 1e-5
    net.close()


def test_grid30_four_free_legs_vs_stored_amplitudes():
    w = configs.build("grid30")
    free_q = list(range(26, 30))
    net = jet.from_network(w.network, precision="fp16x3")
    net.set_free([w.network.open_labels[q] for q in free_q])
    net.path_greedy(seed=1, n_trials=64)
    net.slice_auto(1 << 24, min_n=6, max_n=24)
    rows = np.array(GOLDEN30["outputs"], np.int32)
    got = net.contract(rows)
    assert got.shape == (len(rows), 16)
    e = [int("".join(str(v) for v in r[26:]), 2) for r in rows]
    picked = got[np.arange(len(rows)), e]
    ref = np.array([complex(a, b) for a, b in GOLDEN30["amplitudes"]])
    err = np.linalg.norm(picked - ref) / np.linalg.norm(ref)
    print(f"grid30, 4 free legs: {err:.2e} over {len(rows)} stored amplitudes")
    assert err <= 1e-5
    net.close()
