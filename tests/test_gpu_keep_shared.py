"""Kept shared work (jet_network_keep_shared): a sub-tree whose tensors carry no
fixed label has the same value in every contraction (Section 3.2's shared work,
kept for later slices and amplitudes as the paper's conclusion proposes).  The
first contraction computes it into a device pool; later ones read it.

Checks: a second batch of different rows matches a fresh handle and executes
fewer FLOP; a tensor update inside the kept sub-tree is seen; with every open
leg free the whole network is kept and a repeat call still returns the right
values; against the FP64 state-vector oracle throughout."""
import numpy as np
import pytest

import oracle
from circuits import configs, circuit_to_network, gbs_lattice_circuit, Circuit, Gate, SplitMix64
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu


def rounded(circ):
    return Circuit(n=circ.n, d=circ.d,
                   gates=[Gate(np.asarray(g.matrix, np.complex64).astype(np.complex128), g.qubits, g.params, g.kind)
                          for g in circ.gates],
                   initial=[np.asarray(v, np.complex64).astype(np.complex128) for v in circ.initial])


def _batches(n, d, seed):
    rng = SplitMix64(seed)
    rows = np.array([[rng.randint(d) for _ in range(n)] for _ in range(12)], np.int32)
    return rows[:6], rows[6:]


@pytest.mark.parametrize("case", ["grid12", "lattice2x5"])
def test_second_batch_reads_kept_work(case):
    if case == "grid12":
        w = configs.build("grid12")
        circ, tn, d = w.circuit, w.network, 2
    else:
        circ = gbs_lattice_circuit(2, 5, 4, 2, seed=13)
        tn, d = circuit_to_network(circ), 4
    psi = oracle.sv_state(rounded(circ))
    b1, b2 = _batches(circ.n, d, 5)
    kept = jet.from_network(tn, precision="fp32")
    path_flop = kept.path_greedy_batch(b1, seed=1, n_trials=8)   # bras late: a large bra-free sub-tree
    kept.keep_shared(1 << 10)
    fresh = jet.from_network(tn, precision="fp32")
    fresh.path_set(kept.path_get())
    a1 = kept.contract(b1)
    f1 = kept.stats()["flop_executed"]
    a2 = kept.contract(b2)
    f2 = kept.stats()["flop_executed"]
    r2 = fresh.contract(b2)
    idx = lambda rows: [sum(int(v) * d ** (circ.n - 1 - q) for q, v in enumerate(r)) for r in rows]
    for got, rows in ((a1, b1), (a2, b2)):
        ref = psi[idx(rows)]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
    assert np.allclose(a2, r2, rtol=1e-6, atol=1e-7 * np.abs(r2).max())
    print(f"{case}: FLOP first batch {f1:.3g}, second {f2:.3g} (path {path_flop:.3g})")
    assert f2 < f1
    kept.close()
    fresh.close()


def test_tensor_update_drops_kept_work():
    w = configs.build("grid12")
    b1, b2 = _batches(12, 2, 7)
    net = jet.from_network(w.network, precision="fp32")
    net.path_greedy_batch(b1, seed=1, n_trials=8)
    net.keep_shared(1 << 8)
    net.contract(b1)
    # change the first gate tensor (inside the bra-free part of the network)
    t = w.network.gate_tensor[0]
    new = np.asarray(w.network.data[t], np.complex64) * np.complex64(0.5 + 0.25j)
    net.update(t, new)
    got = net.contract(b2)
    data = list(w.network.data)
    data[t] = new
    ref_net = jet.Network(w.network.labels, data, precision="fp32")
    ref_net.set_open(w.network.open_labels)
    ref_net.path_set(net.path_get())
    ref = ref_net.contract(b2)
    assert np.allclose(got, ref, rtol=1e-6, atol=1e-7 * np.abs(ref).max())
    net.close()
    ref_net.close()


def test_whole_network_kept_with_free_legs():
    w = configs.build("grid12")
    psi = oracle.sv_state(rounded(w.circuit))
    net = jet.from_network(w.network, precision="fp32")
    net.set_free(w.network.open_labels)
    net.path_greedy(seed=1, n_trials=8)
    net.keep_shared(1)
    rows = np.zeros((1, 12), np.int32)
    first = net.contract(rows)[0]
    second = net.contract(rows)[0]
    assert net.stats()["flop_executed"] == 0          # nothing left to launch but the reduction
    assert np.array_equal(first, second)
    assert np.linalg.norm(second - psi) / np.linalg.norm(psi) <= 1e-5
    net.keep_shared(0)
    third = net.contract(rows)[0]
    assert np.allclose(third, first, rtol=1e-6, atol=1e-9)
    net.close()


def test_kept_work_saved_and_loaded_by_another_handle(tmp_path):
    """The kept shared work written to a file and read by a fresh handle of the
    same network (same tensors, path, legs, threshold): its first contraction
    already skips the kept sub-trees and matches; a handle with one tensor
    changed refuses the file."""
    circ = gbs_lattice_circuit(2, 5, 4, 2, seed=13)
    tn = circuit_to_network(circ)
    b1, b2 = _batches(circ.n, 4, 5)
    first = jet.from_network(tn, precision="fp32")
    first.path_greedy_batch(b1, seed=1, n_trials=8)
    path = first.path_get()
    first.keep_shared(1 << 10)
    first.contract(b1)
    ref = first.contract(b2)
    f_kept = first.stats()["flop_executed"]
    fn = str(tmp_path / "kept.bin")
    first.save_shared(fn)
    second = jet.from_network(tn, precision="fp32")
    second.path_set(path)
    second.keep_shared(1 << 10)
    second.load_shared(fn)
    got = second.contract(b2)
    assert second.stats()["flop_executed"] == f_kept
    assert np.allclose(got, ref, rtol=1e-6, atol=1e-7 * np.abs(ref).max())
    data = list(tn.data)
    data[0] = np.asarray(data[0], np.complex64) * np.complex64(0.5)
    other = jet.Network(tn.labels, data, precision="fp32")
    other.set_open(tn.open_labels)
    other.path_set(path)
    other.keep_shared(1 << 10)
    with pytest.raises(jet.JetError):
        other.load_shared(fn)
    for n in (first, second, other):
        n.close()
