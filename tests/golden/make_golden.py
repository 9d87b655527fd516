"""Writes the stored expected values under tests/golden/ for the large workloads.

Calls only the FP64 oracle (`oracle`) and the seeded input generators
(`circuits`): every tensor is rounded to complex64 first, exactly as the CUDA
path receives it, then upcast to complex128.

  grid30.json : 30-qubit 5x6 grid circuit, 14 cycles (seed 2)
     * amplitudes of the workload's bitstring and 7 more seeded bitstrings, from the
       dense 2^30 state vector (O1, 16 GiB);
     * 4 slice partials of the workload bitstring (Eq. sliced_sum) by pairwise
       contraction (O2) for a fixed, rule-chosen set of 6 sliced labels: the wire
       label of qubits 12..17 (grid row 2) just after their 8th single-qubit gate.

  gbs16.json  : 16-mode 4x4 bosonic lattice, Fock cutoff 4, 4 beamsplitter layers
     (seed 5), the workload's 256 seeded photon patterns: the amplitudes of the 8
     even-total patterns of the batch with the smallest totals (N <= 16), each
     from the FP64 state vector of its own total-photon sector (beamsplitters
     conserve the photon number; Section 4, Algorithm 1).  Odd totals are exactly
     zero and need no stored value.

  grid53.json : 53-qubit 9x6-minus-corner grid circuit, 12 cycles (seed 3), the
     workload's bitstring: the oracle's own contraction order (its greedy path,
     improved by exhaustive re-ordering of sub-trees of up to 8 tensors until it
     stops improving) and its own sliced labels (largest intermediate <= 2^28
     elements), and the O2 partials (Eq. sliced_sum) of 8 seeded slice ids.  The
     GPU test contracts the same network along the stored order and slicing.

  grid53_bench.json : the same circuit and bitstring along the order and the 12
     sliced labels the benchmark contracts (tests/golden/grid53_plan.json, read
     as data: Section 2.3 makes the value independent of the order, and the
     sliced labels only say which partial sums s_i of Eq. sliced_sum exist), the
     O2 partials of 8 seeded slice ids, each slice contracted pairwise along that
     order by the oracle's tensordot step.

Usage: python tests/golden/make_golden.py grid30 gbs16 grid53 grid53_bench
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from circuits import configs, random_bitstrings, Circuit, Gate  # noqa: E402


def rounded(circ):
    return Circuit(n=circ.n, d=circ.d,
                   gates=[Gate(np.asarray(g.matrix, np.complex64).astype(np.complex128), g.qubits, g.params, g.kind)
                          for g in circ.gates],
                   initial=[np.asarray(v, np.complex64).astype(np.complex128) for v in circ.initial])


def rule_sliced_labels(w, qubits, nth):
    """Label on each listed qubit's wire right after its nth (0-based) 1-qubit gate."""
    tn = w.network
    count = {q: 0 for q in qubits}
    out = {}
    for gi, g in enumerate(w.circuit.gates):
        if len(g.qubits) == 1 and g.qubits[0] in count:
            q = g.qubits[0]
            if count[q] == nth:
                out[q] = tn.labels[tn.gate_tensor[gi]][0]
            count[q] += 1
    return [out[q] for q in qubits]


def grid30():
    w = configs.build("grid30")
    circ = rounded(w.circuit)
    outs = np.concatenate([w.outputs, random_bitstrings(w.circuit.n, 7, 2024)])
    t0 = time.time()
    amps = oracle.sv_amplitudes(circ, outs)
    t_sv = time.time() - t0
    sliced = rule_sliced_labels(w, list(range(12, 18)), 7)
    slice_ids = [0, 17, 42, 63]
    t0 = time.time()
    parts = oracle.sliced_partials(w.network.as_complex64(), w.outputs[0], sliced, slice_ids)
    t_o2 = time.time() - t0
    rec = {
        "workload": "grid30", "source": "oracle O1 (2^30 state vector) and O2 (pairwise numpy.tensordot)",
        "outputs": outs.tolist(),
        "amplitudes": [[a.real, a.imag] for a in amps],
        "sliced_labels": [int(x) for x in sliced],
        "slice_ids": slice_ids,
        "slice_partials": [[p.real, p.imag] for p in parts],
        "seconds": {"statevector": round(t_sv, 1), "four_slices": round(t_o2, 1)},
    }
    with open(os.path.join(HERE, "grid30.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec["seconds"]))


def gbs16():
    w = configs.build("gbs16")
    circ = rounded(w.circuit)
    tot = w.outputs.sum(axis=1)
    even = [int(i) for i in np.argsort(tot, kind="stable") if tot[i] % 2 == 0]
    pick = [i for i in even if tot[i] <= 16][:8]
    t0 = time.time()
    amps = oracle.sector_amplitudes(circ, w.outputs[pick])
    t_sec = time.time() - t0
    rec = {
        "workload": "gbs16", "source": "oracle O1, per total-photon sector (sector.c)",
        "batch_index": pick,
        "outputs": w.outputs[pick].tolist(),
        "totals": [int(tot[i]) for i in pick],
        "amplitudes": [[a.real, a.imag] for a in amps],
        "seconds": {"sectors": round(t_sec, 1)},
    }
    with open(os.path.join(HERE, "gbs16.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec["seconds"]))


def grid53():
    from oracle.einsum import greedy_path, improve_path, slice_until, network_flops, slice_network, contract_network
    from circuits import SplitMix64
    w = configs.build("grid53")
    tn = w.network.as_complex64()
    dims = {}
    for l, t in zip(tn.labels, tn.data):
        for x, sz in zip(l, t.shape):
            dims[x] = 1 if x in tn.open_labels else sz
    t0 = time.time()
    path = greedy_path(tn.labels, dims)
    prev = None
    while True:
        path = improve_path(tn.labels, dims, path, k=8, passes=5)
        f = network_flops(tn.labels, dims, path)
        if prev is not None and f >= prev:
            break
        prev = f
    sliced = slice_until(tn.labels, dims, path, 1 << 28)
    t_plan = time.time() - t0
    n_sl = 2 ** len(sliced)
    rng = SplitMix64(53)
    ids = sorted({int(rng.next_u64() % n_sl) for _ in range(8)})
    d2 = {x: (1 if x in sliced else v) for x, v in dims.items()}
    parts = []
    t0 = time.time()
    for i in ids:
        digits = [(i >> (len(sliced) - 1 - j)) & 1 for j in range(len(sliced))]
        labs, dat = slice_network(tn.labels, tn.data, list(tn.open_labels) + sliced, list(w.outputs[0]) + digits)
        _, t = contract_network(labs, dat, path)
        parts.append(complex(t))
        print(f"slice {i}: {parts[-1]}", flush=True)
    t_sl = time.time() - t0
    rec = {
        "workload": "grid53", "source": "oracle O2 (pairwise numpy.tensordot) along the oracle's own path and slicing",
        "outputs": w.outputs.tolist(), "path": [list(map(int, p)) for p in path],
        "path_flop": float(f), "sliced_labels": [int(x) for x in sliced],
        "flop_per_slice": float(network_flops(tn.labels, d2, path)),
        "slice_ids": ids, "slice_partials": [[p.real, p.imag] for p in parts],
        "seconds": {"planning": round(t_plan, 1), "slices": round(t_sl, 1)},
    }
    with open(os.path.join(HERE, "grid53.json"), "w") as fh:
        json.dump(rec, fh)
    print(json.dumps(rec["seconds"]))


def grid53_bench():
    from oracle.einsum import slice_network, contract_network
    from circuits import SplitMix64
    w = configs.build("grid53")
    tn = w.network.as_complex64()
    plan = json.load(open(os.path.join(HERE, "grid53_plan.json")))
    path = [tuple(p) for p in plan["path"]]
    sliced = plan["sliced_labels"]
    n = len(sliced)
    # Case selection (no expected value comes from it): with the bras' digits
    # and a slice's digits fixed, a tensor whose remaining sub-tensor is all
    # zero makes that slice's partial exactly zero (here: fSim's zero entries
    # between states of different Hamming weight, next to the bras).  Half of
    # the 4096 slices are such.  Take 8 seeded slices that no tensor zeroes and
    # 2 that one does (their partial must come out exactly zero).
    fixed0 = dict(zip(tn.open_labels, map(int, w.outputs[0])))
    touch = [ti for ti, l in enumerate(tn.labels) if any(x in fixed0 or x in sliced for x in l)]

    def zeroed(sid):
        fx = dict(fixed0)
        fx.update(zip(sliced, [(sid >> (n - 1 - j)) & 1 for j in range(n)]))
        for ti in touch:
            idx = tuple(fx[x] if x in fx else slice(None) for x in tn.labels[ti])
            if not np.any(np.asarray(tn.data[ti])[idx]):
                return True
        return False
    rng = SplitMix64(5353)
    ids, n_zero = [], 0
    while len(ids) < 10:
        i = int(rng.next_u64() % (1 << n))
        if i in ids:
            continue
        z = zeroed(i)
        if z and n_zero < 2:
            ids.append(i)
            n_zero += 1
        elif not z and len(ids) - n_zero < 8:
            ids.append(i)
    ids.sort()
    zero_ids = [i for i in ids if zeroed(i)]
    parts, secs = [], []
    for i in ids:
        digits = [(i >> (n - 1 - j)) & 1 for j in range(n)]
        t0 = time.time()
        # the bra <x| on each open leg fixes that leg to its digit (Section 2.2.1),
        # exactly like a sliced label (Section 2.4)
        sl, sd = slice_network(tn.labels, tn.data, list(tn.open_labels) + sliced, list(w.outputs[0]) + digits)
        _, t = contract_network(sl, sd, path)
        parts.append(complex(t))
        secs.append(time.time() - t0)
        print(f"slice {i}: {parts[-1]} ({secs[-1]:.1f} s)", flush=True)
    rec = {
        "workload": "grid53", "source": "oracle O2 (pairwise numpy.tensordot) along the benchmark's order and "
                                        "sliced labels (tests/golden/grid53_plan.json, read as data)",
        "outputs": w.outputs.tolist(), "sliced_labels": [int(x) for x in sliced],
        "slice_ids": ids, "slice_digits": [[(i >> (n - 1 - j)) & 1 for j in range(n)] for i in ids],
        "structurally_zero_ids": zero_ids,
        "slice_partials": [[p.real, p.imag] for p in parts],
        "seconds": {"slices": round(sum(secs), 1)},
    }
    with open(os.path.join(HERE, "grid53_bench.json"), "w") as fh:
        json.dump(rec, fh, indent=1)
    print(json.dumps(rec["seconds"]))


if __name__ == "__main__":
    which = sys.argv[1:] or ["grid30"]
    for name in which:
        {"grid30": grid30, "gbs16": gbs16, "grid53": grid53, "grid53_bench": grid53_bench}[name]()
