"""The 16-mode 4x4 bosonic lattice (Fock cutoff 4, 4 layers of beamsplitters,
16 squeezed-vacuum inputs; Section 4, Algorithm 1) at full size, contracted as
one batch of 256 seeded photon patterns in the benchmark's configuration: the
batch planner (seed 1, 8 trials, weighted cap 2^32 elements), which keeps the
bras late so the whole network up to the last layer is shared by the batch.

Checks: the stored FP64 amplitudes of the batch's 8 smallest even-total
patterns (tests/golden/gbs16.json, written by tests/golden/make_golden.py from
the per-sector state vector), exact zeros for every odd total (squeezers emit
photon pairs and beamsplitters conserve the photon number), and a second batch
of low-total patterns (the vacuum among them) against the sector oracle live."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from circuits import configs, Circuit, Gate
from circuits.rng import SplitMix64
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "gbs16.json")))


def rounded(circ):
    return Circuit(n=circ.n, d=circ.d,
                   gates=[Gate(np.asarray(g.matrix, np.complex64).astype(np.complex128), g.qubits, g.params, g.kind)
                          for g in circ.gates],
                   initial=[np.asarray(v, np.complex64).astype(np.complex128) for v in circ.initial])


@pytest.fixture(scope="module")
def gbs_path():
    w = configs.build("gbs16")
    net = jet.from_network(w.network)
    net.path_greedy_batch(w.outputs, seed=1, n_trials=8, max_elems=1 << 32)
    return w, net.path_get()


def test_gbs16_batch_vs_sector_statevector(gbs_path):
    w, path = gbs_path
    net = jet.from_network(w.network)
    net.path_set(path)
    amps = net.contract(w.outputs)
    tot = w.outputs.sum(axis=1)
    odd = tot % 2 == 1
    assert odd.sum() > 64
    assert np.all(amps[odd] == 0)
    idx = GOLDEN["batch_index"]
    ref = np.array([complex(a, b) for a, b in GOLDEN["amplitudes"]])
    got = amps[idx]
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    per = np.abs(got - ref) / np.abs(ref)
    print(f"gbs16: normwise rel err {err:.3e}, per-amplitude max {per.max():.3e}")
    assert err <= 1e-5
    net.close()


def _low_total_patterns(count, seed):
    """Seeded patterns with an even total of at most 6 photons (vacuum first)."""
    rng = SplitMix64(seed)
    pats = [[0] * 16]
    while len(pats) < count:
        total = 2 * (1 + int(rng.uniform() * 3))
        p = [0] * 16
        left = total
        while left:
            k = int(rng.uniform() * 16)
            if p[k] < 3:
                p[k] += 1
                left -= 1
        pats.append(p)
    return np.array(pats, np.int32)


def test_gbs16_low_totals_vs_sector_oracle(gbs_path):
    w, path = gbs_path
    pats = _low_total_patterns(16, 77)
    net = jet.from_network(w.network)
    net.path_set(path)
    got = net.contract(pats)
    ref = oracle.sector_amplitudes(rounded(w.circuit), pats)
    vac = np.prod([1 / math.sqrt(math.cosh(r)) for r in w.circuit.squeezing])
    assert abs(ref[0] - vac) <= 1e-7 * vac     # complex64-rounded inputs
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    print(f"gbs16 low totals: normwise rel err {err:.3e}")
    assert err <= 1e-5
    net.close()
