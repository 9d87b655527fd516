"""Slice sharding on one GPU: the ranks' slice ranges contracted one after the
other through jet_contract_slices (no collective; the multi-process gather is
covered by tests/test_shard_gloo.py) and summed in increasing slice id give the
same bits as jet_contract, for 1, 2 and 3 ranks."""
import numpy as np
import pytest

from circuits import random_grid_circuit, circuit_to_network, random_bitstrings
from paper_2107_09793_b300 import jet
from paper_2107_09793_b300.shard import slice_ranges, ordered_sum

pytestmark = pytest.mark.gpu


def test_sharded_slices_equal_single_contraction_bitwise():
    circ = random_grid_circuit(3, 4, 8, seed=71)
    tn = circuit_to_network(circ)
    outs = random_bitstrings(12, 3, 72)
    net = jet.from_network(tn, precision="fp32")
    net.path_greedy(seed=1, n_trials=8)
    net.slice_auto(1 << 6, min_n=4, max_n=16)
    n_sl = net.stats()["n_slices"]
    assert n_sl >= 16
    ref = net.contract(outs)
    for world in (1, 2, 3):
        ranges = slice_ranges(n_sl, world)
        parts = [net.contract_slices(outs, list(range(a, b))) for a, b in ranges]
        got = ordered_sum(parts, ranges)
        assert got.tobytes() == ref.tobytes()
