"""The autotuner (jet_autotune): per tree node, the faster of two kernel forms
that both take the node's shape (GEMM instance blocks or one product per
instance; tensor-core or CUDA-core small-operand application), timed on the
device.  The tuned plan must still match the stored FP64 state-vector
amplitude, must not be slower than the defaults by more than the tuner's
margin, and a second handle reading the tuner's cache must take the same
choices without timing them (bit-identical amplitudes)."""
import json
import os

import numpy as np
import pytest

from circuits import configs
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "grid30.json")


def _net(w, path=None, sliced=None):
    net = jet.from_network(w.network, precision="tf32x3")
    if path is None:
        net.path_greedy(seed=1, n_trials=64)
        sliced = net.slice_auto(1 << 24, min_n=6, max_n=24)
    else:
        net.path_set(path)
        net.slice(sliced)
    return net, net.path_get(), sliced


def test_autotuned_plan_matches_the_oracle_and_its_cache(tmp_path):
    g = json.load(open(GOLDEN))
    w = configs.build("grid30")
    rows = np.array(g["outputs"][:1], np.int32)
    ref = complex(*g["amplitudes"][0])
    cache = str(tmp_path / "tune.txt")
    net, path, sliced = _net(w)
    try:
        base = net.contract(rows)[0]
        t = net.autotune(rows, cache_file=cache)
        assert t["default_ms"] > 0 and t["tuned_ms"] <= 1.02 * t["default_ms"], t
        tuned = net.contract(rows)[0]
        print(f"autotune grid30: {t}")
    finally:
        net.close()
    assert abs(tuned - ref) / abs(ref) <= 1e-5 and abs(base - ref) / abs(ref) <= 1e-5
    assert os.path.getsize(cache) > 0
    net2, _, _ = _net(w, path, sliced)
    try:
        t2 = net2.autotune(rows, cache_file=cache)    # every shape cached: nothing timed twice
        again = net2.contract(rows)[0]
    finally:
        net2.close()
    assert t2["n_changed"] == t["n_changed"]
    assert again == tuned
