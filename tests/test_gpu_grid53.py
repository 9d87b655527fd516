"""The 53-qubit 9x6-minus-corner grid circuit (12 cycles) at full size: slice
partials s_i (Section 2.4, Eq. sliced_sum) of the workload amplitude on the GPU
against the FP64 oracle's pairwise contraction of the same slices, each
partial checked against its own magnitude.

Two stored sets (tests/golden/, written by make_golden.py, which calls only the
oracle):
  * grid53_bench.json: along the order and the 12 sliced labels the benchmark
    contracts (tests/golden/grid53_plan.json), 8 seeded slices that no tensor
    zeroes and 2 that one does (with the bras' digits and the slice's digits
    fixed, an fSim gate next to the bras keeps an all-zero sub-tensor: the
    partial is exactly zero);
  * grid53.json: along the oracle's own order and its own 17 sliced labels,
    8 seeded slices (3 exactly zero, 4 below 1e-25 from fSim(pi/2)'s cos entry
    of 6e-17, one of typical size).

Tolerances per mode, from the arithmetic (u = unit roundoff of an operand
entry's representation; complex64 intermediates accumulate in FP32): normwise
over the nonzero partials (the metric's bar, relative error <= 1e-5 for the
complex64 modes), and per partial against its own magnitude, looser where a
partial is a cancelling sum of larger terms:
  fp32: u = 2^-24; 1e-5 both ways;
  tf32x3, fp16x3, bf16x6: the tensor-core small-operand applications of every
      split mode use TF32 hi + lo, 22 significant bits, u = 2^-22 (4x FP32's
      operand error, then FP32 accumulation); normwise 1e-5, per partial 3e-5;
  bf16x3: hi + lo in BF16 keeps 16 significant bits, u = 2^-17 = 7.6e-6 per
      operand entry of the GEMMs, over the path's dependent steps: 2e-4 / 5e-4;
  tf32: one TF32 product, u = 2^-11 = 4.9e-4 per operand entry: 2e-2 / 5e-2
      (it fails the 1e-5 bar on purpose and is reported for comparison);
  fp64: 1e-12 both ways (complex128 everywhere, FP64 on CUDA cores)."""
import json
import os

import numpy as np
import pytest

from circuits import configs
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu

HERE = os.path.join(os.path.dirname(__file__), "golden")
TOL_NORM = {"fp32": 1e-5, "tf32x3": 1e-5, "fp16x3": 1e-5, "bf16x6": 1e-5, "bf16x3": 2e-4, "tf32": 2e-2, "fp64": 1e-12}
TOL_SLICE = {"fp32": 1e-5, "tf32x3": 3e-5, "fp16x3": 3e-5, "bf16x6": 3e-5, "bf16x3": 5e-4, "tf32": 5e-2, "fp64": 1e-12}


def _load(name):
    p = os.path.join(HERE, name)
    if not os.path.exists(p):
        pytest.fail(f"tests/golden/{name} missing: run tests/golden/make_golden.py")
    return json.load(open(p))


@pytest.fixture(scope="module")
def workload():
    return configs.build("grid53")


def _check_partials(got, ref, zero_ids, ids, prec):
    """Normwise over the partials that are not structurally zero, each of them
    against its own magnitude, and a structurally zero partial exactly zero."""
    big = np.max(np.abs(ref))
    nz = np.array([i not in zero_ids for i in ids])
    norm = float(np.linalg.norm(got[nz] - ref[nz]) / np.linalg.norm(ref[nz]))
    worst = 0.0
    for g, r, i in zip(got, ref, ids):
        if i in zero_ids:
            assert r == 0 and g == 0, (prec, i, g, r)
        elif abs(r) >= 1e-3 * big:
            e = abs(g - r) / abs(r)
            worst = max(worst, e)
            assert e <= TOL_SLICE[prec], (prec, i, e)
        else:   # partials far below the amplitude's scale: at that scale
            assert abs(g - r) <= TOL_SLICE[prec] * big, (prec, i, g, r)
    assert norm <= TOL_NORM[prec], (prec, norm)
    return norm, worst


def _partials(w, prec, path, sliced, outputs, ids):
    net = jet.from_network(w.network, precision=prec)
    try:
        net.path_set([tuple(p) for p in path])
        net.slice(sliced)
        assert net.stats()["max_intermediate"] <= 1 << 28
        return net.contract_slices(np.array(outputs, np.int32), ids)[0]
    finally:
        net.close()


@pytest.mark.parametrize("prec", ["tf32x3", "fp32", "bf16x3", "tf32", "fp16x3", "bf16x6", "fp64"])
def test_grid53_benchmark_plan_slice_partials(workload, prec):
    plan = _load("grid53_plan.json")
    g = _load("grid53_bench.json")
    assert g["sliced_labels"] == plan["sliced_labels"]
    got = _partials(workload, prec, plan["path"], plan["sliced_labels"], g["outputs"], g["slice_ids"])
    ref = np.array([complex(a, b) for a, b in g["slice_partials"]])
    norm, worst = _check_partials(got, ref, set(g["structurally_zero_ids"]), g["slice_ids"], prec)
    print(f"grid53 benchmark plan {prec}: normwise {norm:.3e}, worst per-slice {worst:.3e} over "
          f"{len(ref) - len(g['structurally_zero_ids'])} slices")


@pytest.mark.parametrize("prec", ["tf32x3", "fp32", "fp16x3"])
def test_grid53_oracle_plan_slice_partials(workload, prec):
    g = _load("grid53.json")
    got = _partials(workload, prec, g["path"], g["sliced_labels"], g["outputs"], g["slice_ids"])
    ref = np.array([complex(a, b) for a, b in g["slice_partials"]])
    zero = {i for i, r in zip(g["slice_ids"], ref) if r == 0}
    norm, worst = _check_partials(got, ref, zero, g["slice_ids"], prec)
    print(f"grid53 oracle plan {prec}: normwise {norm:.3e}, worst per-slice {worst:.3e}")
