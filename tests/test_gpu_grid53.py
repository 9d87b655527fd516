"""The 53-qubit 9x6-minus-corner grid circuit (12 cycles) at full size: slices
of the workload amplitude contracted on the GPU along the oracle's own
contraction order and sliced labels (largest intermediate <= 2^28 elements,
2^17 slices), against the FP64 pairwise contraction of the same 8 seeded
slices stored in tests/golden/grid53.json (written by
tests/golden/make_golden.py).  The 2^17-slice sum itself is far too long to run
here; the benchmark reports the per-slice time and the measured fraction."""
import json
import os

import numpy as np
import pytest

from circuits import configs
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu

GOLDEN_PATH = os.path.join(os.path.dirname(__file__), "golden", "grid53.json")


@pytest.fixture(scope="module")
def golden():
    if not os.path.exists(GOLDEN_PATH):
        pytest.fail("tests/golden/grid53.json missing: run tests/golden/make_golden.py grid53")
    return json.load(open(GOLDEN_PATH))


# Normwise over the 8 partials (they span many orders of magnitude; the norm
# is set by the largest).  FP32 and the 3-way-accurate splits: 1e-5.
@pytest.mark.parametrize("prec,tol", [("fp16x3", 1e-5), ("fp32", 1e-5)])
def test_grid53_slice_partials_vs_pairwise_oracle(golden, prec, tol):
    w = configs.build("grid53")
    net = jet.from_network(w.network, precision=prec)
    net.path_set([tuple(p) for p in golden["path"]])
    net.slice(golden["sliced_labels"])
    st = net.stats()
    assert st["max_intermediate"] <= 1 << 28
    got = net.contract_slices(np.array(golden["outputs"], np.int32), golden["slice_ids"])[0]
    ref = np.array([complex(a, b) for a, b in golden["slice_partials"]])
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    print(f"grid53 {prec}: normwise rel err over {len(ref)} slices {err:.3e}")
    assert err <= tol
    net.close()
