"""GEMM route of a pairwise contraction (Section 3.1: transpose, transpose,
matrix multiply) vs the oracle's pairwise step, for every operand layout the
plan compiler distinguishes ([free, K], [K, free], interleaved -> permute),
ragged sizes and batched instances, in every precision mode.

The pair is the whole network, every output leg left free
(jet_network_set_free), so one contraction returns all of C; it is compared
with the oracle element by element: max |C - C_ref| / max |C_ref| <= the
mode's tolerance (a wrong tile or ragged edge shows at its own size)."""
import numpy as np
import pytest

from circuits import SplitMix64
from oracle.einsum import _pair, contract_network
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12, "tf32x3": 1e-5, "bf16x3": 1e-5, "bf16x6": 1e-5, "fp16x3": 1e-5, "tf32": 3e-3}


def _rand(rng, shape):
    n = int(np.prod(shape))
    re = np.array([rng.uniform() - 0.5 for _ in range(n)])
    im = np.array([rng.uniform() - 0.5 for _ in range(n)])
    return (re + 1j * im).reshape(shape).astype(np.complex64)


def _pair_network(la, lb, dims, seed, prec, **opt):
    rng = SplitMix64(seed)
    A = _rand(rng, [dims[l] for l in la])
    B = _rand(rng, [dims[l] for l in lb])
    opens = [l for l in la if l not in lb] + [l for l in lb if l not in la]
    net = jet.Network([la, lb], [A, B], precision=prec, **opt)
    net.set_open(opens)
    net.set_free(opens)
    net.path_set([(0, 1)])
    return net, A, B


def _elementwise_err(got, la, A, lb, B):
    _, ref = _pair(list(la), A.astype(np.complex128), list(lb), B.astype(np.complex128))
    ref = np.asarray(ref).ravel()
    assert got.shape == ref.shape
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


CASES = [
    # (labels A, labels B, dims) - K-major A, K-major B
    ([0, 1, 2, 3, 4, 5, 6, 10, 11, 12, 13, 14, 15], [20, 21, 22, 23, 24, 25, 10, 11, 12, 13, 14, 15], {}),
    # [K, free] A, [K, free] B
    ([10, 11, 12, 13, 14, 15, 0, 1, 2, 3, 4, 5, 6], [10, 11, 12, 13, 14, 15, 20, 21, 22, 23, 24, 25], {}),
    # interleaved: both need a permute; K in different orders
    ([0, 10, 1, 11, 2, 12, 3, 13, 4, 14, 5, 15, 6], [15, 20, 14, 21, 13, 22, 12, 23, 11, 24, 10, 25], {}),
    # ragged: dims 3 and 5 (M, N, K not multiples of the tiles)
    ([0, 1, 2, 3, 10, 11, 12], [10, 11, 12, 20, 21, 22], {0: 3, 1: 5, 2: 3, 3: 3, 10: 5, 11: 3, 12: 5,
                                                        20: 5, 21: 3, 22: 5}),
    # several 128x128 tiles and 16+ K-blocks (wraps the tensor-core stage ring)
    (list(range(0, 8)) + list(range(10, 19)), list(range(10, 19)) + list(range(20, 28)), {}),
]


@pytest.mark.parametrize("prec", ["fp32", "fp64", "tf32", "tf32x3", "bf16x3", "bf16x6", "fp16x3"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_gemm_layouts(prec, case):
    la, lb, dd = CASES[case]
    dims = {l: dd.get(l, 2) for l in la + lb}
    net, A, B = _pair_network(la, lb, dims, 31 + case, prec)
    try:
        got = net.contract(np.zeros((1, len(la) + len(lb) - 2 * len(set(la) & set(lb))), np.int32))[0]
        assert net.stats()["n_gemm_nodes"] >= 1
    finally:
        net.close()
    err = _elementwise_err(got, la, A, lb, B)
    print(f"gemm case {case} {prec}: max elementwise err {err:.3e}")
    assert err <= TOL[prec], err


def test_gemm_batched_instances_under_slicing():
    """The same GEMM node instanced per slice value (reuse DAG) in one launch;
    every value of the free legs compared with the oracle."""
    la = [0, 1, 2, 3, 4, 5, 6, 10, 11, 12, 13, 14, 15, 30]
    lb = [10, 11, 12, 13, 14, 15, 20, 21, 22, 23, 24, 25, 31]
    rng = SplitMix64(5)
    A = _rand(rng, [2] * len(la))
    B = _rand(rng, [2] * len(lb))
    C = _rand(rng, [2, 2])   # joins 30 and 31 so both can be sliced as closed labels
    opens = [l for l in la if l not in lb and l != 30] + [l for l in lb if l not in la and l != 31]
    net = jet.Network([la, lb, [30, 31]], [A, B, C])
    net.set_open(opens)
    net.set_free(opens)
    net.path_set([(0, 1), (3, 2)])
    net.slice([30, 31])
    got = net.contract(np.zeros((1, len(opens)), np.int32))[0]
    assert net.stats()["n_gemm_nodes"] >= 1
    out, ref = contract_network([la, lb, [30, 31]], [A, B, C], [(0, 1), (3, 2)])
    ref = np.transpose(np.asarray(ref), [out.index(l) for l in opens]).ravel()
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    net.close()
    assert err <= 1e-5, err


# Grouped instance blocks: the instances of a GEMM node that pair every
# instance of one operand with the same instances of the other run as one wider
# product (rows j * M + m, columns l * N + n).  The sliced labels s* sit on one
# operand each (a full product of instances), x on both (instances pair only
# when x agrees: two blocks); the small tensors joining them are absorbed after
# the pair, and every free value is compared with the oracle.
GROUPED = {
    # M = 64 per instance, 2 x 2 instances: one block of 128 x 512
    "m64_2x2": (list(range(0, 6)) + list(range(10, 17)) + [40], list(range(10, 17)) + list(range(20, 28)) + [41],
                [[40, 41]], [40, 41]),
    # N = 32 per instance (a skinny side filling a quarter of a tile), 4 x 2 instances
    "n32_4x2": (list(range(0, 12)) + list(range(10 + 20, 18 + 20)) + [40, 42],
                list(range(30, 38)) + list(range(20, 25)) + [41], [[40, 41], [42]], [40, 41, 42]),
    # a sliced label x (50) on both operands: 2 blocks of 2 x 2
    "shared_x": (list(range(0, 7)) + list(range(10, 17)) + [50, 40], list(range(10, 17)) + list(range(20, 27)) + [50, 41],
                 [[40, 41]], [50, 40, 41]),
}


@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3", "bf16x6", "tf32"])
@pytest.mark.parametrize("case", sorted(GROUPED))
def test_gemm_grouped_instance_blocks(prec, case):
    la, lb, extra, sliced = GROUPED[case]
    rng = SplitMix64(77 + sorted(GROUPED).index(case))
    A = _rand(rng, [2] * len(la))
    B = _rand(rng, [2] * len(lb))
    X = [_rand(rng, [2] * len(e)) for e in extra]
    labels = [la, lb] + extra
    opens = [l for l in la if l not in lb and not any(l in e for e in extra)] + \
            [l for l in lb if l not in la and not any(l in e for e in extra)]
    net = jet.Network(labels, [A, B] + X, precision=prec, profile=2)
    try:
        net.set_open(opens)
        net.set_free(opens)
        path = [(0, 1)]
        cur = len(labels)
        for i in range(2, len(labels)):
            path.append((cur, i))
            cur += 1
        net.path_set(path)
        net.slice(sliced)
        got = net.contract(np.zeros((1, len(opens)), np.int32))[0]
        gem = [r for r in net.profile() if r["kind"] == "gemm_tc" and r["node"] == len(labels)]
    finally:
        net.close()
    assert gem and all(r["variant"] & 1 for r in gem), gem   # the pair ran as grouped blocks
    out, ref = contract_network(labels, [A, B] + X, path)
    ref = np.transpose(np.asarray(ref), [out.index(l) for l in opens]).ravel()
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    print(f"grouped {case} {prec}: max elementwise err {err:.3e}")
    assert err <= TOL[prec], err
