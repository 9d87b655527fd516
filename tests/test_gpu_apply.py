"""Small-operand application route (Section 2.3, one pairwise step in the shape
of a gate absorbed into a large state-like tensor): C[r, f] = sum_q B[f, q] A[r, q]
vs the oracle's pairwise contraction, in the tensor-core form (split modes:
TF32 hi + lo, three products; one in plain TF32) and on CUDA cores (FP32 mode,
and the split modes with the tensor-core form switched off).

Shapes cover: one chunk of 32 summed entries with a ragged, non-power-of-two
fiber count; summed and free extents that are not multiples of the 8-entry
blocks (21 x 5, 200 x 3); several chunks per tile (128 and 200 summed entries,
the FP32 register promotion); wide free extents (32, 48 and 64: N = 64, 96 and
128 real columns, the last two with 128 TMEM columns per thread group; 16 x 64
has both free sides of 64 or more, a product the GEMM route would otherwise
take; 72 and 128 free entries with 20 and 32 summed: N up to 256, the chunk
staged in two halves; 128 x 32 and 144 x 24, whose operand planes leave room
only for half chunks: 8 and 9 halves, promoted in pairs); a summed label at
stride 1 in A (fibers at stride 2); and a sliced
summed label, so the node runs as two instances in one launch (the small
operand is rebuilt per instance).  The fast_ cases put the 7 fastest labels of A
on the fibers (one of them reading a leaf that is 8- but not 16-byte aligned).
The tensor-core form is forced on every shape (apply_tc_min_kf=1); the default
routing is checked separately.

The pair is the whole network (plus, for the unaligned case, a 3-entry leaf
joined last by an outer product) and every output leg is left free
(jet_network_set_free), so one contraction returns all of C; it is compared
with the oracle's pairwise contraction element by element:
max |C - C_ref| / max |C_ref| <= the mode's tolerance."""
import numpy as np
import pytest

from circuits.rng import uniform_array
from oracle.einsum import contract_network
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "tf32x3": 1e-5, "bf16x3": 1e-5, "bf16x6": 1e-5, "fp16x3": 1e-5, "tf32": 3e-3}


def _rand(seed, shape):
    n = int(np.prod(shape))
    u = uniform_array(seed, 2 * n)
    return ((u[:n] - 0.5) + 1j * (u[n:] - 0.5)).reshape(shape).astype(np.complex64)


# (labels of A, labels of B, dims, sliced labels); A is the large operand
CASES = {
    # 32 summed (4 x 8) interleaved with the fibers, 16 free; fibers 64 * 32 * 17
    "k32_f16_ragged_fibers": ([10, 0, 11, 1, 2], [20, 10, 11], {0: 64, 1: 32, 2: 17, 10: 4, 11: 8, 20: 16}, []),
    # 21 summed (3 x 7), 5 free, 2^15 fibers, summed labels slowest in A
    "k21_f5": ([10, 11] + list(range(100, 115)), [11, 20, 10], {10: 3, 11: 7, 20: 5}, []),
    # 128 summed over 7 binary labels (4 chunks), 16 free (4 x 4)
    "k128_f16_chunks": ([0] + list(range(10, 17)) + [1], list(range(10, 17)) + [20, 21],
                        {0: 128, 1: 256, 20: 4, 21: 4}, []),
    # 200 summed (8 x 25: 7 chunks, the last one block of 8), 3 free, fibers 33 * 31 * 33
    "k200_f3_chunks": ([0, 1, 2, 10, 11], [20, 11, 10], {0: 33, 1: 31, 2: 33, 10: 8, 11: 25, 20: 3}, []),
    # 16 summed in the middle of A, 32 free: N = 64 real columns
    "k16_f32": ([0, 10, 1], [10, 20], {0: 256, 1: 256, 10: 16, 20: 32}, []),
    # 16 summed, 64 free (N = 128 real columns, three groups); both free sides >= 64
    "k16_f64": ([0, 10, 1], [10, 20], {0: 256, 1: 256, 10: 16, 20: 64}, []),
    # 32 summed (4 x 8), 48 free (N = 96; the operand planes leave room for two groups)
    "k32_f48": ([0, 10, 11, 1], [11, 20, 10], {0: 128, 1: 256, 10: 4, 11: 8, 20: 48}, []),
    # wide: 32 summed, 128 free (N = 256; the chunk staged in two halves of 16)
    "k32_f128_wide": ([0, 10, 11, 1], [10, 20, 11], {0: 128, 1: 256, 10: 4, 11: 8, 20: 128}, []),
    # 128 summed x 32 free: the operand planes (128 KB) leave room only for half
    # chunks, 8 halves promoted in pairs
    "k128_f32_halves": ([0] + list(range(10, 17)) + [1], list(range(10, 17)) + [20], {0: 128, 1: 256, 20: 32}, []),
    # 144 summed (9 x 16) x 24 free: 9 halves, the last one promoted alone
    "k144_f24_halves": ([0, 10, 11, 1], [11, 20, 10], {0: 128, 1: 256, 10: 9, 11: 16, 20: 24}, []),
    # wide with a ragged summed extent (20: one half of 16, one of 4) and 72 free
    "k20_f72_wide": ([0, 10, 11, 1], [11, 20, 10], {0: 128, 1: 256, 10: 4, 11: 5, 20: 72}, []),
    # a summed binary label at stride 1 in A: the fibers sit at stride 2
    "k32_stride2": (list(range(100, 115)) + [10, 11, 12, 13, 14], [20, 10, 11, 12, 13, 14], {20: 8}, []),
    # 64 summed with one label sliced: the node runs as 2 instances of 32 summed
    "k32_two_instances": (list(range(100, 115)) + [10, 11, 12], [10, 11, 12, 20], {10: 4, 11: 8, 12: 2, 20: 8}, [12]),
    # the 7 fastest labels of A are fibers, 128 summed: 4 chunks
    "fast_k128_chunks": ([0] + list(range(10, 17)) + list(range(100, 107)), list(range(10, 17)) + [20, 21],
                       {0: 256, 20: 4, 21: 4}, []),
    # 2 instances (a sliced summed label above the fiber block)
    "fast_k32_two_instances": ([0, 10, 11, 12] + list(range(100, 107)), [12, 11, 10, 20],
                             {0: 256, 10: 4, 11: 8, 12: 2, 20: 16}, [12]),
    # A read from a leaf whose base is 8 but not 16-byte aligned (a 3-entry leaf
    # is stored first)
    "fast_k32_unaligned": ([0, 10, 11] + list(range(100, 107)), [11, 20, 10], {0: 256, 10: 4, 11: 8, 20: 12}, "lead"),
}


def _network(case, prec, **opt):
    la, lb, dd, sliced = CASES[case]
    lead = sliced == "lead"
    sliced = [] if lead else sliced
    dims = {l: dd.get(l, 2) for l in la + lb}
    seed = 1000 + 17 * sorted(CASES).index(case)
    A = _rand(seed, [dims[l] for l in la])
    B = _rand(seed + 1, [dims[l] for l in lb])
    labels, data = [la, lb], [A, B]
    opens = [l for l in la if l not in lb] + [l for l in lb if l not in la]
    path = [(0, 1)]
    if lead:   # a 3-entry leaf ahead of A in the leaf buffer, with an open leg of its own
        labels, data, opens = [[999]] + labels, [_rand(seed - 1, [3])] + data, opens + [999]
        path = [(1, 2), (3, 0)]
    net = jet.Network(labels, data, precision=prec, profile=1, **opt)
    net.set_open(opens)
    net.set_free(opens)
    net.path_set(path)
    if sliced:
        net.slice(sliced)
    return net, labels, data, opens, path


def _reference(labels, data, opens, path):
    out, t = contract_network([list(l) for l in labels], [d.astype(np.complex128) for d in data], path)
    return np.transpose(np.asarray(t), [out.index(l) for l in opens]).ravel()


_REF = {}


def _check(case, prec, expect_tc, **opt):
    net, labels, data, opens, path = _network(case, prec, **opt)
    try:
        got = net.contract(np.zeros((1, len(opens)), np.int32))[0]
        recs = net.profile()
    finally:
        net.close()
    pair = [r for r in recs if r["node"] == len(labels) and r["kind"] == "apply"]
    assert pair, "the pair did not take the small-operand route"
    assert all(bool(r["variant"] & 8) == expect_tc for r in pair), pair
    if case not in _REF:
        _REF[case] = _reference(labels, data, opens, path)
    ref = _REF[case]
    assert got.shape == ref.shape
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    print(f"{case} {prec} tc={expect_tc}: max elementwise err {err:.3e}")
    return err


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3"])
def test_apply_tensor_core_form(case, prec):
    assert _check(case, prec, True, apply_tc_min_kf=1) <= TOL[prec]


@pytest.mark.parametrize("case", ["k32_f16_ragged_fibers", "k128_f16_chunks", "k32_two_instances", "fast_k128_chunks"])
@pytest.mark.parametrize("prec", ["tf32", "bf16x3", "bf16x6"])
def test_apply_tensor_core_other_modes(case, prec):
    assert _check(case, prec, True, apply_tc_min_kf=1) <= TOL[prec]


# 32 x 48, 144 x 24 and the wide shapes are past the CUDA-core forms (held: 1024
# padded entries; streamed: 32 free, 4096 entries with the free ones padded to 16)
@pytest.mark.parametrize("case", sorted(set(CASES) - {"k32_f48", "k32_f128_wide", "k20_f72_wide", "k144_f24_halves"}))
def test_apply_cuda_core_forms(case):
    """FP32 mode, and a split mode with the tensor-core form switched off (the
    GEMM route too, which would take the 16 x 64 product)."""
    assert _check(case, "fp32", False, gemm_min_k=1 << 20) <= TOL["fp32"]
    assert _check(case, "fp16x3", False, apply_tc_min_kf=1 << 20, gemm_min_k=1 << 20) <= TOL["fp16x3"]


@pytest.mark.parametrize("case", sorted(CASES))
def test_apply_default_routing(case):
    """Default threshold: the tensor-core form for small operands of 1024
    entries or more (32 x 32, 128 x 16), and from 512 for one chunk of summed
    entries with nk nf >= 10 (nk + nf) (32 x 16, 16 x 32); the CUDA-core forms
    below."""
    la, lb, dd, sliced = CASES[case]
    sliced = [] if sliced == "lead" else sliced
    dims = {l: dd.get(l, 2) for l in la + lb}
    nk = int(np.prod([dims[l] for l in lb if l in la and l not in sliced]))   # one instance
    nf = int(np.prod([dims[l] for l in lb if l not in la]))
    tc = nk * nf >= 1024 or (nk <= 32 and 2 * nk * nf >= 1024 and nk * nf >= 10 * (nk + nf))
    assert _check(case, "fp16x3", tc) <= TOL["fp16x3"]


@pytest.mark.parametrize("prec", ["fp32", "fp16x3"])
def test_apply_instances_sharing_the_large_operand_run_together(prec):
    """A large operand without sliced labels and a small one with two sliced
    labels: the pair's 4 instances apply 4 small operands to one large one and
    run as one application of an operand 4 times wider (the large one read
    once).  Each output is the same sum as without the grouping (bit for bit),
    and every value matches the oracle."""
    r = list(range(16))
    k, f, s1, s2 = [100, 101], 102, 103, 104
    A = _rand(8100, [2] * (len(r) + 2))
    B = _rand(8101, [2, 2, 2, 2, 2])
    Y = _rand(8102, [2, 2])
    labels, data = [r + k, k + [f, s1, s2], [s1, s2]], [A, B, Y]
    opens = r + [f]
    got = {}
    for grp in (True, False):
        net = jet.Network(labels, data, precision=prec, profile=2, gemm_group=grp)
        try:
            net.set_open(opens)
            net.set_free(opens)
            net.path_set([(0, 1), (3, 2)])
            net.slice([s1, s2])
            got[grp] = net.contract(np.zeros((1, len(opens)), np.int32))[0]
            app = [x for x in net.profile() if x["kind"] == "apply" and x["node"] == 3]
        finally:
            net.close()
        assert len(app) == 1 and app[0]["n_inst"] == 4
        assert app[0]["grid"][1] == (1 if grp else 4), app   # one unit per large instance when grouped
    assert np.array_equal(got[True], got[False])
    out, ref = contract_network([list(l) for l in labels], [d.astype(np.complex128) for d in data], [(0, 1), (3, 2)])
    ref = np.transpose(np.asarray(ref), [out.index(l) for l in opens]).ravel()
    err = float(np.max(np.abs(got[True] - ref)) / np.max(np.abs(ref)))
    assert err <= 1e-5, err
