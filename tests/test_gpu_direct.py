"""Direct pairwise contraction with few outputs and a long summed index
(Section 2.3; the last steps of an amplitude's tree): the summed index is split
across blocks and the per-part partials are added in a second launch.  When
every group of 8 consecutive outputs is the outer product of NA values of A
(fastest) and 8 / NA of B, each operand value is read once per summed entry.

Two tensors A[a..., k...] and B[b..., k...] with 2^16 summed entries (16
binary labels, ordered differently in A and B) and every free leg left open.
Without a consumer the pair's output is laid out as the larger operand's free
labels, then the smaller one's (fastest), which fixes the pattern of each group
of 8 outputs:
- A's values fastest, NA = 2, 4, 8; all 8 from B (NA = 1);
- B's values fastest, NB = 2, 4;
- groups that straddle a dim-3 label (the generic form, 16 loads per summed
  entry);
- a free label of dim 3 (slowest) and two instances (one summed label sliced).
Checked against the oracle's contraction of the same pair, FP32 and FP64."""
import numpy as np
import pytest

from circuits.rng import uniform_array
from oracle.einsum import contract_network
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu

K = list(range(100, 116))   # 16 binary summed labels


def _rand(seed, shape):
    n = int(np.prod(shape))
    u = uniform_array(seed, 2 * n)
    return ((u[:n] - 0.5) + 1j * (u[n:] - 0.5)).reshape(shape)


# name: (A free labels, B free labels, dims, sliced, expected pattern)
CASES = {
    "a_fast_na2": ([1], [11, 12, 13], {}, [], 2),
    "a_fast_na4": ([1, 2], [11, 12, 13], {}, [], 4),
    "a_fast_na8": ([1, 2, 3], [11, 12, 13, 14], {}, [], 8),
    "b_only_na1": ([1, 2, 3, 4], [11, 12, 13], {}, [], 1),
    "b_fast_nb2": ([1, 2, 3], [11], {}, [], 18),
    "b_fast_nb4": ([1, 2, 3], [11, 12], {}, [], 20),
    "generic_dim3_fastest": ([1, 2, 3], [11], {11: 3}, [], 0),
    "dim3_slowest_two_instances": ([1, 2], [11, 12], {11: 3}, [K[5]], 4),
}


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("fp64", 1e-13)])
@pytest.mark.parametrize("case", sorted(CASES))
def test_split_k_forms(case, prec, tol):
    fa, fb, dd, sliced, na = CASES[case]
    dims = {l: dd.get(l, 2) for l in fa + fb + K}
    size = lambda f: int(np.prod([dims[l] for l in f]))
    order = fa + fb if size(fa) >= size(fb) else fb + fa    # the pair's own layout
    ka = list(K)
    kb = list(K[8:]) + list(K[:8])          # B reads the summed labels in another order
    la, lb = ka[:8] + fa + ka[8:], fb + kb
    seed = 5000 + 31 * sorted(CASES).index(case)
    A = _rand(seed, [dims[l] for l in la])
    B = _rand(seed + 1, [dims[l] for l in lb])
    A, B = A.astype(np.complex64), B.astype(np.complex64)   # leaves are complex64 in every mode
    net = jet.Network([la, lb], [A, B], precision=prec, profile=2)
    net.set_open(order)
    net.set_free(order)
    net.path_set([(0, 1)])
    if sliced:
        net.slice(sliced)
    got = net.contract(np.zeros((1, len(order)), np.int32))[0]
    recs = [r for r in net.profile() if r["kind"] == "direct"]
    assert len(recs) == 1 and recs[0]["variant"] & 2, recs        # the split form
    assert recs[0]["variant"] >> 8 == na, (recs[0]["variant"], recs[0]["grid"])
    assert recs[0]["n_inst"] == (2 if sliced else 1)
    rl, ref = contract_network([la, lb], [A.astype(np.complex128), B.astype(np.complex128)])
    ref = np.transpose(ref, [rl.index(l) for l in order]).reshape(-1)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"{case} {prec}: NA {na}, rel err {err:.2e}")
    assert err <= tol
    net.close()


# Dot products of instance blocks: A[x, y..., k...] and B[x, z, k...] with x, the
# y labels and z sliced (x on both operands, the y labels and z joined by Y
# after the pair).  The pair's instances (x, y..., z) form 2 blocks (x = 0, 1)
# of 2^len(y) A instances x 2 B instances; each block's dot products read every
# operand value once (2 x 2 blocks: the two-by-two form, with B staged in shared
# memory when the operands order the summed labels differently (FP32); 4 x 2:
# the general one).
@pytest.mark.parametrize("ny,crossed", [(1, True), (1, False), (2, True)])
@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("fp64", 1e-13)])
def test_split_k_instance_block_dot_products(prec, tol, ny, crossed):
    from oracle.einsum import slice_network
    form = 64 if ny == 2 else 66 if crossed and prec == "fp32" else 65
    x, z = 200, 202
    ys = list(range(210, 210 + ny))
    la, lb = [x] + ys + K[:8] + K[8:], [x, z] + (K[8:] + K[:8] if crossed else K[:8] + K[8:])
    A = _rand(7001 + ny, [2] * len(la)).astype(np.complex64)
    B = _rand(7002, [2] * len(lb)).astype(np.complex64)
    Y = _rand(7003 + ny, [2] * (ny + 1)).astype(np.complex64)
    labels, data = [la, lb, ys + [z]], [A, B, Y]
    sliced = [x] + ys + [z]
    n_sl = 2 ** len(sliced)
    net = jet.Network(labels, data, precision=prec, profile=2)
    try:
        net.set_open([])
        net.path_set([(0, 1), (3, 2)])
        net.slice(sliced)
        got = net.contract_slices(np.zeros((1, 0), np.int32), list(range(n_sl)))[0]
        recs = [r for r in net.profile() if r["kind"] == "direct" and r["node"] == 3]
    finally:
        net.close()
    assert len(recs) == 1 and recs[0]["variant"] >> 8 == form and recs[0]["grid"][2] == 2, recs
    d64 = [t.astype(np.complex128) for t in data]
    ref = []
    for s_ in range(n_sl):
        vals = [(s_ >> (len(sliced) - 1 - j)) & 1 for j in range(len(sliced))]
        sl, sd = slice_network(labels, d64, sliced, vals)
        ref.append(complex(contract_network(sl, sd, [(0, 1), (3, 2)])[1]))
    ref = np.array(ref)
    err = float(np.max(np.abs(got - ref) / np.abs(ref)))
    print(f"block dot products {prec} {form}: max per-slice rel err {err:.2e}")
    assert err <= tol
