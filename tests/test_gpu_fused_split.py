"""A tensor-core GEMM whose output is the large operand of the next GEMM
writes that GEMM's FP16 operand planes and chunk scales from its epilogue
(fused split) instead of complex64 followed by an operand split (Section 3.1:
the transpose in front of the next multiplication).

Network X[a, k] Y[k, b] -> C1[a, b] (GEMM), then C1 Z -> C2 summing labels from
both of C1's sides (4 of a, 2 of b), every output leg of C2 left free, FP16x3.
The plan must take the fused form (the first GEMM marked, no operand split of
C1), and C2 is compared with the oracle's pairwise steps element by element:
max |C2 - ref| / max |ref| <= 1e-5.  The same network with sliced labels on X
and Z (instance blocks on both GEMMs) takes the grouped form."""
import numpy as np
import pytest

from circuits import SplitMix64
from oracle.einsum import contract_network, slice_network
from paper_2107_09793_b300 import jet

A_L = list(range(100, 110))     # C1's rows (10 labels); 106..109 are summed by the second GEMM
K_L = list(range(200, 206))     # X . Y summed labels
B_L = list(range(300, 307))     # C1's columns (7 labels); 305, 306 are summed by the second GEMM
C_L = list(range(400, 407))     # Z's free labels


def _rand(rng, shape):
    n = int(np.prod(shape))
    re = np.array([rng.uniform() - 0.5 for _ in range(n)])
    im = np.array([rng.uniform() - 0.5 for _ in range(n)])
    return (re + 1j * im).reshape(shape).astype(np.complex64)


def _network(sliced):
    rng = SplitMix64(2024)
    xs, zs = ([500], [501]) if sliced else ([], [])
    lx = xs + A_L + K_L
    ly = K_L + B_L
    lz = A_L[6:] + B_L[5:] + C_L + zs
    labels, data = [lx, ly, lz], [_rand(rng, [2] * len(l)) for l in (lx, ly, lz)]
    if sliced:   # a rank-2 tensor joins the sliced labels after the pair
        labels.append(xs + zs)
        data.append(_rand(rng, [2, 2]))
    opens = A_L[:6] + B_L[:5] + C_L
    return labels, data, opens, xs + zs


def plan_network(sliced, prec="fp16x3", fuse=True):
    labels, data, opens, sl = _network(sliced)
    net = jet.Network(labels, data, precision=prec, profile=2, fuse_split=fuse)
    net.set_open(opens)
    net.set_free(opens)
    path = [(0, 1), (4, 2), (5, 3)] if sliced else [(0, 1), (3, 2)]
    net.path_set(path)
    if sl:
        net.slice(sl)
    return net, labels, data, opens, sl, path


def _reference(labels, data, opens, sl, path):
    d64 = [t.astype(np.complex128) for t in data]
    if not sl:
        out, t = contract_network(labels, d64, path)
        return out, np.asarray(t)
    acc = None
    for s in range(2 ** len(sl)):
        vals = [(s >> (len(sl) - 1 - j)) & 1 for j in range(len(sl))]
        sll, sd = slice_network(labels, d64, sl, vals)
        out, t = contract_network(sll, sd, path)
        acc = np.asarray(t) if acc is None else acc + np.asarray(t)
    return out, acc


@pytest.mark.gpu
@pytest.mark.parametrize("sliced", [False, True])
def test_fused_split_matches_the_oracle_element_by_element(sliced):
    net, labels, data, opens, sl, path = plan_network(sliced)
    try:
        outs = np.zeros((1, len(opens)), np.int32)   # (every open leg is free: values unused)
        got = net.contract(outs)[0]
        recs = net.profile()
    finally:
        net.close()
    prod, cons = (4, 5) if sliced else (3, 4)   # the producer GEMM's node, its parent's
    first = [r for r in recs if r["kind"] == "gemm_tc" and r["node"] == prod]
    assert first and all(r["variant"] & 4 for r in first), recs
    # the parent splits only its small operand
    assert [r for r in recs if r["kind"] == "gemm_tc" and r["node"] == cons], recs
    assert all(r["bytes"] < 1e6 for r in recs if r["kind"] == "tc_split" and r["node"] == cons), recs
    out, ref = _reference(labels, data, opens, sl, path)
    # the library returns C2 in the order of its free legs (opens); the oracle in its own
    ref = np.transpose(ref, [out.index(l) for l in opens]).ravel()
    got = np.asarray(got).ravel()
    assert got.shape == ref.shape
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    print(f"fused split (sliced={sliced}): max elementwise err {err:.2e}")
    assert err <= 1e-5


@pytest.mark.gpu
@pytest.mark.parametrize("sliced", [False, True])
def test_fused_planes_equal_the_split_bit_for_bit(sliced):
    """The fused epilogue writes the planes and scales the operand split would
    (same chunk maxima, exponents and roundings), so C2 is bitwise the same
    with jet_options.fuse_split = 0."""
    outs = None
    got = []
    for fuse in (True, False):
        net, labels, data, opens, sl, path = plan_network(sliced, fuse=fuse)
        try:
            outs = np.zeros((1, len(opens)), np.int32)
            got.append(np.asarray(net.contract(outs)[0]).copy())
            fused = any(r["kind"] == "gemm_tc" and r["variant"] & 4 for r in net.profile())
        finally:
            net.close()
        assert fused == fuse
    assert np.array_equal(got[0], got[1])
