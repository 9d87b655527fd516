"""A tensor-core GEMM whose output is contracted with its sibling over every
label (a dot product per instance, the last step of an amplitude: Eq.
sliced_sum's per-slice scalar) forms those dot products in its epilogue, per
128 x 128 tile, instead of writing its output; the parent only adds the tiles'
parts in a fixed order.

Network X[x, x', a, k] Y[k, b] -> C[x, x', a, b] (GEMM, 8192 x 256, K = 16: one
accumulator chunk per tile, many tiles per CTA), then C . D[y, b, a] over a and
b (D in another label order, so the sibling's offsets come from tables), then a
joiner J[x, y, x']; x, x' and y sliced, so each C instance pairs with two D
instances.  D runs along C's rows (its fastest labels are a's) or along its
columns (b's), the two ways the epilogue stages D.  The plan must take the dot
form (the GEMM marked, the parent a sum over tiles), and every slice's value is
compared with the oracle's pairwise steps: max |s - ref| / max |ref| <= 1e-5.
BF16x6, whose pipeline stages leave no room for the staging, keeps the plain
form with the same bound."""
import numpy as np
import pytest

from circuits import SplitMix64
from oracle.einsum import contract_network, slice_network
from paper_2107_09793_b300 import jet

A_L = list(range(100, 113))   # 8192 rows: 64 row tiles per instance
K_L = list(range(200, 204))   # 16 summed (one accumulator chunk per tile)
B_L = list(range(300, 308))   # 256 columns


def _rand(rng, shape):
    n = int(np.prod(shape))
    re = np.array([rng.uniform() - 0.5 for _ in range(n)])
    im = np.array([rng.uniform() - 0.5 for _ in range(n)])
    return (re + 1j * im).reshape(shape).astype(np.complex64)


def network(d_along="rows", form="pairs"):
    """form: "pairs" (x, x' on X, y on D: 4 C instances, each pairing both D
    instances, two to a dot block), "single" (no y: 4 C instances, one D
    instance, U = 8 staged units per step), "unpaired" (no x, x': one C
    instance pairing both D instances, alone in its block), "four" (y, y' on
    D: each C instance pairs four D instances, beyond the form's two)."""
    rng = SplitMix64(4242)
    xs = [] if form == "unpaired" else [500, 502]
    ys = [] if form == "single" else [501, 503] if form == "four" else [501]
    lx, ly = xs + A_L + K_L, K_L + B_L
    if d_along == "rows":
        ld = ys + B_L[::-1] + A_L[4:] + A_L[:4]
    else:
        ld = ys + A_L[::-1] + B_L[4:] + B_L[:4]
    lj = sorted(xs + ys)
    labels = [lx, ly, ld, lj]
    data = [_rand(rng, [2] * len(l)) for l in labels]
    path = [(0, 1), (4, 2), (5, 3)]
    return labels, data, path, lj


def _oracle_slices(labels, data, path, sl):
    d64 = [t.astype(np.complex128) for t in data]
    n = len(sl)
    ref = []
    for s in range(2 ** n):
        sll, sd = slice_network(labels, d64, sl, [(s >> (n - 1 - j)) & 1 for j in range(n)])
        ref.append(complex(contract_network(sll, sd, path)[1]))
    return np.array(ref)


@pytest.mark.gpu
@pytest.mark.parametrize("d_along", ["rows", "cols"])
@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3", "bf16x6"])
def test_dot_epilogue_matches_the_oracle_per_slice(prec, d_along):
    labels, data, path, sl = network(d_along)
    net = jet.Network(labels, data, precision=prec, profile=2)
    try:
        net.set_open([])
        net.path_set(path)
        net.slice(sl)
        got = net.contract_slices(np.zeros((1, 0), np.int32), list(range(8)))[0]
        recs = net.profile()
    finally:
        net.close()
    dot = [r for r in recs if r["kind"] == "gemm_tc" and r["node"] == 4 and r["variant"] & 8]
    if prec == "bf16x6":
        assert not dot and [r for r in recs if r["kind"] == "gemm_tc" and r["node"] == 4], recs
    else:
        assert dot, recs
        assert [r for r in recs if r["kind"] == "splitk_reduce" and r["node"] == 5], recs
    ref = _oracle_slices(labels, data, path, sl)
    err = float(np.max(np.abs(np.asarray(got) - ref)) / np.max(np.abs(ref)))
    print(f"dot epilogue {prec}, D along {d_along}: max per-slice err {err:.2e}")
    assert err <= 1e-5


@pytest.mark.gpu
@pytest.mark.parametrize("d_along", ["rows", "cols"])
@pytest.mark.parametrize("form", ["single", "unpaired"])
def test_dot_epilogue_blocks_with_one_sibling_or_one_instance(form, d_along):
    """Dot blocks that stage one sibling instance (8 units per step) or hold one
    node instance (its tile computed twice, the second tile's products unused)."""
    labels, data, path, sl = network(d_along, form)
    net = jet.Network(labels, data, precision="fp16x3", profile=2)
    try:
        net.set_open([])
        net.path_set(path)
        net.slice(sl)
        got = net.contract_slices(np.zeros((1, 0), np.int32), list(range(2 ** len(sl))))[0]
        recs = net.profile()
    finally:
        net.close()
    assert [r for r in recs if r["kind"] == "gemm_tc" and r["node"] == 4 and r["variant"] & 8], recs
    ref = _oracle_slices(labels, data, path, sl)
    err = float(np.max(np.abs(np.asarray(got) - ref)) / np.max(np.abs(ref)))
    print(f"dot epilogue, {form} blocks, D along {d_along}: max per-slice err {err:.2e}")
    assert err <= 1e-5


@pytest.mark.gpu
def test_autotuner_chooses_between_the_dot_epilogue_and_the_plain_output():
    """The dot epilogue is a tuned choice (the GEMM's and its parent's times
    against the plain output and the parent's dot-product kernel): after
    jet_autotune the plan takes one of the two forms and matches the oracle."""
    labels, data, path, sl = network("cols")
    net = jet.Network(labels, data, precision="fp16x3", profile=2)
    try:
        net.set_open([])
        net.path_set(path)
        net.slice(sl)
        rows = np.zeros((1, 0), np.int32)
        t = net.autotune(rows)
        assert t["tuned_ms"] <= 1.02 * t["default_ms"], t
        got = net.contract_slices(rows, list(range(8)))[0]
        recs = net.profile()
    finally:
        net.close()
    dot = [r for r in recs if r["kind"] == "gemm_tc" and r["node"] == 4 and r["variant"] & 8]
    plain = [r for r in recs if r["kind"] == "direct" and r["node"] == 5]
    assert bool(dot) != bool(plain), recs
    ref = _oracle_slices(labels, data, path, sl)
    err = float(np.max(np.abs(np.asarray(got) - ref)) / np.max(np.abs(ref)))
    print(f"autotuned ({'dot epilogue' if dot else 'plain output'}): {t}, max per-slice err {err:.2e}")
    assert err <= 1e-5
