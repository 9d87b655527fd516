"""GEMM route of a pairwise contraction (Section 3.1: transpose, transpose,
matrix multiply) vs the oracle's pairwise step, for every operand layout the
plan compiler distinguishes ([free, K], [K, free], interleaved -> permute),
ragged sizes and batched instances, in every precision mode."""
import numpy as np
import pytest

from circuits import SplitMix64
from oracle.einsum import contract_network
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12, "tf32x3": 1e-5, "bf16x3": 1e-5, "bf16x6": 1e-5, "fp16x3": 1e-5, "tf32": 3e-3}


def _rand(rng, shape):
    n = int(np.prod(shape))
    re = np.array([rng.uniform() - 0.5 for _ in range(n)])
    im = np.array([rng.uniform() - 0.5 for _ in range(n)])
    return (re + 1j * im).reshape(shape).astype(np.complex64)


# The pair contraction is the GEMM node; each of its free legs is then absorbed
# by a seeded (dim x 3) selector whose second leg is an output, so the pair
# result is a full M x N matrix inside the tree.
def _gemm_network(la, lb, dims, seed, prec):
    rng = SplitMix64(seed)
    A = _rand(rng, [dims[l] for l in la])
    B = _rand(rng, [dims[l] for l in lb])
    fa = [l for l in la if l not in lb]
    fb = [l for l in lb if l not in la]
    vecs = [_rand(rng, [dims[l], 3]) for l in fa + fb]
    labels = [la, lb] + [[l, 1000 + i] for i, l in enumerate(fa + fb)]
    data = [A, B] + vecs
    net = jet.Network(labels, data, precision=prec)
    opens = [1000 + i for i in range(len(fa + fb))]
    net.set_open(opens)
    # pair first (the GEMM node), then absorb the selector vectors one by one
    n = len(labels)
    path = [(0, 1)]
    cur = n
    for i in range(2, n):
        path.append((cur, i))
        cur += 1
    net.path_set(path)
    return net, labels, data, opens


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
    net, labels, data, opens = _gemm_network(la, lb, dims, 31 + case, prec)
    rng = SplitMix64(7 + case)
    outs = np.array([[rng.randint(3) for _ in opens] for _ in range(4)], np.int32)
    amps = net.contract(outs)
    st = net.stats()
    assert st["n_gemm_nodes"] >= 1
    ref = []
    for o in outs:
        lab = [list(l) for l in labels]
        dat = [d.astype(np.complex128) for d in data]
        for lbl, x in zip(opens, o):
            e = np.zeros(3)
            e[x] = 1
            lab.append([lbl])
            dat.append(e)
        ref.append(complex(contract_network(lab, dat)[1]))
    ref = np.array(ref)
    err = np.linalg.norm(amps - ref) / np.linalg.norm(ref)
    assert err <= TOL[prec], err


def test_gemm_batched_instances_under_slicing():
    """The same GEMM node instanced per slice value (reuse DAG) in one launch."""
    la = [0, 1, 2, 3, 4, 5, 6, 10, 11, 12, 13, 14, 15, 30]
    lb = [10, 11, 12, 13, 14, 15, 20, 21, 22, 23, 24, 25, 31]
    dims = {l: 2 for l in la + lb}
    rng = SplitMix64(5)
    A = _rand(rng, [2] * len(la))
    B = _rand(rng, [2] * len(lb))
    C = _rand(rng, [2, 2])   # joins 30 and 31 so both can be sliced as closed labels
    fa = [l for l in la if l not in lb and l != 30]
    fb = [l for l in lb if l not in la and l != 31]
    vecs = [_rand(rng, [2, 2]) for _ in fa + fb]
    labels = [la, lb, [30, 31]] + [[l, 1000 + i] for i, l in enumerate(fa + fb)]
    data = [A, B, C] + vecs
    net = jet.Network(labels, data)
    opens = [1000 + i for i in range(len(fa + fb))]
    net.set_open(opens)
    path = [(0, 1)]
    cur = len(labels)
    for i in range(2, len(labels)):
        path.append((cur, i))
        cur += 1
    net.path_set(path)
    net.slice([30, 31])
    outs = np.zeros((1, len(opens)), np.int32)
    amp = net.contract(outs)[0]
    assert net.stats()["n_gemm_nodes"] >= 1
    lab = [list(l) for l in labels] + [[o] for o in opens]
    dat = [d.astype(np.complex128) for d in data] + [np.array([1.0, 0.0])] * len(opens)
    ref = complex(contract_network(lab, dat)[1])
    assert abs(amp - ref) <= 1e-5 * abs(ref)
