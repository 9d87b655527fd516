"""Allocation-free pairwise contraction (jet_pair_contract_noalloc) against the
library's regular, allocating path (a two-tensor network through jet_contract)
and against the FP64 oracle's pairwise step, element by element.

This entry point exists for callers that cannot allocate device memory: a
process whose GPU memory is already reserved by its own allocator (an extra
cudaMalloc can fail or fragment that pool) or a latency-critical loop that must
avoid the implicit synchronisation of cudaMalloc/cudaFree.  Its scratch is a
fixed array inside the library that every call reuses, so consecutive calls on
different shapes must not see each other's leftovers.  The file is named to be
collected last."""
import numpy as np
import pytest

from circuits.rng import uniform_array
from oracle.einsum import _pair
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu

TOL = 1e-5   # complex64 contraction, FP32 accumulation (the library's FP32 tolerance)

CASES = [
    # few outputs, long summed index: the sum is split across blocks (partials in the scratch)
    (([0, 1] + list(range(10, 22)), [2] * 14), (list(range(10, 22)) + [30, 31], [2] * 14)),
    # more outputs, shorter summed index, summed labels in reverse order in B
    (([0, 1, 2, 3, 4, 10, 11, 12, 13, 14, 15], [2] * 11), ([15, 14, 13, 12, 11, 10, 30, 31, 32, 33], [2] * 10)),
    # dims 3 and 4 (offsets decoded by division, not by shifts), summed labels interleaved
    (([0, 10, 1, 11, 12], [3, 4, 4, 3, 4]), ([12, 30, 10, 11, 31], [4, 3, 4, 3, 4])),
]


def _rand(seed, shape):
    n = int(np.prod(shape))
    u = uniform_array(seed, 2 * n) - 0.5
    return (u[:n] + 1j * u[n:]).reshape(shape).astype(np.complex64)


def _oracle(la, A, lb, B):
    """C by the oracle's FP64 pairwise step (numpy.tensordot over the shared labels)."""
    _, t = _pair(list(la), A.astype(np.complex128), list(lb), B.astype(np.complex128))
    return np.asarray(t).ravel()


def _allocating(la, A, lb, B):
    """Entries of C (row-major, A's free labels then B's) through jet_contract."""
    net = jet.Network([la, lb], [A, B])
    opens = [l for l in la if l not in lb] + [l for l in lb if l not in la]
    dims = [A.shape[la.index(l)] if l in la else B.shape[lb.index(l)] for l in opens]
    net.set_open(opens)
    net.path_set([(0, 1)])
    pats = np.indices(dims).reshape(len(opens), -1).T.astype(np.int32)
    out = net.contract(pats)
    net.close()
    return out


def _noalloc(torch, la, A, lb, B):
    a = torch.from_numpy(A.ravel()).cuda()
    b = torch.from_numpy(B.ravel()).cuda()
    n_out = int(np.prod([A.shape[i] for i, l in enumerate(la) if l not in lb] +
                        [B.shape[i] for i, l in enumerate(lb) if l not in la]))
    c = torch.full((n_out,), complex(np.nan, np.nan), dtype=torch.complex64, device="cuda")   # caller-owned output
    s = torch.cuda.current_stream()
    jet.pair_contract_noalloc(la, A.shape, a.data_ptr(), lb, B.shape, b.data_ptr(), c.data_ptr(), 0, s.cuda_stream)
    s.synchronize()
    return c.cpu().numpy().astype(np.complex128)


def _err(got, ref):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


def test_noalloc_matches_allocating_path_and_oracle_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    order = [0, 1, 2, 0]   # calls in a row on different shapes, then the first shape again
    for call, case in enumerate(order):
        (la, da), (lb, db) = CASES[case]
        A = _rand(100 + case, da)
        B = _rand(200 + case, db)
        got = _noalloc(torch, la, A, lb, B)
        ref = _oracle(la, A, lb, B)
        alloc = _allocating(la, A, lb, B)
        assert got.shape == ref.shape
        e_orc, e_alloc = _err(got, ref), _err(got, alloc)
        assert e_orc <= TOL, (call, case, e_orc)       # every element, against the FP64 oracle
        assert e_alloc <= TOL, (call, case, e_alloc)   # and against the allocating entry point


def test_noalloc_ignores_dim1_labels():
    torch = pytest.importorskip("torch")
    # 40 labels of dim 1 on A, 29 of dim 1 and 11 of dim 2 on B, none shared:
    # an outer product of 2^11 entries whose 80 output labels are mostly trivial
    la, da = list(range(40)), [1] * 40
    lb, db = list(range(100, 140)), [1] * 29 + [2] * 11
    A = _rand(300, da)
    B = _rand(301, db)
    got = _noalloc(torch, la, A, lb, B)
    # the oracle's step on the same tensors with their dim-1 axes squeezed out
    # (80 output axes exceed numpy's limit; a dim-1 axis holds one entry)
    lb2 = [l for l, d in zip(lb, db) if d > 1]
    ref = _oracle([], A.reshape(()), lb2, B.reshape([2] * len(lb2)))
    assert _err(got, ref) <= TOL


def test_noalloc_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    x = torch.zeros(4, dtype=torch.complex64, device="cuda")
    la, lb = list(range(0, 20)), [0, 30]          # 2^19 * 2 = 2^20 outputs > 524280
    with pytest.raises(jet.JetError) as e:
        jet.pair_contract_noalloc(la, [2] * 20, x.data_ptr(), lb, [2, 2], x.data_ptr(), x.data_ptr(), 0, 0)
    assert e.value.code == jet.JET_EINVAL and "at most" in str(e.value)
    with pytest.raises(jet.JetError) as e:          # a shared label with different dims
        jet.pair_contract_noalloc([0, 1], [2, 2], x.data_ptr(), [1, 2], [4, 1], x.data_ptr(), x.data_ptr(), 0, 0)
    assert e.value.code == jet.JET_EINVAL
    with pytest.raises(jet.JetError) as e:          # more than 40 labels on one tensor
        jet.pair_contract_noalloc(list(range(41)), [1] * 41, x.data_ptr(), [0], [1], x.data_ptr(), x.data_ptr(), 0, 0)
    assert e.value.code == jet.JET_EINVAL
    with pytest.raises(ValueError):                 # one dim per label
        jet.pair_contract_noalloc([0, 1], [2], x.data_ptr(), [1], [2], x.data_ptr(), x.data_ptr(), 0, 0)
