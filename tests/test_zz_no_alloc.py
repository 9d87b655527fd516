"""Allocation-free pairwise contraction (jet_pair_contract_noalloc) against the
library's regular, allocating path (a two-tensor network through jet_contract).

This entry point exists for callers that cannot allocate device memory: a
process whose GPU memory is already reserved by its own allocator (an extra
cudaMalloc can fail or fragment that pool) or a latency-critical loop that must
avoid the implicit synchronisation of cudaMalloc/cudaFree.  Its scratch is a
fixed array inside the library that every call reuses, so consecutive calls on
different shapes must not see each other's leftovers.  The file is named to be
collected last."""
import numpy as np
import pytest

from circuits import SplitMix64
from paper_2107_09793_b300 import jet

pytestmark = pytest.mark.gpu

TOL = 1e-5

CASES = [
    # few outputs, long summed index: the sum is split across blocks (partials in the scratch)
    ([0, 1] + list(range(10, 22)), list(range(10, 22)) + [30, 31]),
    # more outputs, shorter summed index, summed labels in reverse order in B
    ([0, 1, 2, 3, 4, 10, 11, 12, 13, 14, 15], [15, 14, 13, 12, 11, 10, 30, 31, 32, 33]),
]


def _rand(seed, rank):
    rng = SplitMix64(seed)
    n = 2 ** rank
    v = np.array([complex(rng.uniform() - 0.5, rng.uniform() - 0.5) for _ in range(n)])
    return v.reshape([2] * rank).astype(np.complex64)


def _reference(la, A, lb, B):
    """Entries of C (row-major, A's free labels then B's) through jet_contract."""
    net = jet.Network([la, lb], [A, B])
    opens = [l for l in la if l not in lb] + [l for l in lb if l not in la]
    net.set_open(opens)
    net.path_set([(0, 1)])
    pats = np.indices([2] * len(opens)).reshape(len(opens), -1).T.astype(np.int32)
    return net.contract(pats)


def _noalloc(torch, la, A, lb, B):
    a = torch.from_numpy(A).cuda()
    b = torch.from_numpy(B).cuda()
    n_free = len([l for l in la if l not in lb]) + len([l for l in lb if l not in la])
    c = torch.zeros(2 ** n_free, dtype=torch.complex64, device="cuda")   # the caller owns the output
    s = torch.cuda.current_stream()
    jet.pair_contract_noalloc(la, A.shape, a.data_ptr(), lb, B.shape, b.data_ptr(), c.data_ptr(), 0, s.cuda_stream)
    s.synchronize()
    return c.cpu().numpy().astype(np.complex128), (a, b, c)


def test_noalloc_matches_allocating_path_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    order = [0, 1, 0]   # two calls in a row on different shapes, then the first shape again
    for call, case in enumerate(order):
        la, lb = CASES[case]
        A = _rand(100 + case, len(la))
        B = _rand(200 + case, len(lb))
        got, _ = _noalloc(torch, la, A, lb, B)
        ref = _reference(la, A, lb, B)
        err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        assert err <= TOL, (call, case, err)


def test_noalloc_rejects_outputs_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    la, lb = list(range(0, 20)), [0, 30]          # 2^19 * 2 = 2^20 outputs > 524280
    x = torch.zeros(4, dtype=torch.complex64, device="cuda")
    with pytest.raises(jet.JetError) as e:
        jet.pair_contract_noalloc(la, [2] * 20, x.data_ptr(), lb, [2, 2], x.data_ptr(), x.data_ptr(), 0, 0)
    assert e.value.code == jet.JET_EINVAL and "at most" in str(e.value)
