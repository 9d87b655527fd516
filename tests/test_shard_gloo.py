"""Multi-process slicing (Section 2.4: slices are independent, one FP64 sum at
the end) with world_size 2 on the CPU: two gloo ranks each take a contiguous
range of slice ids, produce their per-slice partials (here from the FP64
oracle, standing in for jet_contract_slices on a GPU), gather them and sum in
increasing slice id.  The result must equal the unsliced oracle amplitude and,
bit for bit, the single-process ordered sum."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from circuits import random_grid_circuit, circuit_to_network, random_bitstrings
from paper_2107_09793_b300.shard import slice_ranges, ordered_sum, gather_partials

SLICED = None   # chosen in _case()


def _case():
    circ = random_grid_circuit(2, 3, 6, seed=61)
    tn = circuit_to_network(circ)
    out = random_bitstrings(6, 1, 62)[0]
    # four closed wire labels (the first four labels held by two tensors)
    owners = {}
    for i, ls in enumerate(tn.labels):
        for l in ls:
            owners.setdefault(l, []).append(i)
    sliced = [l for l in sorted(owners) if len(owners[l]) == 2][5:9]
    return tn, out, sliced


def test_slice_ranges_cover_every_id_once():
    for n, w in [(64, 2), (64, 3), (5, 8), (0, 2), (1048576, 7)]:
        r = slice_ranges(n, w)
        assert len(r) == w and r[0][0] == 0 and r[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        sizes = [b - a for a, b in r]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slice_ranges(4, 0)


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tn, out, sliced = _case()
    n_sl = 2 ** len(sliced)
    start, stop = slice_ranges(n_sl, world)[rank]
    local = oracle.sliced_partials(tn, out, sliced, list(range(start, stop))).reshape(1, -1)
    parts = gather_partials(local, world)
    amp = ordered_sum(parts, slice_ranges(n_sl, world))
    q.put((rank, amp.tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_slices_in_order():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    tn, out, sliced = _case()
    n_sl = 2 ** len(sliced)
    every = oracle.sliced_partials(tn, out, sliced, list(range(n_sl))).reshape(1, -1)
    single = ordered_sum([every], [(0, n_sl)])
    for r in (0, 1):
        got = np.array(res[r])
        assert got.tobytes() == single.tobytes()          # same FP64 order, any rank count
    assert abs(single[0] - oracle.amplitude(tn, out)) <= 1e-13


def test_range_slice_ids_partition_every_slice_once():
    from paper_2107_09793_b300.shard import range_slice_ids
    for dims, pos in [([2] * 6, [1, 4]), ([2, 3, 4], [0, 2]), ([2] * 12, [1, 3]), ([3, 2], [])]:
        rs = range_slice_ids(dims, pos)
        flat = sorted(i for r in rs for i in r)
        assert flat == list(range(int(np.prod(dims))))
        assert all(r == sorted(r) for r in rs)
        assert len(rs) == int(np.prod([dims[j] for j in pos])) if pos else len(rs) == 1


class _OracleNet:
    """Stands in for a library handle on the CPU: partials from the FP64 oracle;
    the partition fixes the first sliced labels, more of them for smaller caps."""
    def __init__(self, tn, out, sliced):
        self.tn, self.out, self.sliced = tn, out, sliced

    def _outputs(self, outputs):
        return np.asarray(outputs, np.int32).reshape(1, -1)

    def plan_ranges(self, outputs, cap):
        k = 1 if cap >= 1 << 30 else 2
        return {"fixed_labels": [self.sliced[0], self.sliced[2]][:k], "n_ranges": 2 ** k}

    def contract_slices(self, outputs, ids, stream=0):
        return oracle.sliced_partials(self.tn, self.out, self.sliced, ids).reshape(1, -1)


def _range_rank_main(rank, world, port, q):
    import torch.distributed as dist
    from paper_2107_09793_b300.shard import contract_sharded_ranges
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    tn, out, sliced = _case()
    net = _OracleNet(tn, out, sliced)
    amp = contract_sharded_ranges(net, [out], rank, world, 1 << 30, sliced, [2] * len(sliced))
    q.put((rank, np.asarray(amp).tolist()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_the_slice_ranges():
    """Each rank runs every other sharing-aware range; the gathered partials,
    in increasing slice id, sum (in the library) to the single-process sum."""
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_range_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    tn, out, sliced = _case()
    n_sl = 2 ** len(sliced)
    every = oracle.sliced_partials(tn, out, sliced, list(range(n_sl))).reshape(1, -1)
    single = ordered_sum([every], [(0, n_sl)])
    for r in (0, 1):
        assert np.array(res[r]).tobytes() == single.tobytes()
    assert abs(single[0] - oracle.amplitude(tn, out)) <= 1e-13
