"""Slices of one contraction spread over several processes (one GPU each).

Section 2.4 (Eq. sliced_sum): the slices of an amplitude are independent
contractions whose results are summed, so a multi-GPU run needs no exchange
while contracting.  Each rank takes one contiguous range of slice ids (mixed
radix, first sliced label most significant, so a range shares its high-order
digits and with them the shared subtrees of Section 3.2), contracts it with
jet_contract_slices, and the per-slice partials (n_amps x n_ids complex128,
a few KB) are gathered to every rank and summed in increasing slice id: the
same FP64 order as a single-GPU jet_contract, so the result does not depend
on the number of ranks.
"""
from typing import List, Sequence, Tuple

import numpy as np


def slice_ranges(n_slices: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous [start, stop) ranges of slice ids, one per rank, sizes differing by at most one."""
    if n_slices < 0 or world < 1:
        raise ValueError("need n_slices >= 0 and world >= 1")
    base, extra = divmod(n_slices, world)
    out, start = [], 0
    for r in range(world):
        stop = start + base + (1 if r < extra else 0)
        out.append((start, stop))
        start = stop
    return out


def ordered_sum(partials_by_rank: Sequence[np.ndarray], ranges: Sequence[Tuple[int, int]]) -> np.ndarray:
    """amp_b = sum over slice ids in increasing order of the gathered partials
    (rank r's array is n_amps x (stop_r - start_r)): the ranks' partials are
    concatenated in increasing slice id and summed by the library
    (jet_sum_partials, FP64, in that order)."""
    from .jet import sum_partials
    n_amps = next((p.shape[0] for p in partials_by_rank if p.size), 0)
    parts = []
    for (start, stop), p in sorted(zip(ranges, partials_by_rank), key=lambda x: x[0][0]):
        if stop <= start:
            continue
        if p.shape[1] != stop - start:
            raise ValueError("a rank's partials do not match its slice range")
        parts.append(np.asarray(p, np.complex128))
    if not parts:
        return np.zeros(n_amps, dtype=np.complex128)
    return sum_partials(np.concatenate(parts, axis=1))


def gather_partials(local: np.ndarray, world: int, group=None) -> List[np.ndarray]:
    """Every rank's partials on every rank (torch.distributed, any backend)."""
    if world == 1:
        return [local]
    import torch
    import torch.distributed as dist
    out: List = [None] * world
    dist.all_gather_object(out, np.ascontiguousarray(local), group=group)
    return [np.asarray(x) for x in out]


def contract_sharded(net, outputs, rank: int, world: int, group=None, stream: int = 0) -> np.ndarray:
    """This rank's slice range through jet_contract_slices, then the ordered
    FP64 sum over all ranks' partials.  Every rank returns the amplitudes."""
    n_slices = net.stats()["n_slices"]
    ranges = slice_ranges(n_slices, world)
    start, stop = ranges[rank]
    o = net._outputs(outputs)
    if stop > start:
        local = net.contract_slices(o, list(range(start, stop)), stream=stream)
    else:
        local = np.zeros((o.shape[0], 0), dtype=np.complex128)
    return ordered_sum(gather_partials(local, world, group), ranges)


def range_slice_ids(sliced_dims: Sequence[int], fixed_pos: Sequence[int]) -> List[List[int]]:
    """Slice ids of each range of a partition that fixes the digits of the
    sliced labels at fixed_pos (positions in the sliced-label order, mixed
    radix, first label most significant): range k holds every slice whose
    digits at fixed_pos are the mixed-radix digits of k, in increasing id."""
    n = len(sliced_dims)
    w = [1] * n
    for j in range(n - 2, -1, -1):
        w[j] = w[j + 1] * sliced_dims[j + 1]
    total = w[0] * sliced_dims[0] if n else 1
    n_ranges = 1
    for j in fixed_pos:
        n_ranges *= sliced_dims[j]
    out: List[List[int]] = [[] for _ in range(n_ranges)]
    for s in range(total):
        k = 0
        for j in fixed_pos:
            k = k * sliced_dims[j] + (s // w[j]) % sliced_dims[j]
        out[k].append(s)
    return out


def contract_sharded_ranges(net, outputs, rank: int, world: int, max_bytes: int, sliced: Sequence[int],
                            sliced_dims: Sequence[int], group=None, stream: int = 0) -> np.ndarray:
    """One amplitude's slices over `world` ranks, by the library's sharing-aware
    slice ranges (jet_plan_ranges): the workspace cap is halved until there are
    at least `world` ranges, rank r contracts ranges r, r + world, ... (each one
    plan, jet_contract_slices), and the partials of every rank, concatenated in
    increasing slice id, are summed by the library (jet_sum_partials).  Every
    rank returns the amplitudes, bitwise the same for any rank count that gives
    the same partition."""
    o = net._outputs(outputs)
    cap = int(max_bytes)
    part = net.plan_ranges(o, cap)
    while part["n_ranges"] < world and cap > (1 << 20):
        cap //= 2
        part = net.plan_ranges(o, cap)
    pos = [list(sliced).index(x) for x in part["fixed_labels"]]
    ranges = range_slice_ids(list(sliced_dims), pos)
    mine_ids, mine_parts = [], []
    for k in range(rank, len(ranges), world):
        ids = ranges[k]
        mine_ids += ids
        mine_parts.append(net.contract_slices(o, ids, stream=stream))
    local_ids = np.array(mine_ids, np.int64)
    local = np.concatenate(mine_parts, axis=1) if mine_parts else np.zeros((o.shape[0], 0), np.complex128)
    if world > 1:
        import torch.distributed as dist
        got: List = [None] * world
        dist.all_gather_object(got, (local_ids, np.ascontiguousarray(local)), group=group)
    else:
        got = [(local_ids, local)]
    ids_all = np.concatenate([g[0] for g in got])
    parts_all = np.concatenate([g[1] for g in got], axis=1)
    order = np.argsort(ids_all, kind="stable")
    from .jet import sum_partials
    return sum_partials(parts_all[:, order])
