"""O2: FP64 pairwise contraction of a tensor network.  Test infrastructure only.

Section 2.3 (Eq. sequence): the network is reduced two tensors at a time; each
pairwise step sums over the indices the two tensors share and keeps the rest.
The step is numpy.tensordot (a library contraction); there is no blocking,
fusion or reordering beyond that.  Section 2.4 (Eq. sliced_sum): slicing an
index fixes its value in every tensor that carries it; the amplitude is the sum
of the partial contractions over all values.  Section 2.2.1: an amplitude <x|
attaches a rank-1 basis bra to every open leg.
"""
from itertools import product
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np


def attach_bras(labels, data, open_labels, pattern, d):
    """Append one rank-1 bra e_{x_q} per open leg q (the <a_i| tensors)."""
    labels = [list(l) for l in labels]
    data = list(data)
    for lab, x in zip(open_labels, pattern):
        e = np.zeros(d, dtype=np.complex128)
        e[int(x)] = 1.0
        labels.append([lab])
        data.append(e)
    return labels, data


def slice_network(labels, data, sliced_labels, values):
    """Fix every sliced label to its value in each tensor that carries it."""
    fix = dict(zip(sliced_labels, values))
    out_l, out_d = [], []
    for lab, t in zip(labels, data):
        t = np.asarray(t)
        keep = []
        for pos, l in enumerate(lab):
            if l in fix:
                pass
            else:
                keep.append(l)
        idx = tuple(fix[l] if l in fix else slice(None) for l in lab)
        out_l.append(keep)
        out_d.append(np.asarray(t[idx]))
    return out_l, out_d


def _size(labels, dims):
    s = 1
    for l in labels:
        s *= dims[l]
    return s


def greedy_path(labels, dims: Dict[int, int]) -> List[Tuple[int, int]]:
    """SSA path (tensor ids 0..n-1, step k creates id n+k): repeatedly contract
    the connected pair minimising size(out) - size(A) - size(B); ties go to
    the smallest ids.  Disconnected pieces are joined last, smallest first."""
    live = {i: list(l) for i, l in enumerate(labels)}
    owner: Dict[int, set] = {}
    for i, l in live.items():
        for x in l:
            owner.setdefault(x, set()).add(i)
    nxt = len(labels)
    path = []
    while len(live) > 1:
        best = None
        seen = set()
        for x, ts in owner.items():
            if len(ts) != 2:
                continue
            a, b = sorted(ts)
            if (a, b) in seen:
                continue
            seen.add((a, b))
            la, lb = live[a], live[b]
            out = [y for y in la if y not in lb] + [y for y in lb if y not in la]
            score = _size(out, dims) - _size(la, dims) - _size(lb, dims)
            key = (score, a, b)
            if best is None or key < best[0]:
                best = (key, a, b, out)
        if best is None:   # no shared index left: outer product of the two smallest
            ids = sorted(live, key=lambda i: (_size(live[i], dims), i))
            a, b = sorted(ids[:2])
            out = live[a] + live[b]
        else:
            _, a, b, out = best
        for x in live[a] + live[b]:
            owner[x].discard(a)
            owner[x].discard(b)
        del live[a], live[b]
        live[nxt] = out
        for x in out:
            owner.setdefault(x, set()).add(nxt)
        for x in [x for x, ts in owner.items() if not ts]:
            del owner[x]
        path.append((a, b))
        nxt += 1
    return path


def _pair(la, ta, lb, tb):
    shared = [x for x in la if x in lb]
    ia = [la.index(x) for x in shared]
    ib = [lb.index(x) for x in shared]
    t = np.tensordot(ta, tb, axes=(ia, ib))
    out = [x for x in la if x not in shared] + [x for x in lb if x not in shared]
    return out, t


def contract_network(labels, data, path: Optional[Sequence[Tuple[int, int]]] = None):
    """Contract the whole network pairwise along an SSA path (default: greedy).
    Returns (remaining labels, tensor); a closed network gives a 0-d tensor."""
    labels = [list(l) for l in labels]
    data = [np.asarray(t, dtype=np.complex128) for t in data]
    if len(data) == 1:
        return labels[0], data[0]
    if path is None:
        dims = {}
        for l, t in zip(labels, data):
            for x, s in zip(l, t.shape):
                dims[x] = s
        path = greedy_path(labels, dims)
    live_l = dict(enumerate(labels))
    live_t = dict(enumerate(data))
    nxt = len(labels)
    for a, b in path:
        out, t = _pair(live_l.pop(a), live_t.pop(a), live_l.pop(b), live_t.pop(b))
        live_l[nxt], live_t[nxt] = out, t
        nxt += 1
    (k,) = live_l.keys()
    return live_l[k], live_t[k]


def amplitude(tn, pattern, sliced: Sequence[int] = (), path=None) -> complex:
    """<x|U|psi0> by pairwise contraction; with sliced labels, as the explicit
    sum of all slice partials (Eq. sliced_sum)."""
    labels, data = attach_bras(tn.labels, tn.data, tn.open_labels, pattern, tn.dim)
    if not sliced:
        _, t = contract_network(labels, data, path)
        return complex(t)
    return complex(np.sum(sliced_partials(tn, pattern, sliced)))


def sliced_partials(tn, pattern, sliced: Sequence[int], slice_ids=None) -> np.ndarray:
    """s_i for every slice id i (mixed radix over the sliced labels, the first
    sliced label most significant), or only for the given ids."""
    labels, data = attach_bras(tn.labels, tn.data, tn.open_labels, pattern, tn.dim)
    dims = {}
    for l, t in zip(labels, data):
        for x, s in zip(l, np.shape(t)):
            dims[x] = s
    radix = [dims[x] for x in sliced]
    total = int(np.prod(radix)) if radix else 1
    ids = range(total) if slice_ids is None else slice_ids
    out = []
    sl0, sd0 = slice_network(labels, data, sliced, [0] * len(sliced))
    path = greedy_path(sl0, {x: dims[x] for x in dims if x not in sliced})
    for i in ids:
        vals, r = [], int(i)
        for R in reversed(radix):
            vals.append(r % R)
            r //= R
        vals = vals[::-1]
        sl, sd = slice_network(labels, data, sliced, vals)
        _, t = contract_network(sl, sd, path)
        out.append(complex(t))
    return np.array(out, dtype=np.complex128)


def network_flops(labels, dims: Dict[int, int], path) -> int:
    """Real FLOP of a pairwise path: 8 per complex multiply-add over the union
    of the two operands' indices."""
    live = {i: list(l) for i, l in enumerate(labels)}
    nxt = len(labels)
    total = 0
    for a, b in path:
        la, lb = live.pop(a), live.pop(b)
        union = list(dict.fromkeys(la + lb))
        total += 8 * _size(union, dims)
        live[nxt] = [x for x in la if x not in lb] + [x for x in lb if x not in la]
        nxt += 1
    return total
