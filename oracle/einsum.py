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


def contract_pairs(labels, data, path: Sequence[Tuple[int, int]]):
    """contract_network one pairwise step at a time, for a caller that times
    parts of a contraction: a generator that performs the next tensordot of
    the path on each next() and yields (step index, labels, tensor) of that
    step's result; the last one yielded is the contraction's result."""
    live_l = dict(enumerate([list(l) for l in labels]))
    live_t = dict(enumerate([np.asarray(t, dtype=np.complex128) for t in data]))
    nxt = len(live_l)
    for i, (a, b) in enumerate(path):
        out, t = _pair(live_l.pop(a), live_t.pop(a), live_l.pop(b), live_t.pop(b))
        live_l[nxt], live_t[nxt] = out, t
        nxt += 1
        yield i, out, t


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


def _tree_flop(children, labels_of, dims, node):
    """FLOP of the internal steps under `node` (8 per complex multiply-add)."""
    total, stack = 0, [node]
    while stack:
        v = stack.pop()
        if v in children:
            a, b = children[v]
            u = set(labels_of[a]) | set(labels_of[b])
            total += 8 * _size(u, dims)
            stack += [a, b]
    return total


def improve_path(labels, dims: Dict[int, int], path, k: int = 8, passes: int = 4, cap=None):
    """Local re-optimisation of a pairwise path (Section 2.3: any order gives the
    same result, only the cost differs).  For every internal node, the sub-tree
    below it is opened down to at most k tensors (splitting the largest first)
    and their cheapest contraction order is found by exhaustive dynamic
    programming over subsets; it replaces the old sub-tree when it costs fewer
    FLOP and creates no intermediate above `cap` (default: the path's largest).
    Returns a new SSA path over the same tensors."""
    n = len(labels)
    labels_of = {i: frozenset(l) for i, l in enumerate(labels)}
    children = {}
    for s, (a, b) in enumerate(path):
        children[n + s] = (a, b)
        labels_of[n + s] = labels_of[a] ^ labels_of[b]
    root = n + len(path) - 1
    if cap is None:
        cap = max(_size(labels_of[v], dims) for v in children)
    fresh = [root + 1]
    for _ in range(passes):
        changed = False
        order, stack = [], [root]
        while stack:
            v = stack.pop()
            if v in children:
                order.append(v)
                stack += list(children[v])
        for v in order:
            if v not in children:
                continue
            front, inner = [v], []
            while len(front) < k:
                cand = [x for x in front if x in children]
                if not cand:
                    break
                x = max(cand, key=lambda y: _size(labels_of[y], dims))
                front.remove(x)
                inner.append(x)
                front += list(children[x])
            m = len(front)
            if m < 3:
                continue
            current = sum(8 * _size(labels_of[children[x][0]] | labels_of[children[x][1]], dims) for x in inner)
            outs = {}
            for S in range(1, 1 << m):
                o = frozenset()
                for i in range(m):
                    if S >> i & 1:
                        o = o ^ labels_of[front[i]]
                outs[S] = o
            full = (1 << m) - 1
            best = {1 << i: (0, None) for i in range(m)}
            for S in range(1, full + 1):
                if S & (S - 1) == 0:
                    continue
                if S != full and _size(outs[S], dims) > cap:
                    best[S] = (float("inf"), None)
                    continue
                choice = (float("inf"), None)
                s1 = (S - 1) & S
                while s1:
                    s2 = S ^ s1
                    if s1 < s2:
                        c = best[s1][0] + best[s2][0] + 8 * _size(outs[s1] | outs[s2], dims)
                        if c < choice[0]:
                            choice = (c, (s1, s2))
                    s1 = (s1 - 1) & S
                best[S] = choice
            if best[full][0] < current:
                for x in inner:
                    if x != v:
                        del children[x]

                def build(S):
                    if S & (S - 1) == 0:
                        return front[S.bit_length() - 1]
                    s1, s2 = best[S][1]
                    a, b = build(s1), build(s2)
                    node = v if S == full else fresh[0]
                    if S != full:
                        fresh[0] += 1
                    children[node] = (a, b)
                    labels_of[node] = labels_of[a] ^ labels_of[b]
                    return node
                build(full)
                changed = True
        if not changed:
            break
    out, ssa, nxt = [], {i: i for i in range(n)}, [n]

    def emit(v):
        if v < n:
            return v
        a, b = emit(children[v][0]), emit(children[v][1])
        out.append((min(a, b), max(a, b)))
        ssa[v] = nxt[0]
        nxt[0] += 1
        return ssa[v]
    emit(root)
    return out


def slice_until(labels, dims: Dict[int, int], path, cap: int, max_n: int = 64):
    """Choose labels to slice (Section 2.4) along a fixed path until no
    intermediate exceeds `cap` elements: each time, among the labels of the
    largest intermediate, the one whose slicing gives the smallest total FLOP
    over all slices.  Returns the list of sliced labels."""
    sliced = []
    while True:
        d = {x: (1 if x in sliced else s) for x, s in dims.items()}
        n = len(labels)
        live = {i: list(l) for i, l in enumerate(labels)}
        biggest, where = 0, None
        for s, (a, b) in enumerate(path):
            out = [x for x in live[a] if x not in live[b]] + [x for x in live[b] if x not in live[a]]
            live[n + s] = out
            sz = _size(out, d)
            if sz > biggest:
                biggest, where = sz, out
        if biggest <= cap:
            return sliced
        if len(sliced) >= max_n:
            raise ValueError("slice_until: cap not reached")
        best = None
        for x in where:
            if d[x] == 1:
                continue
            d2 = dict(d)
            d2[x] = 1
            total = network_flops(labels, d2, path) * int(np.prod([dims[y] for y in sliced + [x]]))
            if best is None or total < best[0]:
                best = (total, x)
        sliced.append(best[1])
