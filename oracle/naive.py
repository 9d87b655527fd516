"""Literal sum over every index assignment (Eq. naive_summation).  Test
infrastructure only; pure-Python loops, for networks of at most ~16 indices."""
from itertools import product

import numpy as np


def naive_sum(labels, data, open_labels=()):
    """Sum over all assignments of the closed labels of the product of every
    tensor's entry.  With open labels, returns the tensor over those labels (in
    the given order); otherwise a complex scalar."""
    dims = {}
    for l, t in zip(labels, data):
        for x, s in zip(l, np.shape(t)):
            if x in dims and dims[x] != s:
                raise ValueError(f"label {x}: dims {dims[x]} vs {s}")
            dims[x] = s
    closed = [x for x in dims if x not in open_labels]
    opens = list(open_labels)
    out = np.zeros([dims[x] for x in opens], dtype=np.complex128)
    for ov in product(*[range(dims[x]) for x in opens]):
        acc = 0j
        for cv in product(*[range(dims[x]) for x in closed]):
            val = dict(zip(closed, cv))
            val.update(zip(opens, ov))
            term = 1 + 0j
            for l, t in zip(labels, data):
                term *= complex(np.asarray(t)[tuple(val[x] for x in l)])
                if term == 0:
                    break
            acc += term
        out[ov] = acc
    return out if opens else complex(out)
