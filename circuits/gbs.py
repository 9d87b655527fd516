"""Random Gaussian-boson-sampling lattices in a truncated Fock basis
(Algorithm 1 of Section 4; dim = 2 for the 2-D lattice, any dim for
gbs_nd_circuit), bosonic qudit networks with every index of dimension d (the
Fock cutoff).

Readings of what the paper leaves open:
  * Squeezed vacuum S(r)|0>, squeezing phase 0, truncated at d and NOT
    renormalised: c_{2n} = (-tanh r)^n sqrt((2n)!) / (2^n n!) / sqrt(cosh r),
    odd entries 0.
  * BS(theta, phi) = exp(theta (e^{i phi} a1 a2^dag - e^{-i phi} a1^dag a2)).
    The generator conserves the total photon number N, so the exact unitary is
    block-diagonal over N; each (N+1)-dim block is exponentiated exactly and the
    result truncated to n1, n2 < d (a d^2 x d^2 matrix U[(m1 m2), (n1 n2)]).
  * Only true lattice neighbours are coupled: per cycle the horizontal bonds
    (r,c)-(r,c+1) in increasing mode order, then the vertical bonds
    (r,c)-(r+1,c).  theta ~ U[0, pi/2], phi ~ U[0, 2 pi), r ~ U[0.5, 1.0].
  * n dimensions (Algorithm 1's llens[l] = width^(l-1) strides): modes are
    numbered in mixed radix over the lattice shape, last axis fastest; per cycle
    the bonds along the fastest axis (stride 1), then along each slower axis in
    turn, each in increasing mode order, true neighbours only.  For a 2-D shape
    this is the 2-D lattice above, draw for draw.
"""
import math
from typing import Tuple

import numpy as np
import scipy.linalg

from .rng import SplitMix64
from .rqc import Circuit, Gate, grid_layout


def squeezed_vacuum(r: float, d: int) -> np.ndarray:
    v = np.zeros(d, dtype=np.complex128)
    t = math.tanh(r)
    for n in range(0, (d + 1) // 2):
        if 2 * n >= d:
            break
        v[2 * n] = ((-t) ** n) * math.sqrt(math.factorial(2 * n)) / (2 ** n * math.factorial(n))
    return v / math.sqrt(math.cosh(r))


def beamsplitter(theta: float, phi: float, d: int) -> np.ndarray:
    U = np.zeros((d * d, d * d), dtype=np.complex128)
    ep, em = np.exp(1j * phi), np.exp(-1j * phi)
    for N in range(0, 2 * d - 1):
        # sector basis |n1, N - n1>, n1 = 0..N
        dim = N + 1
        H = np.zeros((dim, dim), dtype=np.complex128)
        for n1 in range(dim):
            n2 = N - n1
            if n1 >= 1:   # a1 a2^dag |n1,n2> = sqrt(n1 (n2+1)) |n1-1, n2+1>
                H[n1 - 1, n1] += theta * ep * math.sqrt(n1 * (n2 + 1))
            if n2 >= 1:   # a1^dag a2 |n1,n2> = sqrt((n1+1) n2) |n1+1, n2-1>
                H[n1 + 1, n1] -= theta * em * math.sqrt((n1 + 1) * n2)
        E = scipy.linalg.expm(H)
        for m1 in range(dim):
            for n1 in range(dim):
                m2, n2 = N - m1, N - n1
                if max(m1, m2, n1, n2) < d:
                    U[m1 * d + m2, n1 * d + n2] = E[m1, n1]
    return U


def gbs_lattice_circuit(rows: int, cols: int, d: int, layers: int, seed: int,
                        r_range: Tuple[float, float] = (0.5, 1.0),
                        theta_range: Tuple[float, float] = (0.0, math.pi / 2),
                        phi_range: Tuple[float, float] = (0.0, 2 * math.pi)) -> Circuit:
    sites, idx = grid_layout(rows, cols)
    n = len(sites)
    rng = SplitMix64(seed)
    circ = Circuit(n=n, d=d, sites=sites)
    rs = [rng.uniform_range(*r_range) for _ in range(n)]
    circ.initial = [squeezed_vacuum(r, d) for r in rs]
    circ.squeezing = rs
    bonds = [(idx[(r, c)], idx[(r, c + 1)]) for r in range(rows) for c in range(cols - 1)]
    bonds += [(idx[(r, c)], idx[(r + 1, c)]) for r in range(rows - 1) for c in range(cols)]
    for _ in range(layers):
        for (a, b) in bonds:
            th = rng.uniform_range(*theta_range)
            ph = rng.uniform_range(*phi_range)
            circ.gates.append(Gate(beamsplitter(th, ph, d), (a, b), (th, ph), kind="bs"))
    return circ


def gbs_nd_circuit(shape: Tuple[int, ...], d: int, layers: int, seed: int,
                   r_range: Tuple[float, float] = (0.5, 1.0),
                   theta_range: Tuple[float, float] = (0.0, math.pi / 2),
                   phi_range: Tuple[float, float] = (0.0, 2 * math.pi)) -> Circuit:
    shape = tuple(int(w) for w in shape)
    n = int(np.prod(shape))
    strides = [int(np.prod(shape[a + 1:])) for a in range(len(shape))]
    coords = [tuple((i // strides[a]) % shape[a] for a in range(len(shape))) for i in range(n)]
    rng = SplitMix64(seed)
    circ = Circuit(n=n, d=d, sites=coords)
    rs = [rng.uniform_range(*r_range) for _ in range(n)]
    circ.initial = [squeezed_vacuum(r, d) for r in rs]
    circ.squeezing = rs
    bonds = []
    for a in reversed(range(len(shape))):   # fastest axis first
        bonds += [(i, i + strides[a]) for i in range(n) if coords[i][a] < shape[a] - 1]
    for _ in range(layers):
        for (p, q) in bonds:
            th = rng.uniform_range(*theta_range)
            ph = rng.uniform_range(*phi_range)
            circ.gates.append(Gate(beamsplitter(th, ph, d), (p, q), (th, ph), kind="bs"))
    return circ


def random_patterns(n: int, count: int, seed: int, d: int) -> np.ndarray:
    """Photon-number patterns, each mode uniform in [0, d)."""
    rng = SplitMix64(seed)
    return np.array([[rng.randint(d) for _ in range(n)] for _ in range(count)],
                    dtype=np.int32).reshape(count, n)
