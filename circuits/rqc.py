"""Random quantum circuits on rectangular qubit grids, shaped like the
Sycamore-53 workloads of Section 4 (the circuit files themselves are not used:
these are synthetic stand-ins of the same gate family).

Conventions (readings of points the paper leaves open):
  * Qubit q of an R x C grid sits at (r, c) with q numbered row-major over the
    sites that are present (a removed corner is skipped).
  * A 1-qubit gate is a 2x2 matrix U[out, in]; a 2-qubit gate on (q1, q2) is a
    4x4 matrix U[(o1 o2), (i1 i2)] with q1 the more significant bit.
  * Coupler pattern "ABCDCDAB": A = horizontal bonds (r,c)-(r,c+1), c even;
    B = horizontal, c odd; C = vertical (r,c)-(r+1,c), r even; D = vertical,
    r odd.  Cycle t uses letter "ABCDCDAB"[t mod 8]; each cycle is a layer of
    1-qubit gates followed by the 2-qubit layer.
  * sqrt(X), sqrt(Y), sqrt(W) with W = (X+Y)/sqrt(2); the first cycle draws
    uniformly from the three, later cycles from the two that differ from the
    qubit's previous gate.
  * fSim(theta, phi) = [[1,0,0,0],[0,cos,-i sin,0],[0,-i sin,cos,0],[0,0,0,e^{-i phi}]].
"""
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple
import math

import numpy as np

from .rng import SplitMix64

_S2 = 1.0 / math.sqrt(2.0)


def sqrt_x() -> np.ndarray:
    return _S2 * np.array([[1, -1j], [-1j, 1]], dtype=np.complex128)


def sqrt_y() -> np.ndarray:
    return _S2 * np.array([[1, -1], [1, 1]], dtype=np.complex128)


def sqrt_w() -> np.ndarray:
    # sqrt(W), W = (X + Y)/sqrt(2): off-diagonals -sqrt(i) and sqrt(-i)
    si = np.exp(1j * math.pi / 4)
    smi = np.exp(-1j * math.pi / 4)
    return _S2 * np.array([[1, -si], [smi, 1]], dtype=np.complex128)


def fsim(theta: float, phi: float) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[1, 0, 0, 0],
                     [0, c, -1j * s, 0],
                     [0, -1j * s, c, 0],
                     [0, 0, 0, np.exp(-1j * phi)]], dtype=np.complex128)


def rz(a: float) -> np.ndarray:
    return np.array([[np.exp(-0.5j * a), 0], [0, np.exp(0.5j * a)]], dtype=np.complex128)


def ry(b: float) -> np.ndarray:
    c, s = math.cos(0.5 * b), math.sin(0.5 * b)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rzry(a: float, b: float) -> np.ndarray:
    """Rz(a) . Ry(b): Ry acts first."""
    return rz(a) @ ry(b)


def drzry(a: float, b: float) -> Tuple[np.ndarray, np.ndarray]:
    """Analytic derivatives d/da and d/db of Rz(a) Ry(b)."""
    drz = np.array([[-0.5j * np.exp(-0.5j * a), 0], [0, 0.5j * np.exp(0.5j * a)]],
                   dtype=np.complex128)
    c, s = math.cos(0.5 * b), math.sin(0.5 * b)
    dry = 0.5 * np.array([[-s, -c], [c, -s]], dtype=np.complex128)
    return drz @ ry(b), rz(a) @ dry


def dfsim(theta: float, phi: float) -> Tuple[np.ndarray, np.ndarray]:
    """Analytic derivatives d/dtheta and d/dphi of fSim(theta, phi)."""
    c, s = math.cos(theta), math.sin(theta)
    dt = np.array([[0, 0, 0, 0],
                   [0, -s, -1j * c, 0],
                   [0, -1j * c, -s, 0],
                   [0, 0, 0, 0]], dtype=np.complex128)
    dp = np.zeros((4, 4), dtype=np.complex128)
    dp[3, 3] = -1j * np.exp(-1j * phi)
    return dt, dp


@dataclass
class Gate:
    matrix: np.ndarray          # (d^k, d^k) complex128, U[out, in]
    qubits: Tuple[int, ...]     # k qudits, first = most significant
    params: Tuple[float, ...] = ()
    kind: str = ""              # "sx", "sy", "sw", "fsim", "rzry", "sq", "bs"


@dataclass
class Circuit:
    n: int                      # number of qudits
    d: int                      # local dimension
    gates: List[Gate] = field(default_factory=list)
    initial: List[np.ndarray] = field(default_factory=list)  # per-qudit initial vector (d,)
    sites: List[Tuple[int, int]] = field(default_factory=list)

    def n_params(self) -> int:
        return sum(len(g.params) for g in self.gates)


def grid_layout(rows: int, cols: int, removed: Sequence[Tuple[int, int]] = ()):
    """Row-major qubit numbering of the present sites; returns (sites, index map)."""
    removed = set(removed)
    sites = [(r, c) for r in range(rows) for c in range(cols) if (r, c) not in removed]
    return sites, {s: i for i, s in enumerate(sites)}


def coupler_layers(rows: int, cols: int, removed: Sequence[Tuple[int, int]] = ()):
    """Qubit pairs of each coupler letter A, B, C, D (see module docstring)."""
    sites, idx = grid_layout(rows, cols, removed)
    layers = {"A": [], "B": [], "C": [], "D": []}
    for r in range(rows):
        for c in range(cols - 1):
            if (r, c) in idx and (r, c + 1) in idx:
                layers["A" if c % 2 == 0 else "B"].append((idx[(r, c)], idx[(r, c + 1)]))
    for r in range(rows - 1):
        for c in range(cols):
            if (r, c) in idx and (r + 1, c) in idx:
                layers["C" if r % 2 == 0 else "D"].append((idx[(r, c)], idx[(r + 1, c)]))
    return layers


PATTERN = "ABCDCDAB"


def _zero_state(d: int) -> np.ndarray:
    v = np.zeros(d, dtype=np.complex128)
    v[0] = 1.0
    return v


def random_grid_circuit(rows: int, cols: int, cycles: int, seed: int,
                        removed: Sequence[Tuple[int, int]] = (),
                        theta: float = math.pi / 2, phi: float = math.pi / 6) -> Circuit:
    """Sycamore-style random circuit: per cycle a random sqrt(X|Y|W) layer, then
    fSim(theta, phi) on the bonds of the cycle's coupler letter."""
    sites, _ = grid_layout(rows, cols, removed)
    n = len(sites)
    layers = coupler_layers(rows, cols, removed)
    rng = SplitMix64(seed)
    one_q = [("sx", sqrt_x()), ("sy", sqrt_y()), ("sw", sqrt_w())]
    prev = [-1] * n
    circ = Circuit(n=n, d=2, initial=[_zero_state(2) for _ in range(n)], sites=sites)
    fs = fsim(theta, phi)
    for t in range(cycles):
        for q in range(n):
            if prev[q] < 0:
                k = rng.randint(3)
            else:
                choices = [j for j in range(3) if j != prev[q]]
                k = choices[rng.randint(2)]
            prev[q] = k
            circ.gates.append(Gate(one_q[k][1], (q,), kind=one_q[k][0]))
        for (a, b) in layers[PATTERN[t % 8]]:
            circ.gates.append(Gate(fs.copy(), (a, b), (theta, phi), kind="fsim"))
    return circ


def param_grid_circuit(rows: int, cols: int, cycles: int, seed: int) -> Circuit:
    """Parameterised grid circuit: per cycle Rz(a)Ry(b) on every qubit with
    a, b ~ U[0, 2pi), then fSim(theta, phi) with theta, phi ~ U[0, pi] on the
    cycle's coupler letter."""
    sites, _ = grid_layout(rows, cols)
    n = len(sites)
    layers = coupler_layers(rows, cols)
    rng = SplitMix64(seed)
    circ = Circuit(n=n, d=2, initial=[_zero_state(2) for _ in range(n)], sites=sites)
    for t in range(cycles):
        for q in range(n):
            a = rng.uniform_range(0.0, 2 * math.pi)
            b = rng.uniform_range(0.0, 2 * math.pi)
            circ.gates.append(Gate(rzry(a, b), (q,), (a, b), kind="rzry"))
        for (p, q) in layers[PATTERN[t % 8]]:
            th = rng.uniform_range(0.0, math.pi)
            ph = rng.uniform_range(0.0, math.pi)
            circ.gates.append(Gate(fsim(th, ph), (p, q), (th, ph), kind="fsim"))
    return circ


def gate_with_params(g: Gate, params: Sequence[float]) -> np.ndarray:
    """Rebuild a parameterised gate's matrix at new parameter values."""
    if g.kind == "rzry":
        return rzry(*params)
    if g.kind == "fsim":
        return fsim(*params)
    raise ValueError(f"gate kind {g.kind!r} has no parameters")


def gate_param_derivs(g: Gate) -> List[np.ndarray]:
    if g.kind == "rzry":
        return list(drzry(*g.params))
    if g.kind == "fsim":
        return list(dfsim(*g.params))
    return []


def random_bitstrings(n: int, count: int, seed: int, d: int = 2) -> np.ndarray:
    """count seeded output patterns, each n digits in [0, d)."""
    rng = SplitMix64(seed)
    return np.array([[rng.randint(d) for _ in range(n)] for _ in range(count)],
                    dtype=np.int32).reshape(count, n)
