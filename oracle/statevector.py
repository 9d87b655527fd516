"""O1: FP64 state-vector route (ctypes over sv.c).  Test infrastructure only."""
import ctypes
from typing import List, Optional, Sequence

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        P = ctypes.c_void_p
        _lib.oracle_sv_run.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P, P, P, P, P]
        _lib.oracle_sv_run.restype = None
        _lib.oracle_sv_env.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P, P, P, P, P, P]
        _lib.oracle_sv_env.restype = ctypes.c_int
    return _lib


def gate_arrays(circ, gate_mats: Optional[Sequence[np.ndarray]] = None):
    """Flatten a circuit's gate list into the arrays sv.c reads."""
    mats = gate_mats if gate_mats is not None else [g.matrix for g in circ.gates]
    k = np.array([len(g.qubits) for g in circ.gates], dtype=np.int32)
    q = np.zeros(2 * len(circ.gates), dtype=np.int32)
    for i, g in enumerate(circ.gates):
        q[2 * i:2 * i + len(g.qubits)] = g.qubits
    sizes = np.array([np.asarray(m).size for m in mats], dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    flat = np.concatenate([np.asarray(m, dtype=np.complex128).ravel() for m in mats]) \
        if len(mats) else np.zeros(0, np.complex128)
    return k, q, np.ascontiguousarray(flat), off


def _init(circ, init: Optional[Sequence[np.ndarray]]):
    vecs = init if init is not None else circ.initial
    return np.ascontiguousarray(np.concatenate([np.asarray(v, np.complex128) for v in vecs]))


def sv_state(circ, gate_mats=None, init=None) -> np.ndarray:
    """Final state U|psi0> as a d^n complex128 vector (qudit 0 most significant)."""
    lib = _load()
    n, d = circ.n, circ.d
    k, q, flat, off = gate_arrays(circ, gate_mats)
    iv = _init(circ, init)
    psi = np.empty(d ** n, dtype=np.complex128)
    lib.oracle_sv_run(n, d, iv.ctypes.data, len(circ.gates), k.ctypes.data, q.ctypes.data,
                      flat.ctypes.data, off.ctypes.data, psi.ctypes.data)
    return psi


def index_of(pattern: Sequence[int], d: int) -> int:
    x = 0
    for v in pattern:
        x = x * d + int(v)
    return x


def sv_amplitudes(circ, patterns, gate_mats=None, init=None) -> np.ndarray:
    psi = sv_state(circ, gate_mats, init)
    return np.array([psi[index_of(p, circ.d)] for p in np.atleast_2d(patterns)])


def sv_env(circ, patterns, cot, gate_mats=None, init=None) -> List[np.ndarray]:
    """Per gate g: env_g = sum_b cot_b d amp_b / d U_g  (a (d^k, d^k) matrix)."""
    lib = _load()
    n, d = circ.n, circ.d
    k, q, flat, off = gate_arrays(circ, gate_mats)
    iv = _init(circ, init)
    lam = np.zeros(d ** n, dtype=np.complex128)
    for p, c in zip(np.atleast_2d(patterns), np.atleast_1d(cot)):
        lam[index_of(p, d)] += c
    env = np.zeros_like(flat)
    rc = lib.oracle_sv_env(n, d, iv.ctypes.data, len(circ.gates), k.ctypes.data, q.ctypes.data,
                           flat.ctypes.data, off.ctypes.data, lam.ctypes.data, env.ctypes.data)
    if rc != 0:
        raise MemoryError("oracle_sv_env: allocation failed")
    out = []
    for g, gate in enumerate(circ.gates):
        m = d ** len(gate.qubits)
        out.append(env[off[g]:off[g] + m * m].reshape(m, m).copy())
    return out
