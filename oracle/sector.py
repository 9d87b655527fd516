"""O1 for photon-number-conserving bosonic networks: the FP64 state vector
restricted to one total-photon sector at a time (ctypes over sector.c).
Test infrastructure only."""
import ctypes

import numpy as np

from . import build as _build
from .statevector import gate_arrays, _init

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        P = ctypes.c_void_p
        _lib.oracle_sector_amplitudes.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P, P, P, P,
                                                  ctypes.c_int, P, P, ctypes.c_int64]
        _lib.oracle_sector_amplitudes.restype = ctypes.c_int
        _lib.oracle_sector_dim.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        _lib.oracle_sector_dim.restype = ctypes.c_int64
    return _lib


def sector_dim(n: int, d: int, total: int) -> int:
    """Number of photon patterns of n modes below cutoff d with the given total."""
    return int(_load().oracle_sector_dim(n, d, total))


def sector_amplitudes(circ, patterns, gate_mats=None, init=None, max_dim: int = 1 << 28) -> np.ndarray:
    """<p|U|psi0> for every pattern p, each from the state vector of its own
    total-photon sector.  Raises ValueError if a gate mixes sectors."""
    lib = _load()
    n, d = circ.n, circ.d
    k, q, flat, off = gate_arrays(circ, gate_mats)
    iv = _init(circ, init)
    pats = np.ascontiguousarray(np.atleast_2d(np.asarray(patterns, dtype=np.int32)))
    assert pats.shape[1] == n
    amps = np.zeros(pats.shape[0], dtype=np.complex128)
    rc = lib.oracle_sector_amplitudes(n, d, iv.ctypes.data, len(circ.gates), k.ctypes.data, q.ctypes.data,
                                      flat.ctypes.data, off.ctypes.data, pats.shape[0], pats.ctypes.data,
                                      amps.ctypes.data, int(max_dim))
    if rc == 1:
        raise ValueError("sector_amplitudes: a gate does not conserve the total photon number")
    if rc == 2:
        raise MemoryError("sector_amplitudes: allocation failed")
    if rc == 3:
        raise ValueError("sector_amplitudes: sector larger than max_dim")
    if rc != 0:
        raise ValueError(f"sector_amplitudes: bad sizes (code {rc})")
    return amps
