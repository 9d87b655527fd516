"""The synthetic workloads (sizes, seeds and parameter ranges).

  grid12  : 12-qubit 3x4 grid, 8 cycles, fSim(pi/2, pi/6), one bitstring, no slicing
  grid30  : 30-qubit 5x6 grid, 14 cycles, 6 sliced indices (64 slices), max 2^24
  grid53  : 53 qubits (9x6 minus corner (0,0)), 12 cycles, max intermediate 2^28
  param20 : 20-qubit 4x5 parameterised circuit, 12 cycles, 64 bitstrings, loss = sum |amp|^2
  gbs16   : 16 modes on 4x4, Fock cutoff 4, 4 beamsplitter layers, 256 photon patterns
  gbs3d   : 18 modes on a 2x3x3 lattice, Fock cutoff 4, 2 beamsplitter layers, 16 photon patterns
  gbs88d8 : 64 modes on 8x8, Fock cutoff 8, 1 beamsplitter layer, r = 0.5, one pattern with
            every mode in [0, 4) (the 2-D lattice the paper times, at its larger cutoff)
"""
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np

from .rqc import random_grid_circuit, param_grid_circuit, random_bitstrings
from .gbs import gbs_lattice_circuit, gbs_nd_circuit, random_patterns
from .network import circuit_to_network


@dataclass
class Workload:
    name: str
    circuit: object
    network: object
    outputs: np.ndarray            # (n_amps, n_qudits) int32
    n_sliced: int                  # number of sliced indices (0 = none)
    max_elems: Optional[int]       # intermediate-size cap that drives slicing
    seed: int


SPECS = {
    "grid12": dict(kind="rqc", rows=3, cols=4, cycles=8, seed=1, n_amps=1, n_sliced=0, max_elems=None),
    "grid30": dict(kind="rqc", rows=5, cols=6, cycles=14, seed=2, n_amps=1, n_sliced=6, max_elems=1 << 24),
    "grid53": dict(kind="rqc", rows=9, cols=6, cycles=12, seed=3, n_amps=1, n_sliced=None,
                   max_elems=1 << 28, removed=((0, 0),)),
    "param20": dict(kind="param", rows=4, cols=5, cycles=12, seed=4, n_amps=64, n_sliced=0, max_elems=None),
    "gbs16": dict(kind="gbs", rows=4, cols=4, cycles=4, seed=5, n_amps=256, n_sliced=0, max_elems=None, d=4),
    "gbs3d": dict(kind="gbsnd", shape=(2, 3, 3), cycles=2, seed=6, n_amps=16, n_sliced=0, max_elems=None, d=4),
    "gbs88d8": dict(kind="gbsnd", shape=(8, 8), cycles=1, seed=7, n_amps=1, n_sliced=0, max_elems=None, d=8,
                    r_range=(0.5, 0.5), pattern_max=4),
}


def build(name: str, **override) -> Workload:
    spec = dict(SPECS[name])
    spec.update(override)
    kind = spec["kind"]
    if kind == "rqc":
        circ = random_grid_circuit(spec["rows"], spec["cols"], spec["cycles"], spec["seed"],
                                   removed=spec.get("removed", ()))
        outs = random_bitstrings(circ.n, spec["n_amps"], spec["seed"] + 1000)
    elif kind == "param":
        circ = param_grid_circuit(spec["rows"], spec["cols"], spec["cycles"], spec["seed"])
        outs = random_bitstrings(circ.n, spec["n_amps"], spec["seed"] + 1000)
    elif kind == "gbs":
        circ = gbs_lattice_circuit(spec["rows"], spec["cols"], spec["d"], spec["cycles"], spec["seed"])
        outs = random_patterns(circ.n, spec["n_amps"], spec["seed"] + 1000, spec["d"])
    elif kind == "gbsnd":
        circ = gbs_nd_circuit(spec["shape"], spec["d"], spec["cycles"], spec["seed"],
                              r_range=spec.get("r_range", (0.5, 1.0)))
        outs = random_patterns(circ.n, spec["n_amps"], spec["seed"] + 1000, spec.get("pattern_max", spec["d"]))
    else:
        raise ValueError(kind)
    return Workload(name, circ, circuit_to_network(circ), outs, spec["n_sliced"] or 0,
                    spec["max_elems"], spec["seed"])
