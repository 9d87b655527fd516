"""Seeded synthetic workloads: random grid circuits, a parameterised circuit and a
2-D Gaussian-boson-sampling (GBS) lattice, plus the circuit -> tensor-network
mapping of Section 2.2.1 (one tensor per gate, one rank-1 tensor per initial
|0>, open legs for the output qudits).

This module holds the inputs only.  It performs no contraction, no slicing and
no reduction: both the CUDA path and the FP64 oracle consume the tensors it
builds, so that the two sides see bit-identical operands.
"""
from .rng import SplitMix64
from .rqc import (Circuit, Gate, grid_layout, coupler_layers, random_grid_circuit,
                  param_grid_circuit, fsim, sqrt_x, sqrt_y, sqrt_w, rz, ry, rzry,
                  random_bitstrings)
from .gbs import gbs_lattice_circuit, gbs_nd_circuit, squeezed_vacuum, beamsplitter, random_patterns
from .network import TensorNetwork, circuit_to_network
from . import configs

__all__ = [
    "SplitMix64", "Circuit", "Gate", "grid_layout", "coupler_layers",
    "random_grid_circuit", "param_grid_circuit", "fsim", "sqrt_x", "sqrt_y", "sqrt_w",
    "rz", "ry", "rzry", "random_bitstrings", "gbs_lattice_circuit", "gbs_nd_circuit", "squeezed_vacuum",
    "beamsplitter", "random_patterns", "TensorNetwork", "circuit_to_network", "configs",
]
