"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package only *generates* inputs: gate matrices, random grid circuits of the
paper's gate family (Sec. 6: Sycamore-style random quantum circuits), the
translation of a circuit into a tensor network (Sec. 2.1.1: tensors are
vertices, indices are edges) and contraction paths given as input (the paper
takes its paths from an external path finder). It performs no contraction, no
slicing and no planning of slices, so it holds none of the method's
arithmetic; both the oracle and the library consume what it produces.
"""

from .gates import sqrt_x, sqrt_y, sqrt_w, fsim, hadamard, cnot, cz, s_gate, identity2
from .circuits import Circuit, Gate, grid_rqc, lattice_53q_rqc, coupler_layers
from .network import TensorNetwork, circuit_to_network, projection_leaves, random_bitstrings, bitstring_variants
from .paths import stem_path

__all__ = [
    "sqrt_x", "sqrt_y", "sqrt_w", "fsim", "hadamard", "cnot", "cz", "s_gate",
    "identity2", "Circuit", "Gate", "grid_rqc", "lattice_53q_rqc",
    "coupler_layers", "TensorNetwork", "circuit_to_network", "stem_path",
    "projection_leaves", "random_bitstrings", "bitstring_variants",
]
