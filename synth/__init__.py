"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This package holds input preparation only: random fields and the maps built
from them.  It contains none of the model's arithmetic (no stencil, no solver,
no ODE, no automaton rule), so both sides may use it without sharing method
code.
"""

from .maps import MapSet, biopsy_maps, gaussian_random_field, make_maps, replicate_sizes

__all__ = ["MapSet", "biopsy_maps", "gaussian_random_field", "make_maps", "replicate_sizes"]
