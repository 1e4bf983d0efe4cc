"""Seeded synthetic inputs shared by the FP64 oracle tests, the GPU tests and the bench.

This package only draws geometry (solid indicator phi0 and initial fluid
fraction phi1 on the lattice) from the paper's initial-condition recipes.  It
holds none of the lattice Boltzmann arithmetic: neither the oracle nor the CUDA
library imports anything else from the other side.
"""
from .geometry import *  # noqa: F401,F403
