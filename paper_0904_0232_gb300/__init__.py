"""GB300-native GRPIC hot path (general-relativistic electromagnetic particle-in-cell in
Cartesian Kerr-Schild coordinates, after Watson & Nishikawa, arXiv:0904.0232).

The timestep runs in hand-written CUDA kernels for sm_103a behind the C ABI of
include/grpic.h (libgrpic.so, built by ``paper_0904_0232_gb300.build``); ``grpic`` is its
ctypes binding and ``synth`` the seeded input generators.
"""
from . import synth  # noqa: F401
from .grpic import GrpicError, Simulation, load_library  # noqa: F401
