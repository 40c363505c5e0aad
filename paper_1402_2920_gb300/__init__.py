"""GB300 library for the consistent two-phase lattice Boltzmann method
(Zelko & Duenweg, arXiv:1402.2920): the per-time-step update on D2Q21 and
D3Q59 as hand-written CUDA kernels behind a C ABI (include/lbm.h).

``lbm`` is the thin ctypes binding (same names as the C functions);
``workloads`` builds the seeded synthetic inputs.
"""
from . import lbm  # noqa: F401
from .lbm import *  # noqa: F401,F403
