"""FP64 CPU oracle of the two-phase lattice Boltzmann step (test infrastructure only).

Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py may
import this package.  The CUDA library and its Python binding never do.
"""
