"""GB300-native D3Q27 central-moment lattice Boltzmann solver with external forcing
(De Rosis, Huang & Coreixas, arXiv 1905.10182).

The compute path is the CUDA library libcmlbm.so (C ABI in include/cmlbm.h); ``Solver`` is a
thin binding over it.  ``build()`` compiles the library for sm_103a.
"""
from .buildlib import build  # noqa: F401
from .solver import BatchSolver, Solver  # noqa: F401
