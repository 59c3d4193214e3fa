"""GB300-native (sm_103a) D3Q27 central-moment MRT kinetic solver with direct-forcing
immersed boundaries, after arXiv 2101.11856.

The compute path is the C-ABI CUDA library ``liblbm.so`` (sources in ``csrc/``, header
``include/lbm.h``); ``lbm`` is its thin ctypes binding.  Build with ``build.build()``.
"""
from . import lbm
from .lbm import Solver, LBMError, LBMSolve, lbm_solve

__all__ = ["lbm", "Solver", "LBMError", "LBMSolve", "lbm_solve"]
