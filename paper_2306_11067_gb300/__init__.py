"""GB300 (sm_103a) multigrid-preconditioned CG for regularized least squares.

The compute path is the CUDA library ``liblcmg.so`` (C ABI in
``include/lcmg.h``); ``lcmg`` is its ctypes binding.
"""
from . import lcmg  # noqa: F401
from .lcmg import Server, Solver, LcmgError  # noqa: F401
