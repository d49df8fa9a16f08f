"""GB300-native cascaded D3Q19 lattice Boltzmann method for power-law fluids.

The compute path is the C-ABI library ``libclbm.so`` (hand-written sm_103a
CUDA, declared in ``include/clbm.h``); ``clbm`` is its ctypes binding.
"""
from . import build  # noqa: F401

__all__ = ["build", "clbm"]
