"""GB300-native (sm_103a) D3Q19 pseudo-potential lattice Boltzmann step.

The compute path is the CUDA library liblbm.so (C ABI in include/lbm.h),
built in-tree by ``paper_1904_11792_gb300.build.build()``; ``lbm`` is its
ctypes binding.  There is no CPU fallback: ``lbm.load()`` raises when the
library has not been built, and every lattice call fails without a GB300.
"""
from . import build, lbm  # noqa: F401

__all__ = ["build", "lbm"]
