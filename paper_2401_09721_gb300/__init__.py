"""GB300 (sm_103a) implementation of FGBD, the fast graph-based point-cloud colour denoiser.

Modules:
  build   compiles the CUDA library libfgbd.so in-tree with nvcc
  fgbd    ctypes binding of the C ABI in include/fgbd.h (no CPU fallback)
  synth   seeded synthetic voxelized frames used by tests and benchmarks

Importing the package loads nothing; ``fgbd.lib()`` loads the library on first use.
"""
__all__ = ["build", "fgbd", "synth"]
