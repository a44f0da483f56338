"""GB300-native SANS Fourier sums (NuMagSANS hot path) behind a C ABI.

Submodules:
  nms     -- ctypes binding of libnms (include/nms.h), same function names.
  inputs  -- seeded synthetic real-space fields shaped like the paper's workloads.
  build   -- in-tree nvcc build of libnms.so for sm_103a.
"""
__all__ = ["nms", "inputs", "build"]
