"""GB300-native (sm_103a) SPH-with-boids step: CUDA kernels behind a C ABI.

Modules:
  scenes -- seeded synthetic workloads (inputs only)
  sph    -- ctypes binding of libsph_gb300.so (same names as include/sph.h)
  build  -- in-tree nvcc build of the library
"""
__all__ = ["scenes", "sph", "build"]
