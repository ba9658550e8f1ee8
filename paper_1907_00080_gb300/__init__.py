"""GB300-native LB-IB solver for red cells and adhesive carriers in a capillary.

Submodules:
  lbib    -- ctypes binding of the C ABI (include/lbib.h) of liblbib.so
  build   -- nvcc build of liblbib.so for sm_103a
  inputs  -- seeded synthetic workloads (geometry and parameters only)
  tuning  -- tile-shape choice for the fused kernel
"""
__all__ = ["lbib", "build", "inputs", "tuning"]
