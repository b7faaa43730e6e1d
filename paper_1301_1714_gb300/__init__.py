"""GB300-native soft-sphere DEM timestep (Washizawa & Nakahara, "Parallel Computing of
Discrete Element Method on GPU").

Submodules:
  dem      Python binding of the C ABI (include/dem.h, libdemgb.so)
  scenes   seeded synthetic inputs (particles, walls, parameters)
  _build   in-tree nvcc build of libdemgb.so for sm_103a
Importing the package loads nothing; `dem.lib()` loads the CUDA library.
"""
__all__ = ["dem", "scenes"]
