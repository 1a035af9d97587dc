"""GB300-native LDPM explicit central-difference step (arXiv 2603.13190).

Modules:
  specimen   seeded synthetic specimens (placement, Delaunay mesh, 12-facet tessellation)
  workloads  material parameters, boundary conditions and the synthetic benchmark workloads
  ldpm       ctypes binding of libldpm.so (the CUDA library; entry points of include/ldpm.h)
  build      in-tree nvcc build of libldpm.so for sm_103a
"""
