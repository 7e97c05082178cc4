"""GB300-native (sm_103a) FS-1: Sinkhorn for the Wasserstein-1 metric on uniform
grids with O(N) recurrences (Liao et al., "Fast Sinkhorn I").

Layout
  csrc/      CUDA kernels and the host runtime behind the C ABI (include/fs1.h)
  build.py   in-tree nvcc build of csrc/ into _build/libfs1.so
  fs1.py     ctypes binding with the C names, and a torch-facing Solver
  inputs.py  seeded synthetic histograms of the workloads (no solver arithmetic)

Importing the package does not load the CUDA library; ``fs1.load()`` does, and
raises if it was not built.
"""
__all__ = ["build", "fs1", "inputs"]
