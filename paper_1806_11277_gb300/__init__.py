"""GB300-native elastic Helmholtz shifted-Laplacian multigrid / DD solver.

The compute path is libehs.so (CUDA, sm_103a) behind the C ABI in
include/ehs.h; ``ehs`` is its ctypes binding and ``synth`` generates seeded
synthetic media.  See ``ehs.Solver``.
"""
