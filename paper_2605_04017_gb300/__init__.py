"""GB300-native lens transport (Precomputed Lens Transport Maps).

The compute path is liblt.so (hand-written sm_103a CUDA kernels behind the
C ABI in include/lt.h); ``lt`` is its ctypes binding and ``workloads`` the
seeded synthetic inputs.
"""
__all__ = ["lt", "workloads", "build"]
