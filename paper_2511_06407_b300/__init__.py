"""B300-native (sm_103a) SoftAbs-RMHMC for hierarchical Gaussian-process models.

The compute path is the CUDA library built from ``csrc/`` (``librmhmc.so``, C ABI declared in
``include/rmhmc.h``); ``rmhmc`` is its thin ctypes binding. Importing this package does not load
the library; the first call into ``rmhmc`` does, and raises if it is missing.
"""
__all__ = ["workloads", "rmhmc"]
