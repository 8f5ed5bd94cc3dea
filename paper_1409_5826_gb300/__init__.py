"""GB300-native batched explicit asymptotic integration of reaction networks.

The integrator runs in hand-written sm_103a CUDA kernels behind the C ABI in
include/kn.h (libkn.so, built in-tree by ``paper_1409_5826_gb300.build``);
``paper_1409_5826_gb300.kn`` is the ctypes binding.  Importing this package
loads nothing; the first call into ``kn`` loads libkn.so and raises if it is
missing.
"""
__all__ = ["kn", "build"]
