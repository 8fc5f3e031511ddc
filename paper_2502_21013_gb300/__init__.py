"""GB300-native solver for nonlinear degenerate time-periodic parabolic problems.

The compute path is libptp.so (hand-written CUDA for sm_103a behind the C ABI
of include/ptp.h); `paper_2502_21013_gb300.ptp` is its ctypes binding.
Importing the binding raises if the library has not been built.
"""
__all__ = ["ptp", "build"]
