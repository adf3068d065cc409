"""GB300-native (sm_103a) exact multi-limb integer add / sub / mul after
DigitsOnTurbo (arxiv 2604.21566): carry-decoupled addition with warp-ballot
lookahead and decoupled look-back, and column-sum multiplication with a
separate carry-resolution pass.

The compute lives in libdot.so (CUDA kernels behind the C ABI of
include/dot.h); ``dot`` is its thin ctypes binding and ``workloads`` holds
the seeded synthetic input generators.
"""
__all__ = ["dot", "workloads", "build"]
