"""GB300-native FMM-accelerated Galerkin boundary-integral Poisson-Boltzmann solver.

The compute path is the CUDA library ``libpb.so`` (C ABI in ``include/pb.h``), built from
``csrc/`` by ``paper_2110_13778_gb300.build``; ``paper_2110_13778_gb300.pb`` is its ctypes
binding and ``inputs`` holds the seeded synthetic inputs.
"""
__all__ = ["pb", "inputs", "build"]
