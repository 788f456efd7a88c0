"""CPU FP64 oracle for the FMM-accelerated Galerkin Poisson-Boltzmann matvec and solve.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or run anything in this package. The CUDA library never calls it
and shares no code with it; the two meet only through the seeded inputs of
``paper_2110_13778_gb300.inputs``.

Modules:
  dense     -- dense Galerkin assembly (C, ``pb_oracle.c``), LU solve, RHS, energy
  kirkwood  -- closed-form and series Kirkwood energies of a dielectric sphere
  taylor    -- Taylor coefficients of G0 / Gk by truncated power-series arithmetic
  fmm       -- the six-step Cartesian FMM of Section 2.4 in plain numpy
  linear    -- the piecewise-linear (continuous hat function) Galerkin system of Section 2.3

Parity status of each function is stated in its module header.
"""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "pb_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (plain -O2, no fused multiply-add contraction)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            c_int, c_double = ctypes.c_int, ctypes.c_double
            L.orc_gauss_legendre01.argtypes = [c_int, dp, dp]
            L.orc_kernel_point.argtypes = [dp, dp, dp, dp, c_double, c_double, dp]
            L.orc_geometry.argtypes = [dp, ip, c_int, dp, dp, dp]
            L.orc_ss_points.argtypes = [c_int, c_double, c_double, c_double, c_double, dp, dp, dp]
            L.orc_ss_points.restype = c_int
            L.orc_pair_integrals.argtypes = [dp, ip, c_int, c_int, c_double, c_double, c_int, c_int, dp, dp, dp, dp]
            L.orc_pair_terms.argtypes = [dp, ip, c_int, c_int, c_double, c_int, dp]
            L.orc_pair_terms.restype = c_int
            L.orc_assemble.argtypes = [dp, ip, c_int, c_double, c_double, c_int, c_int, dp, dp, dp, dp]
            L.orc_rows_matvec.argtypes = [dp, ip, c_int, c_double, c_double, c_int, c_int, dp, dp, dp, c_int, ip, dp,
                                          dp]
            L.orc_rhs.argtypes = [dp, ip, c_int, dp, dp, c_int, c_double, c_int, dp, dp, dp, dp]
            L.orc_energy.argtypes = [dp, ip, c_int, dp, dp, c_int, c_double, c_double, c_int, dp, dp, dp, dp]
            L.orc_energy.restype = c_double
            L.orc_p1_pair_integrals.argtypes = [dp, ip, c_int, c_int, c_double, c_double, c_int, c_int, dp, dp, dp,
                                                dp]
            L.orc_p1_pair_terms.argtypes = [dp, ip, c_int, c_int, c_double, c_int, dp]
            L.orc_p1_pair_terms.restype = c_int
            L.orc_p1_matvec.argtypes = [dp, ip, c_int, c_int, c_double, c_double, c_int, c_int, dp, dp, dp, dp, dp]
            L.orc_p1_assemble.argtypes = [dp, ip, c_int, c_int, c_double, c_double, c_int, c_int, dp, dp, dp, dp]
            L.orc_p1_rhs.argtypes = [dp, ip, c_int, c_int, dp, dp, c_int, c_double, c_int, dp, dp, dp, dp]
            L.orc_p1_energy.argtypes = [dp, ip, c_int, c_int, dp, dp, c_int, c_double, c_double, c_int, dp, dp, dp,
                                        dp]
            L.orc_p1_energy.restype = c_double
            _lib = L
    return _lib
