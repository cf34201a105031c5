"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA library.

Only input generation lives here: counter-based random numbers, SU(3) links
U = exp(i*eps*A) with A = sum_a c_a lambda_a/2 (c_a ~ N(0,1)), Gaussian and
point sources.  No operator arithmetic.  The numerics are in ``gen.c``; this
file compiles it on first use and wraps it with numpy.

Canonical layouts (numpy complex128, x fastest in memory):
  links   (L3, L2, L1, L0, 4, 3, 3)   = [t][z][y][x][mu][row][col]
  spinors (nrhs, L3, L2, L1, L0, 4, 3) = [rhs][t][z][y][x][spin][colour]
``dims`` is always (L0, L1, L2, L3) = (x, y, z, t).

Seed convention for the standard workloads: gauge seed 1000+k and source seed
2000+k for workload k; batched lattice j uses gauge seed 3000+j.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libgen.so beside it (gcc, portable flags only)."""
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.gen_uniform.argtypes = [ctypes.c_long, ctypes.c_uint64, dp]
            lib.gen_gaussian.argtypes = [ctypes.c_long, ctypes.c_uint64, dp]
            lib.gen_su3.argtypes = [ctypes.c_long, ctypes.c_double, ctypes.c_uint64, dp]
            lib.gen_su3_generator.argtypes = [ctypes.c_long, ctypes.c_uint64, dp]
            lib.gen_gauge.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_uint64, dp]
            for f in (lib.gen_uniform, lib.gen_gaussian, lib.gen_su3, lib.gen_su3_generator, lib.gen_gauge):
                f.restype = None
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    assert a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def volume(dims) -> int:
    return int(dims[0]) * int(dims[1]) * int(dims[2]) * int(dims[3])


def uniform(n: int, seed: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().gen_uniform(n, seed, _dptr(out))
    return out


def gaussian(n: int, seed: int) -> np.ndarray:
    """n independent N(0,1) reals (Box-Muller on SplitMix64 counters)."""
    out = np.empty(n, dtype=np.float64)
    _load().gen_gaussian(n, seed, _dptr(out))
    return out


def su3_matrices(n: int, eps: float, seed: int) -> np.ndarray:
    """n matrices exp(i*eps*A), shape (n, 3, 3) complex128."""
    out = np.empty((n, 3, 3), dtype=np.complex128)
    _load().gen_su3(n, float(eps), seed, _dptr(out.view(np.float64)))
    return out


def su3_generator(k: int, seed: int) -> np.ndarray:
    """The Hermitian traceless A of matrix number k of stream ``seed``."""
    out = np.empty((3, 3), dtype=np.complex128)
    _load().gen_su3_generator(k, seed, _dptr(out.view(np.float64)))
    return out


def gauge_field(dims, eps: float, seed: int) -> np.ndarray:
    """Links U_mu(x) = exp(i*eps*A), shape (L3, L2, L1, L0, 4, 3, 3)."""
    L = [int(d) for d in dims]
    out = np.empty((L[3], L[2], L[1], L[0], 4, 3, 3), dtype=np.complex128)
    arr = (ctypes.c_int * 4)(*L)
    _load().gen_gauge(arr, float(eps), seed, _dptr(out.view(np.float64)))
    return out


def unit_gauge(dims) -> np.ndarray:
    L = [int(d) for d in dims]
    out = np.zeros((L[3], L[2], L[1], L[0], 4, 3, 3), dtype=np.complex128)
    out[..., 0, 0] = out[..., 1, 1] = out[..., 2, 2] = 1.0
    return out


def gaussian_spinor(dims, seed: int, nrhs: int = 1) -> np.ndarray:
    """Every real component ~ N(0,1); shape (nrhs, L3, L2, L1, L0, 4, 3)."""
    L = [int(d) for d in dims]
    n = nrhs * volume(L) * 24
    re = gaussian(n, seed)
    return re.view(np.complex128).reshape(nrhs, L[3], L[2], L[1], L[0], 4, 3)


def point_sources(dims, site=(0, 0, 0, 0)) -> np.ndarray:
    """The 12 spin-colour point sources delta_{x,site} e_(s,c); shape (12, ...)."""
    L = [int(d) for d in dims]
    out = np.zeros((12, L[3], L[2], L[1], L[0], 4, 3), dtype=np.complex128)
    x0, x1, x2, x3 = site
    for s in range(4):
        for c in range(3):
            out[3 * s + c, x3, x2, x1, x0, s, c] = 1.0
    return out
