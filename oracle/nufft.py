"""Python side of O2, the Gaussian-gridding NUFFT of Section 2 (C code in gauss_nufft.c).

TEST INFRASTRUCTURE ONLY.  Parameter settings:
  * "parity"  sigma = 3, w = 28, tau = 5.5 / N^2.  Per axis the aliasing error is
                exp(-sigma (sigma-1) N^2 tau) = e^-33, the truncation error
                exp(-(w pi / (sigma N))^2 / (4 tau)) = e^-39, and FP64 rounding is amplified by
                the deconvolution factor exp(N^2 tau / 4) <= e^1.4 per axis (about 1e-14 in 3D);
  * "fine"    sigma = 2, w = 24, tau = (w pi / sigma) / (2 N^2 sqrt(sigma (sigma - 1))), which
                balances aliasing against truncation (about 1e-11 in 3D, limited by rounding
                amplified by exp(3 N^2 tau / 4) at the corner modes);
  * "fp32ref" sigma = 2, w = 16, tau balanced as for "fine" (0.6-1.0e-8 against the direct
                sums on 12^3, 16^3 and 32^2 grids, pinned below 3e-8): a reference for FP32
                results at a third of the cost of "fine";
  * "paper12" the paper's 12-digit setting: Mr = 2N, tau = 12 / N^2, 24 points;
  * "paper6"  the paper's 6-digit setting:  Mr = 2N, tau = 6 / N^2, 12 points.
The balanced tau is this project's reading (the paper states only the two settings above);
every setting is checked against the direct sums of ``oracle.direct``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gauss_nufft.c")
_LIB = os.path.join(_HERE, "liboracle_nufft.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, OpenMP); returns the shared-library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_fft.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int]
        lib.orc_type2.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_long, dp, dp,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int]
        lib.orc_type1.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_long, dp, dp, dp,
                                  ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())


def params(N: int, setting: str = "parity"):
    """(Mr, w, tau) for a grid of N modes per axis."""
    if setting == "parity":
        return 3 * N, 28, 5.5 / N ** 2
    if setting in ("fine", "fp32ref"):
        sigma, w = 2, (24 if setting == "fine" else 16)
        tau = (w * np.pi / sigma) / (2.0 * N ** 2 * np.sqrt(sigma * (sigma - 1.0)))
        return sigma * N, w, tau
    if setting == "paper12":
        return 2 * N, 24, 12.0 / N ** 2
    if setting == "paper6":
        return 2 * N, 12, 6.0 / N ** 2
    raise ValueError(setting)


def fft(x: np.ndarray, sign: int) -> np.ndarray:
    """d-dimensional DFT of a cubic complex array with kernel exp(sign 2 pi i j k / n)."""
    a = np.ascontiguousarray(x, dtype=np.complex128).copy()
    Mr = a.shape[0]
    _load().orc_fft(a.ndim, Mr, int(sign), _ptr(a.view(np.float64)), threads())
    return a


def type2(f: np.ndarray, t: np.ndarray, setting: str = "parity", nthreads: int | None = None):
    """F_j = sum_m f_m exp(-i t_j . m), m in [-N/2, N/2)^d (array index i = m + N/2)."""
    f = np.ascontiguousarray(f, dtype=np.complex128)
    d, N = f.ndim, f.shape[0]
    t = np.ascontiguousarray(t, dtype=np.float64)
    Mr, w, tau = params(N, setting)
    out = np.empty(t.shape[0], dtype=np.complex128)
    rc = _load().orc_type2(d, N, _ptr(f.view(np.float64)), t.shape[0], _ptr(t),
                           _ptr(out.view(np.float64)), Mr, w, tau, nthreads or threads())
    if rc != 0:
        raise RuntimeError(f"orc_type2 failed ({rc})")
    return out


def type1(c: np.ndarray, t: np.ndarray, d: int, N: int, setting: str = "parity",
          nthreads: int | None = None):
    """u_m = sum_j c_j exp(+i t_j . m) on the N^d modes (complex array)."""
    c = np.ascontiguousarray(c, dtype=np.complex128)
    t = np.ascontiguousarray(t, dtype=np.float64)
    Mr, w, tau = params(N, setting)
    out = np.empty((N,) * d, dtype=np.complex128)
    rc = _load().orc_type1(d, N, t.shape[0], _ptr(t), _ptr(c.view(np.float64)),
                           _ptr(out.view(np.float64)), Mr, w, tau, nthreads or threads())
    if rc != 0:
        raise RuntimeError(f"orc_type1 failed ({rc})")
    return out
