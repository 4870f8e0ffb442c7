"""GB300-native free-space Coulomb / dipole convolution (Jiang, Greengard & Bao, Algorithm 1).

Thin Python binding over the C-ABI in ``include/nlint.h`` (``libnlint.so``).  The binding only
marshals arguments: every step of the computation runs in the library's CUDA kernels.  PyTorch
is used for device memory and streams.  There is no CPU fallback: if the library is missing or
fails to load, importing the binding raises.

    plan = Plan(d=3, n=256, L=32.0, kernel="coulomb", eps=1e-6)   # FP32 path
    u, E = plan.eval_energy(rho, lam=1.0)                           # rho: CUDA tensor (n,n,n)
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnlint.so")

NLINT_COULOMB, NLINT_DIPOLE = 0, 1
NLINT_FP32, NLINT_FP64 = 0, 1
STATUS = {0: "NLINT_OK", -1: "NLINT_EINVAL", -2: "NLINT_ENOMEM", -3: "NLINT_ECUDA",
          -4: "NLINT_ETIMEOUT", -5: "NLINT_EUNSUPPORTED"}

EXPORTED = [
    "nlint_params_default", "nlint_plan_create", "nlint_plan_create_ex", "nlint_plan_info",
    "nlint_plan_check",
    "nlint_plan_destroy", "nlint_eval", "nlint_eval_energy", "nlint_energy", "nlint_eval_host",
    "nlint_eval_host_many",
    "nlint_type2", "nlint_type1", "nlint_plan_nodes", "nlint_set_stage_timing",
    "nlint_stage_times", "nlint_launch_count", "nlint_energy_noalloc", "nlint_batch_create",
    "nlint_batch_eval", "nlint_batch_info", "nlint_batch_destroy", "nlint_autotune",
    "nlint_autotune_batch",
    "nlint_energy_only", "nlint_plan_toeplitz", "nlint_eval_toeplitz", "nlint_last_error",
]


class NlintError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class nlint_params(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.c_int64), ("L", ctypes.c_double),
                ("kernel", ctypes.c_int), ("axis", ctypes.c_double * 3),
                ("n_r", ctypes.c_int64), ("n_theta", ctypes.c_int64), ("n_phi", ctypes.c_int64),
                ("P", ctypes.c_double), ("eps", ctypes.c_double), ("precision", ctypes.c_int),
                ("w", ctypes.c_int), ("sigma", ctypes.c_double), ("device", ctypes.c_int),
                ("axis2", ctypes.c_double * 3), ("alpha", ctypes.c_double),
                ("max_sub", ctypes.c_int), ("crowd_min", ctypes.c_int),
                ("algorithm", ctypes.c_int), ("pu_a", ctypes.c_double),
                ("pu_r0", ctypes.c_double), ("pu_r1", ctypes.c_double), ("P2", ctypes.c_double),
                ("bin_shape", ctypes.c_int), ("fft_sched", ctypes.c_int)]


class nlint_tune_report(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int), ("max_sub", ctypes.c_int), ("err", ctypes.c_double),
                ("ms", ctypes.c_double), ("from_cache", ctypes.c_int), ("bin_shape", ctypes.c_int),
                ("w_alt", ctypes.c_int), ("err_alt", ctypes.c_double), ("fft_sched", ctypes.c_int)]


class nlint_batch_tune_report(ctypes.Structure):
    _fields_ = [("choice", ctypes.c_int), ("classes", ctypes.c_int), ("ms", ctypes.c_double * 3)]


class nlint_info(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("precision", ctypes.c_int), ("w", ctypes.c_int),
                ("kernel", ctypes.c_int), ("n", ctypes.c_int64), ("n_fine", ctypes.c_int64),
                ("n_nodes", ctypes.c_int64), ("n_half_nodes", ctypes.c_int64),
                ("n_r", ctypes.c_int64), ("n_theta", ctypes.c_int64), ("n_phi", ctypes.c_int64),
                ("L", ctypes.c_double), ("h", ctypes.c_double), ("P", ctypes.c_double),
                ("sigma", ctypes.c_double), ("beta", ctypes.c_double),
                ("workspace_bytes", ctypes.c_size_t), ("n_bins", ctypes.c_int64),
                ("n_subproblems", ctypes.c_int64), ("n_crowd_bins", ctypes.c_int64),
                ("bin", ctypes.c_int * 3), ("device", ctypes.c_int),
                ("algorithm", ctypes.c_int), ("pu_a", ctypes.c_double),
                ("pu_r0", ctypes.c_double), ("pu_r1", ctypes.c_double), ("P2", ctypes.c_double),
                ("toeplitz", ctypes.c_int), ("bin_shape", ctypes.c_int), ("fft_sched", ctypes.c_int)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libnlint.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libnlint.so not found at {path}; run __graft_entry__.build() "
                          "or python paper_1311_4120_gb300/build.py")
    lib = ctypes.CDLL(path)
    vp, i64, dbl, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    pplan = ctypes.POINTER(vp)
    lib.nlint_params_default.argtypes = [ctypes.POINTER(nlint_params)]
    lib.nlint_params_default.restype = None
    lib.nlint_plan_create.argtypes = [ci, i64, dbl, ci, ctypes.POINTER(dbl), dbl, pplan]
    lib.nlint_plan_create_ex.argtypes = [ctypes.POINTER(nlint_params), pplan]
    lib.nlint_plan_info.argtypes = [vp, ctypes.POINTER(nlint_info)]
    lib.nlint_plan_check.argtypes = [vp]
    lib.nlint_plan_destroy.argtypes = [vp]
    lib.nlint_plan_destroy.restype = None
    lib.nlint_eval.argtypes = [vp, vp, vp, vp]
    lib.nlint_eval_energy.argtypes = [vp, vp, vp, dbl, vp, vp]
    lib.nlint_energy.argtypes = [vp, vp, vp, dbl, vp, ctypes.POINTER(dbl), vp]
    lib.nlint_eval_host.argtypes = [vp, vp, vp, dbl, ctypes.POINTER(dbl), vp]
    lib.nlint_eval_host_many.argtypes = [vp, ci, ctypes.POINTER(vp), ctypes.POINTER(vp), dbl,
                                         ctypes.POINTER(dbl), vp]
    lib.nlint_type2.argtypes = [vp, vp, vp, vp]
    lib.nlint_type1.argtypes = [vp, vp, vp, vp]
    lib.nlint_plan_nodes.argtypes = [vp, vp, vp]
    lib.nlint_set_stage_timing.argtypes = [vp, ci]
    lib.nlint_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_char_p), ci, ctypes.POINTER(ci)]
    lib.nlint_launch_count.argtypes = [vp, ctypes.POINTER(i64)]
    lib.nlint_energy_noalloc.argtypes = [ci, i64, dbl, ci, vp, vp, dbl, vp, vp]
    lib.nlint_batch_create.argtypes = [ci, ctypes.POINTER(vp), ci, pplan]
    lib.nlint_batch_eval.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), dbl, vp, vp]
    lib.nlint_batch_info.argtypes = [vp, ctypes.POINTER(ci), ctypes.POINTER(ci), ctypes.POINTER(i64)]
    lib.nlint_batch_destroy.argtypes = [vp]
    lib.nlint_batch_destroy.restype = None
    lib.nlint_autotune.argtypes = [ctypes.POINTER(nlint_params), dbl, ctypes.c_char_p,
                                   ctypes.POINTER(nlint_params), ctypes.POINTER(nlint_tune_report)]
    lib.nlint_autotune_batch.argtypes = [ci, ctypes.POINTER(nlint_params), dbl, ctypes.c_char_p, ci,
                                         ctypes.POINTER(nlint_params),
                                         ctypes.POINTER(nlint_tune_report),
                                         ctypes.POINTER(nlint_batch_tune_report)]
    lib.nlint_energy_only.argtypes = [vp, vp, dbl, vp, ctypes.POINTER(dbl), vp]
    lib.nlint_plan_toeplitz.argtypes = [vp, vp]
    lib.nlint_eval_toeplitz.argtypes = [vp, vp, vp, dbl, vp, vp]
    lib.nlint_last_error.argtypes = []
    lib.nlint_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("nlint_params_default", "nlint_plan_destroy", "nlint_last_error",
                        "nlint_batch_destroy"):
            getattr(lib, name).restype = ci
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        msg = load_library().nlint_last_error().decode(errors="replace")
        raise NlintError(rc, msg)


def _torch():
    import torch
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def make_params(d: int, n: int, L: float, kernel: str = "coulomb", axis=None, axis2=None,
                alpha: float = 0.0, eps: float = 1e-6, precision: Optional[str] = None, nodes=None,
                w: int = 0, sigma: float = 0.0, P: float = 0.0, device: int = -1,
                max_sub: int = 0, crowd_min: int = 0, algorithm: int = 1, pu_a: float = 0.0,
                pu_r0: float = 0.0, pu_r1: float = 0.0, P2: float = 0.0,
                bin_shape: int = 0, fft_sched: int = 0) -> nlint_params:
    """A filled nlint_params (the C-ABI's complete parameter set)."""
    lib = load_library()
    prm = nlint_params()
    lib.nlint_params_default(ctypes.byref(prm))
    prm.d, prm.n, prm.L = int(d), int(n), float(L)
    prm.kernel = {"coulomb": NLINT_COULOMB, "dipole": NLINT_DIPOLE}[kernel]
    for a in range(3):
        prm.axis[a] = float(axis[a]) if axis is not None else 0.0
        prm.axis2[a] = float(axis2[a]) if axis2 is not None else 0.0
    prm.alpha = float(alpha)
    if nodes is not None:
        if d == 3:
            prm.n_r, prm.n_theta, prm.n_phi = (int(v) for v in nodes)
        else:
            prm.n_r, prm.n_phi = (int(v) for v in nodes)
    prm.eps = float(eps)
    prm.precision = {None: -1, "fp32": NLINT_FP32, "fp64": NLINT_FP64}[precision]
    prm.w, prm.sigma, prm.P, prm.device = int(w), float(sigma), float(P), int(device)
    prm.max_sub, prm.crowd_min = int(max_sub), int(crowd_min)
    prm.algorithm, prm.pu_a, prm.pu_r0, prm.pu_r1, prm.P2 = (int(algorithm), float(pu_a),
                                                             float(pu_r0), float(pu_r1), float(P2))
    prm.bin_shape = int(bin_shape)
    prm.fft_sched = int(fft_sched)
    return prm


def autotune(params: nlint_params, tol: float, cache_path: Optional[str] = None):
    """Tuned copy of ``params`` for relative L-inf tolerance ``tol`` and the tuner's report."""
    lib = load_library()
    out = nlint_params()
    rep = nlint_tune_report()
    _check(lib.nlint_autotune(ctypes.byref(params), float(tol),
                              cache_path.encode() if cache_path else None, ctypes.byref(out),
                              ctypes.byref(rep)))
    return out, {f: getattr(rep, f) for f, _ in nlint_tune_report._fields_}


def autotune_batch(params: Sequence[nlint_params], tol: float, cache_path: Optional[str] = None,
                   branches: int = 0):
    """Tuned copies of the batch members' ``params`` (nlint_autotune_batch): per-member reports
    and the batch report (which decomposition was kept, both measured batch times)."""
    lib = load_library()
    count = len(params)
    arr = (nlint_params * count)(*params)
    out = (nlint_params * count)()
    reps = (nlint_tune_report * count)()
    brep = nlint_batch_tune_report()
    _check(lib.nlint_autotune_batch(count, arr, float(tol),
                                    cache_path.encode() if cache_path else None, int(branches),
                                    out, reps, ctypes.byref(brep)))
    members = [{f: getattr(r, f) for f, _ in nlint_tune_report._fields_} for r in reps]
    batch = {"choice": brep.choice, "classes": brep.classes, "ms": list(brep.ms)}
    return list(out), members, batch


class Plan:
    """A plan for u = U * rho and E = (lambda/2) <u, rho> on an n^d grid over [-L/2, L/2)^d.

    kernel: "coulomb" (3D: 1/(4 pi |x|); 2D: 1/(2 pi |x|)) or "dipole" (needs ``axis``, a 3-vector;
    ``axis2`` a second orientation, default the same; ``alpha`` the 2.5D constant).
    eps picks the precision (>= 1e-7: FP32, else FP64) and the spreading width unless given.
    nodes: (n_r, n_theta, n_phi) in 3D or (n_r, n_phi) in 2D; default from n.
    algorithm=2 selects Algorithm 2 (partition of unity, eq. 3.9): ``pu_a`` (3D, p_3 of eq. 3.10)
    or ``pu_r0``, ``pu_r1`` (2D, p_2 of eq. 3.12), ``P2`` the radius of I_2's nodes (0 = default);
    ``nodes`` are then I_2's node counts.
    """

    def __init__(self, d: int, n: int, L: float, kernel: str = "coulomb",
                 axis: Optional[Sequence[float]] = None, eps: float = 1e-6,
                 precision: Optional[str] = None, nodes: Optional[Sequence[int]] = None,
                 w: int = 0, sigma: float = 0.0, P: float = 0.0, device: Optional[int] = None,
                 axis2: Optional[Sequence[float]] = None, alpha: float = 0.0,
                 max_sub: int = 0, crowd_min: int = 0, algorithm: int = 1, pu_a: float = 0.0,
                 pu_r0: float = 0.0, pu_r1: float = 0.0, P2: float = 0.0,
                 bin_shape: int = 0, fft_sched: int = 0,
                 params: Optional["nlint_params"] = None):
        lib = load_library()
        prm = nlint_params()
        lib.nlint_params_default(ctypes.byref(prm))
        prm.d, prm.n, prm.L = int(d), int(n), float(L)
        prm.kernel = {"coulomb": NLINT_COULOMB, "dipole": NLINT_DIPOLE}[kernel]
        if axis is not None:
            for a in range(3):
                prm.axis[a] = float(axis[a])
        if axis2 is not None:
            for a in range(3):
                prm.axis2[a] = float(axis2[a])
        prm.alpha = float(alpha)
        if nodes is not None:
            if d == 3:
                prm.n_r, prm.n_theta, prm.n_phi = (int(v) for v in nodes)
            else:
                prm.n_r, prm.n_phi = (int(v) for v in nodes)
        prm.eps = float(eps)
        prm.precision = {None: -1, "fp32": NLINT_FP32, "fp64": NLINT_FP64}[precision]
        prm.w, prm.sigma, prm.P = int(w), float(sigma), float(P)
        if device is None:
            torch = _torch()
            device = torch.cuda.current_device() if torch.cuda.is_available() else -1
        prm.device = int(device)
        prm.max_sub, prm.crowd_min = int(max_sub), int(crowd_min)
        prm.algorithm, prm.pu_a, prm.pu_r0, prm.pu_r1, prm.P2 = (
            int(algorithm), float(pu_a), float(pu_r0), float(pu_r1), float(P2))
        prm.bin_shape = int(bin_shape)
        prm.fft_sched = int(fft_sched)
        if params is not None:  # a complete parameter set, e.g. from autotune()
            prm = params
            prm.device = int(device)
        h = ctypes.c_void_p()
        _check(lib.nlint_plan_create_ex(ctypes.byref(prm), ctypes.byref(h)))
        self._h = h
        self._lib = lib
        info = nlint_info()
        _check(lib.nlint_plan_info(h, ctypes.byref(info)))
        self.info = {f: getattr(info, f) for f, _ in nlint_info._fields_}
        self.info["bin"] = tuple(info.bin)
        self.d, self.n, self.L = int(info.d), int(info.n), float(info.L)
        self.device = int(device)
        self.precision = "fp32" if info.precision == NLINT_FP32 else "fp64"

    # ------------------------------------------------------------------ helpers
    @property
    def dtype(self):
        torch = _torch()
        return torch.float32 if self.precision == "fp32" else torch.float64

    @property
    def cdtype(self):
        torch = _torch()
        return torch.complex64 if self.precision == "fp32" else torch.complex128

    def _dev(self, t, shape, dtype, name):
        torch = _torch()
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {dtype} tensor of shape {tuple(shape)}")
        if t.device.index != self.device:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the plan on cuda:{self.device}")
        return t.data_ptr()

    @property
    def grid_shape(self):
        return (self.n,) * self.d

    # ------------------------------------------------------------------ entry points
    def eval(self, rho, out=None, stream=None):
        torch = _torch()
        u = out if out is not None else torch.empty(self.grid_shape, dtype=self.dtype, device=rho.device)
        _check(self._lib.nlint_eval(self._h, self._dev(rho, self.grid_shape, self.dtype, "rho"),
                                    self._dev(u, self.grid_shape, self.dtype, "u"), _stream_ptr(stream)))
        return u

    def eval_energy(self, rho, lam: float = 1.0, out=None, E_out=None, stream=None):
        torch = _torch()
        u = out if out is not None else torch.empty(self.grid_shape, dtype=self.dtype, device=rho.device)
        E = E_out if E_out is not None else torch.empty((), dtype=torch.float64, device=rho.device)
        _check(self._lib.nlint_eval_energy(self._h, self._dev(rho, self.grid_shape, self.dtype, "rho"),
                                           self._dev(u, self.grid_shape, self.dtype, "u"), float(lam),
                                           E.data_ptr(), _stream_ptr(stream)))
        return u, E

    def energy(self, rho, u, lam: float = 1.0, stream=None) -> float:
        Eh = ctypes.c_double()
        _check(self._lib.nlint_energy(self._h, self._dev(rho, self.grid_shape, self.dtype, "rho"),
                                      self._dev(u, self.grid_shape, self.dtype, "u"), float(lam),
                                      None, ctypes.byref(Eh), _stream_ptr(stream)))
        return Eh.value

    def toeplitz(self, stream=None):
        """Precompute the Toeplitz kernel's DFT (synchronous); enables eval_toeplitz."""
        _check(self._lib.nlint_plan_toeplitz(self._h, _stream_ptr(stream)))

    def eval_toeplitz(self, rho, lam: float = 1.0, out=None, E_out=None, stream=None):
        """u (and E) by the precomputed-kernel FFT convolution (same operator as eval)."""
        torch = _torch()
        u = out if out is not None else torch.empty(self.grid_shape, dtype=self.dtype, device=rho.device)
        E = E_out if E_out is not None else torch.empty((), dtype=torch.float64, device=rho.device)
        _check(self._lib.nlint_eval_toeplitz(self._h, self._dev(rho, self.grid_shape, self.dtype, "rho"),
                                             self._dev(u, self.grid_shape, self.dtype, "u"), float(lam),
                                             E.data_ptr(), _stream_ptr(stream)))
        return u, E

    def energy_only(self, rho, lam: float = 1.0, E_out=None, stream=None):
        """E = (lam/2) sum_j W_j |rho_hat_j|^2 from the type-2 half of the path (no potential).
        Returns a device float64 scalar tensor (no synchronisation)."""
        torch = _torch()
        E = E_out if E_out is not None else torch.empty((), dtype=torch.float64, device=rho.device)
        _check(self._lib.nlint_energy_only(self._h, self._dev(rho, self.grid_shape, self.dtype, "rho"),
                                           float(lam), E.data_ptr(), None, _stream_ptr(stream)))
        return E

    def eval_host(self, rho_host, lam: float = 1.0, u_host=None, stream=None):
        """End-to-end call with host buffers (numpy arrays or CPU tensors, pinned is best)."""
        torch = _torch()
        if isinstance(rho_host, np.ndarray):
            rho_host = torch.from_numpy(np.ascontiguousarray(rho_host))
        if rho_host.is_cuda or rho_host.dtype != self.dtype or tuple(rho_host.shape) != self.grid_shape:
            raise ValueError("rho_host must be a CPU array of the plan's dtype and grid shape")
        u = u_host if u_host is not None else torch.empty(self.grid_shape, dtype=self.dtype)
        Eh = ctypes.c_double()
        _check(self._lib.nlint_eval_host(self._h, rho_host.data_ptr(), u.data_ptr(), float(lam),
                                         ctypes.byref(Eh), _stream_ptr(stream)))
        return u, Eh.value

    def _host(self, a, name):
        torch = _torch()
        if isinstance(a, np.ndarray):
            a = torch.from_numpy(np.ascontiguousarray(a))
        if a.is_cuda or a.dtype != self.dtype or tuple(a.shape) != self.grid_shape or not a.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CPU array of the plan's dtype and grid shape")
        return a

    def eval_host_many(self, rhos_host, lam: float = 1.0, us_host=None, energies: bool = True,
                       stream=None):
        """Many densities from host buffers, copies overlapped with the evaluations (pinned host
        memory is best).  Returns (list of u host tensors, list of E or None)."""
        torch = _torch()
        rhos = [self._host(r, "rho_host") for r in rhos_host]
        if not rhos:
            raise ValueError("rhos_host is empty")
        us = (list(us_host) if us_host is not None
              else [torch.empty(self.grid_shape, dtype=self.dtype) for _ in rhos])
        if len(us) != len(rhos):
            raise ValueError("us_host must have one array per density")
        us = [self._host(u, "u_host") for u in us]
        vp = ctypes.c_void_p
        rp = (vp * len(rhos))(*[r.data_ptr() for r in rhos])
        up = (vp * len(us))(*[u.data_ptr() for u in us])
        E = (ctypes.c_double * len(rhos))() if energies else None
        _check(self._lib.nlint_eval_host_many(self._h, len(rhos), rp, up, float(lam),
                                              E if energies else None, _stream_ptr(stream)))
        return us, (list(E) if energies else None)

    def type2(self, rho, out=None, stream=None):
        torch = _torch()
        M = self.info["n_nodes"]
        r = out if out is not None else torch.empty((M,), dtype=self.cdtype, device=rho.device)
        _check(self._lib.nlint_type2(self._h, self._dev(rho, self.grid_shape, self.dtype, "rho"),
                                     self._dev(r, (M,), self.cdtype, "rho_hat"), _stream_ptr(stream)))
        return r

    def type1(self, c, out=None, stream=None):
        torch = _torch()
        M = self.info["n_nodes"]
        u = out if out is not None else torch.empty(self.grid_shape, dtype=self.dtype, device=c.device)
        _check(self._lib.nlint_type1(self._h, self._dev(c, (M,), self.cdtype, "c"),
                                     self._dev(u, self.grid_shape, self.dtype, "u"), _stream_ptr(stream)))
        return u

    def nodes(self):
        M = self.info["n_nodes"]
        k = np.empty((M, self.d), dtype=np.float64)
        W = np.empty(M, dtype=np.float64)
        _check(self._lib.nlint_plan_nodes(self._h, k.ctypes.data, W.ctypes.data))
        return k, W

    def set_stage_timing(self, enable: bool = True):
        _check(self._lib.nlint_set_stage_timing(self._h, 1 if enable else 0))

    def stage_times(self):
        ms = (ctypes.c_float * 32)()
        names = (ctypes.c_char_p * 32)()
        k = ctypes.c_int()
        _check(self._lib.nlint_stage_times(self._h, ms, names, 32, ctypes.byref(k)))
        return [(names[i].decode(), ms[i]) for i in range(k.value)]

    def check(self):
        """Raise NlintError (NLINT_ETIMEOUT) if a bounded device-side wait of this plan's kernels
        ran out since the last check (synchronises the device)."""
        _check(self._lib.nlint_plan_check(self._h))

    def launch_count(self) -> int:
        """Kernels this plan has launched so far (a host-side counter kept by the library)."""
        c = ctypes.c_int64()
        _check(self._lib.nlint_launch_count(self._h, ctypes.byref(c)))
        return c.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.nlint_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent densities, one plan each, evaluated together by one CUDA graph.

    ``plans`` must stay alive as long as the batch.  ``eval(rhos, lam)`` takes one CUDA tensor
    per plan and returns the list of potentials and a float64 tensor of the energies.  The graph
    is captured on the first call and re-captured only when the tensors or lam change.
    """

    def __init__(self, plans, branches: int = 0):
        self._lib = load_library()
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(self._lib.nlint_batch_create(len(self.plans), arr, int(branches), ctypes.byref(h)))
        self._h = h
        self._u = None
        self._E = None

    def info(self):
        c, b, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        _check(self._lib.nlint_batch_info(self._h, ctypes.byref(c), ctypes.byref(b), ctypes.byref(k)))
        return {"count": c.value, "branches": b.value, "kernels_per_eval": k.value}

    def eval(self, rhos, lam: float = 1.0, outs=None, E_out=None, stream=None):
        torch = _torch()
        if len(rhos) != len(self.plans):
            raise ValueError("one density per plan")
        if outs is None:
            if self._u is None or any(u.data_ptr() == r.data_ptr() for u, r in zip(self._u, rhos)):
                self._u = [torch.empty(p.grid_shape, dtype=p.dtype, device=r.device)
                           for p, r in zip(self.plans, rhos)]
            outs = self._u
        if E_out is None:
            if self._E is None:
                self._E = torch.empty(len(self.plans), dtype=torch.float64, device=rhos[0].device)
            E_out = self._E
        rp = (ctypes.c_void_p * len(rhos))(*[p._dev(r, p.grid_shape, p.dtype, "rho")
                                             for p, r in zip(self.plans, rhos)])
        up = (ctypes.c_void_p * len(outs))(*[p._dev(u, p.grid_shape, p.dtype, "u")
                                             for p, u in zip(self.plans, outs)])
        _check(self._lib.nlint_batch_eval(self._h, rp, up, float(lam), E_out.data_ptr(),
                                          _stream_ptr(stream)))
        return outs, E_out

    def close(self):
        if getattr(self, "_h", None):
            self._lib.nlint_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
