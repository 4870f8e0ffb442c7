"""Algorithm 1 (Section 3.2) assembled from the oracle parts, FP64.  TEST INFRASTRUCTURE ONLY.

Given d, the grid (n points per axis on [-L/2, L/2)), the node counts and the kernel:
  1. nodes k_j and weights W_j of eq. 3.7                       (oracle.quadrature)
  2. rho_hat_j = h^d sum_m rho_m e^{-i k_j . x_m}  (eq. 3.2)    type-2 sum
  3. c_j = W_j rho_hat_j                                          multiply
  4. u_m = Re sum_j c_j e^{+i k_j . x_m}           (eq. 3.7)    type-1 sum
  5. E = (lambda/2) h^d sum_m u_m rho_m            (Remark 3.3) energy
Since x_m = m h for the centred index m = i - n/2, k_j . x_m = t_j . m with t_j = k_j h, which
is the form the NUFFT of Section 2 evaluates.  ``method="direct"`` uses the plain sums of
oracle.direct; ``method="nufft"`` uses O2 at the named accuracy setting.
"""
from __future__ import annotations

import math

import numpy as np

from . import direct, nufft, quadrature


def nodes_weights(d, n, L, nodes, kernel="coulomb", axis=None, axis2=None, alpha=0.0, P=None):
    return quadrature.nodes_weights(d, n, L, nodes, kernel, axis, axis2, alpha, P)


def type2(rho: np.ndarray, L: float, k: np.ndarray, method: str = "nufft",
          setting: str = "parity") -> np.ndarray:
    d, n = rho.ndim, rho.shape[0]
    h = L / n
    if method == "direct":
        return direct.type2(rho, L, k)
    return (h ** d) * nufft.type2(rho.astype(np.complex128), k * h, setting)


def type1(c: np.ndarray, d: int, n: int, L: float, k: np.ndarray, method: str = "nufft",
          setting: str = "parity") -> np.ndarray:
    h = L / n
    if method == "direct":
        return direct.type1(c, d, n, L, k)
    return nufft.type1(c, k * h, d, n, setting)


def energy(u: np.ndarray, rho: np.ndarray, L: float, lam: float = 1.0) -> float:
    n = rho.shape[0]
    h = L / n
    return 0.5 * lam * (h ** rho.ndim) * math.fsum((np.asarray(u, np.float64) *
                                                    np.asarray(rho, np.float64)).ravel().tolist())


def energy_dual(rho_hat: np.ndarray, W: np.ndarray, lam: float = 1.0) -> float:
    """(lambda/2) sum_j W_j |rho_hat_j|^2: equal to the grid energy for the discrete operator."""
    return 0.5 * lam * math.fsum((W * np.abs(rho_hat) ** 2).tolist())


def energy_scale(rho_hat: np.ndarray, W: np.ndarray, lam: float = 1.0) -> float:
    """(lambda/2) sum_j |W_j| |rho_hat_j|^2: the scale used for energy errors (E may be ~0)."""
    return 0.5 * lam * math.fsum((np.abs(W) * np.abs(rho_hat) ** 2).tolist())


def oracle_eval(rho: np.ndarray, L: float, nodes, kernel: str = "coulomb", axis=None,
                axis2=None, alpha: float = 0.0, lam: float = 1.0, P=None,
                method: str = "nufft", setting: str = "parity") -> dict:
    """Run Algorithm 1 on a real density; returns u, E, diagnostics and the node data."""
    rho = np.asarray(rho, dtype=np.float64)
    d, n = rho.ndim, rho.shape[0]
    k, W = nodes_weights(d, n, L, nodes, kernel, axis, axis2, alpha, P)
    rh = type2(rho, L, k, method, setting)
    f = type1(W * rh, d, n, L, k, method, setting)
    u = f.real.copy()
    return {
        "u": u,
        "E": energy(u, rho, L, lam),
        "E_dual": energy_dual(rh, W, lam),
        "E_scale": energy_scale(rh, W, lam),
        "imag_max": float(np.max(np.abs(f.imag))),
        "rho_hat": rh,
        "k": k,
        "W": W,
    }
