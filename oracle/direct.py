"""O1: the discrete operator of Algorithm 1 written out as plain sums (FP64, NumPy).

  rho_hat_j = h^d sum_m rho_m exp(-i k_j . x_m)          (eq. 3.2, trapezoidal rule)
  u_m       = Re sum_j W_j rho_hat_j exp(+i k_j . x_m)   (eq. 3.7)
  E         = (lambda / 2) h^d sum_m u_m rho_m           (Remark 3.3, trapezoidal rule)

with x_m = -L/2 + i h on each axis.  The cost is O(n^d N_f): tiny grids only.  The only
library routine is complex exponentiation and a dense matrix-vector product.
"""
from __future__ import annotations

import numpy as np


def grid_points(d: int, n: int, L: float) -> np.ndarray:
    """All grid points as an (n^d, d) array in (x, y[, z]) order, C-order over (z, y, x)."""
    h = L / n
    x1 = -L / 2 + h * np.arange(n)
    if d == 3:
        Z, Y, X = np.meshgrid(x1, x1, x1, indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    Y, X = np.meshgrid(x1, x1, indexing="ij")
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def type2(rho: np.ndarray, L: float, k: np.ndarray, chunk: int = 2048) -> np.ndarray:
    """rho_hat(k_j) by the trapezoidal rule of eq. 3.2, one node chunk at a time."""
    d = rho.ndim
    n = rho.shape[0]
    h = L / n
    x = grid_points(d, n, L)
    r = rho.reshape(-1).astype(np.complex128)
    out = np.empty(k.shape[0], dtype=np.complex128)
    for s in range(0, k.shape[0], chunk):
        ph = x @ k[s:s + chunk].T                        # (n^d, chunk)
        out[s:s + chunk] = (h ** d) * (r @ np.exp(-1j * ph))
    return out


def type1(c: np.ndarray, d: int, n: int, L: float, k: np.ndarray,
          chunk: int = 2048) -> np.ndarray:
    """f(x_m) = sum_j c_j exp(+i k_j . x_m) on the grid (complex, shape (n,)*d)."""
    x = grid_points(d, n, L)
    out = np.zeros(x.shape[0], dtype=np.complex128)
    for s in range(0, k.shape[0], chunk):
        ph = x @ k[s:s + chunk].T
        out += np.exp(1j * ph) @ c[s:s + chunk]
    return out.reshape((n,) * d)


def energy(u: np.ndarray, rho: np.ndarray, L: float, lam: float = 1.0) -> float:
    """(lambda/2) h^d sum u rho, summed with math.fsum (correctly rounded)."""
    import math
    n = rho.shape[0]
    h = L / n
    return 0.5 * lam * (h ** rho.ndim) * math.fsum((u * rho).ravel().tolist())


def apply(rho: np.ndarray, L: float, k: np.ndarray, W: np.ndarray, lam: float = 1.0):
    """Algorithm 1 by direct sums: returns (u, E, max|Im|, rho_hat)."""
    d = rho.ndim
    n = rho.shape[0]
    rh = type2(rho, L, k)
    f = type1(W * rh, d, n, L, k)
    u = f.real.copy()
    return u, energy(u, rho, L, lam), float(np.max(np.abs(f.imag))), rh
