"""Phase-space quadrature of Section 3.1 (eqs. 3.5 and 3.7) and the kernel symbols (int3dd).

The truncated inverse transform (eq. 3.3) is written in spherical (3D) or polar (2D)
coordinates (eq. 3.5); the Jacobian |k|^{d-1} cancels the singularity of U_hat at k = 0.
Eq. 3.7 discretises it with Gauss-Legendre rules in r (on [0, P]) and, in 3D, in theta
(on [0, pi]), and the trapezoidal rule in phi (on [0, 2 pi)).

Readings of the paper used here:
  * the weight w_j of eq. 3.7 includes the sin(theta) of eq. 3.5 (eq. 3.7 omits it);
  * trapezoidal nodes are phi_l = 2 pi l / N_phi, l = 0..N_phi-1;
  * k = r (sin t cos p, sin t sin p, cos t) in 3D and r (cos p, sin p) in 2D, listed in
    (k_x, k_y, k_z) / (k_x, k_y) order;
  * the 3D dipole symbol is -1 + 3 (n.k)^2/|k|^2 (eq. dipkernelF), and -(m.n) +
    3 (n.k)(m.k)/|k|^2 for two orientations (eq. dipkerneldF).

Node order ("canonical"): index j = (a * N_theta + b) * N_phi + c in 3D and j = a * N_phi + c
in 2D, with a the radial, b the polar and c the azimuthal index.
"""
from __future__ import annotations

import numpy as np


def _legendre_and_derivative(m: int, x: np.ndarray):
    """P_m(x) and P_m'(x) by the three-term recurrence (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1}
    and P_m' = m (P_{m-1} - x P_m) / ((1 - x)(1 + x))."""
    p0 = np.ones_like(x)
    p1 = x.copy()
    for j in range(1, m):
        p0, p1 = p1, ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0)
    if m == 1:
        p0 = np.ones_like(x)
    dp = m * (p0 - x * p1) / ((1.0 - x) * (1.0 + x))
    return p1, dp


def gauss_legendre(m: int, a: float, b: float):
    """m-point Gauss-Legendre rule on [a, b].

    numpy's leggauss supplies the starting nodes; its end weights lose accuracy as m grows
    (about 1e-11 relative at m = 128 and 2e-10 at m = 320), so the nodes are polished by
    Newton steps on P_m and the weights recomputed as w = 2 / ((1 - x)(1 + x) P_m'(x)^2),
    the factored 1 - x^2 avoiding cancellation near the ends.  Pinned against a
    high-precision rule in the tests.
    """
    xi, _ = np.polynomial.legendre.leggauss(m)
    for _ in range(3):
        p, dp = _legendre_and_derivative(m, xi)
        xi = xi - p / dp
    _, dp = _legendre_and_derivative(m, xi)
    om = 2.0 / ((1.0 - xi) * (1.0 + xi) * dp * dp)
    x = a + (b - a) * (1.0 + xi) / 2.0
    w = (b - a) * om / 2.0
    return x, w


def u_hat(k: np.ndarray, d: int, kernel: str, axis=None, axis2=None, alpha: float = 0.0):
    """Fourier symbol U_hat(k) of eq. (int3dd); k has shape (M, d) in (k_x, k_y[, k_z])."""
    k2 = np.sum(k * k, axis=1)
    if kernel == "coulomb":
        return 1.0 / k2 if d == 3 else 1.0 / np.sqrt(k2)
    if kernel == "dipole":
        n = np.asarray(axis, dtype=np.float64)
        n = n / np.linalg.norm(n)
        m = n if axis2 is None else np.asarray(axis2, dtype=np.float64) / np.linalg.norm(axis2)
        if d == 3:
            return -np.dot(m, n) + 3.0 * (k @ n) * (k @ m) / k2
        # 2.5D (eq. dipkernelF2dd): n, m are 3-vectors, their in-plane parts act on k
        kn = k @ n[:2]
        km = k @ m[:2]
        kk = np.sqrt(k2)
        return -alpha + 3.0 * (kn * km - n[2] * m[2] * k2) / (2.0 * kk)
    raise ValueError(kernel)


def nodes_weights(d: int, n: int, L: float, nodes, kernel: str = "coulomb", axis=None,
                  axis2=None, alpha: float = 0.0, P: float | None = None):
    """Nodes k_j (M, d) and weights W_j (M,) with u(x) ~ Re sum_j W_j rho_hat(k_j) e^{i k_j.x}.

    W_j = (2 pi)^{-d} w_j |k_j|^{d-1} U_hat(k_j), w_j = w_r w_theta sin(theta) w_phi (3D) or
    w_r w_phi (2D).  The cutoff defaults to P = pi / h, the Nyquist radius of the grid.
    """
    h = L / n
    if P is None:
        P = np.pi / h
    if d == 3:
        nr, nt, nphi = nodes
        r, wr = gauss_legendre(nr, 0.0, P)
        th, wt = gauss_legendre(nt, 0.0, np.pi)
        ph = 2.0 * np.pi * np.arange(nphi) / nphi
        wp = 2.0 * np.pi / nphi
        R, T, F = np.meshgrid(r, th, ph, indexing="ij")
        WR, WT, _ = np.meshgrid(wr, wt, ph, indexing="ij")
        st = np.sin(T)
        k = np.stack([R * st * np.cos(F), R * st * np.sin(F), R * np.cos(T)], axis=-1)
        k = k.reshape(-1, 3)
        w = (WR * WT * st * wp).reshape(-1)
        rr = R.reshape(-1)
        W = w * rr ** 2 * u_hat(k, 3, kernel, axis, axis2, alpha) / (2.0 * np.pi) ** 3
        return k, W
    if d == 2:
        nr, nphi = nodes
        r, wr = gauss_legendre(nr, 0.0, P)
        ph = 2.0 * np.pi * np.arange(nphi) / nphi
        wp = 2.0 * np.pi / nphi
        R, F = np.meshgrid(r, ph, indexing="ij")
        WR, _ = np.meshgrid(wr, ph, indexing="ij")
        k = np.stack([R * np.cos(F), R * np.sin(F)], axis=-1).reshape(-1, 2)
        w = (WR * wp).reshape(-1)
        rr = R.reshape(-1)
        W = w * rr * u_hat(k, 2, kernel, axis, axis2, alpha) / (2.0 * np.pi) ** 2
        return k, W
    raise ValueError("d must be 2 or 3")
