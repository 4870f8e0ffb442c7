"""Algorithm 2 (Section 3.3): the partition-of-unity split u = I_1 + I_2 of eq. 3.9, FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The truncated inverse transform of eq. 3.3 is split with a smooth p_d that is 1 near k = 0:
  I_1 = (2 pi)^{-d} int_{|k|<=P} e^{ik.x} U_hat(k) (1 - p_d(k)) rho_hat(k) dk
  I_2 = (2 pi)^{-d} int_{|k|<=P} e^{ik.x} U_hat(k) p_d(k) rho_hat(k) dk
with p_3(k) = exp(-|k|^2 / a) (eq. 3.10) and p_2(k) = erfc(12 (|k| - (R0+R1)/2) / (R1-R0)) / 2
(eq. 3.12).  U_hat (1 - p_d) is smooth, so I_1 is evaluated by the regular FFT with
oversampling factor 2 (Algorithm 2, step 3); I_2 by the NUFFT of Algorithm 1 on a small node
set, since p_d confines it to a ball of radius P2 around the origin (step 4).

Discrete definitions (the readings this oracle fixes; the GPU path computes the same):
  * I_1 is the trapezoidal rule in k on the grid of the n_pad-point DFT (n_pad >= 2n: the
    oversampling factor 2 of step 3; n_pad = 2n unless given), k_g = 2 pi g / (n_pad h) with
    g in numpy's fftfreq order (index n_pad/2 is frequency -n_pad/2).  With rho zero-padded to
    n_pad points per axis and F = DFT_{n_pad}(rho_pad),
        u1_m = n_pad^{-d} sum_g e^{2 pi i g.m / n_pad} M_g F_g,    m = 0..n-1 (array index),
    because (2 pi)^{-d} (2 pi / (n_pad h))^d h^d = n_pad^{-d}.  M_g = U_hat(k_g) (1 - p_d(k_g)) on
    the closed ball |k_g| <= P (points on the sphere are included; the test uses a relative
    margin of 1e-12) and 0 outside it.  At k = 0 the symbol takes its limit: 1/a for the 3D
    Coulomb kernel ((1 - e^{-k^2/a}) / k^2 -> 1/a), 0 for the dipole kernels (1 - p_3 ~ k^2/a
    against a bounded symbol) and for every 2D kernel (1 - p_2(0) = erfc(x_0)/2 is below
    double rounding for the admissible R0, R1, see below).
  * I_2 is Algorithm 1 (oracle.pipeline) with the radial Gauss-Legendre rule on [0, P2] in
    place of [0, P] and weights W_j p_d(k_j).
  * The cutoff must satisfy P <= pi / h, so that the ball stays inside the DFT's frequency
    cube (no Nyquist-plane ambiguity), and P2 <= P.
  * The energy is the trapezoidal rule of Remark 3.3 on u = u1 + u2.

Parameters.  The paper ties a and R0, R1 to the mesh (a = 2 / h^2, R0 = 0.8 / h, R1 = 10 / h)
by a dimensional argument; with those values p_d is far from 0 over the whole Nyquist ball
and I_2 needs as many nodes as Algorithm 1.  This module takes a, R0, R1, P2 as inputs;
``default_parameters`` gives the values used by the tests, from the aliasing bound of I_1:
the real-space kernel of U_hat (1 - p_d) decays like erfc(sqrt(a) r / 2) (3D Coulomb), so its
images at distance >= L (the padding) are below 1e-16 when sqrt(a) L / 2 >= 5.9.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

from . import pipeline, quadrature

SPHERE_MARGIN = 1e-12


def p3(k: np.ndarray, a: float) -> np.ndarray:
    """Eq. 3.10: exp(-|k|^2 / a); k has shape (M, 3)."""
    return np.exp(-np.sum(k * k, axis=1) / a)


def p2(k: np.ndarray, r0: float, r1: float) -> np.ndarray:
    """Eq. 3.12: erfc(12 (|k| - (R0 + R1)/2) / (R1 - R0)) / 2; k has shape (M, 2)."""
    kk = np.sqrt(np.sum(k * k, axis=1))
    return 0.5 * special.erfc(12.0 * (kk - 0.5 * (r0 + r1)) / (r1 - r0))


def partition(k: np.ndarray, d: int, a=None, r0=None, r1=None) -> np.ndarray:
    return p3(k, a) if d == 3 else p2(k, r0, r1)


def default_parameters(d: int, n: int, L: float, precision: str = "fp64") -> dict:
    """a (3D) or R0, R1 (2D), the I_2 cutoff P2 and its node counts.

    3D: sqrt(a) = 11.8 / L (I_1's kernel images below 1e-16), P2 = 6.1 sqrt(a)
    (p_3(P2) = e^{-37}).  2D: R1 - R0 = 148 / L (the same bound for the erfc transition,
    whose width is (R1 - R0)/12), R0 = 12 / L, P2 = R1 (p_2(R1) = erfc(6)/2 = 1e-17).
    Every radius is capped by the grid's Nyquist radius pi / h.  P2 L and the phase
    P2 |x| over the box do not depend on L, so the node counts are fixed: measured against
    closed forms on off-centre mixtures, 3D 32x32x64 gives about 6e-10 and 40x40x80 7e-13;
    2D 48x96 about 1e-7 and 64x128 below 1e-12 (the paper's Remarks quote 24^3 / 40^3 and
    40^2 / 60^2 for 6 / 12 digits).
    """
    h = L / n
    P = math.pi / h
    fp32 = precision == "fp32"
    if d == 3:
        a = (11.8 / L) ** 2
        P2 = min(P, 6.1 * math.sqrt(a))
        return {"a": a, "P2": P2, "nodes2": (32, 32, 64) if fp32 else (40, 40, 80)}
    r0, r1 = 12.0 / L, 160.0 / L
    return {"r0": r0, "r1": r1, "P2": min(P, r1), "nodes2": (48, 96) if fp32 else (64, 128)}


def frequencies(d: int, n: int, L: float, n_pad: int | None = None) -> list:
    """k values per axis of the n_pad-point DFT grid, fftfreq order: 2 pi g / (n_pad h)."""
    h = L / n
    return [2.0 * np.pi * np.fft.fftfreq(n_pad or 2 * n, d=h)] * d


def multiplier_I1(d: int, n: int, L: float, kernel: str = "coulomb", axis=None, axis2=None,
                  alpha: float = 0.0, a=None, r0=None, r1=None, P=None,
                  n_pad: int | None = None) -> np.ndarray:
    """M_g = U_hat(k_g) (1 - p_d(k_g)) on |k_g| <= P, shape (n_pad,)*d in fftfreq order.

    Array axis 0 is the slowest (z in 3D, y in 2D), as for the densities."""
    h = L / n
    if P is None:
        P = math.pi / h
    if P > math.pi / h * (1.0 + SPHERE_MARGIN):
        raise ValueError("Algorithm 2 needs P <= pi / h")
    n_pad = n_pad or 2 * n
    if n_pad < 2 * n:
        raise ValueError("I_1 needs n_pad >= 2n (oversampling factor 2)")
    ks = np.meshgrid(*frequencies(d, n, L, n_pad), indexing="ij")
    # arrays are C-order over (z, y[, x]); U_hat takes k in (k_x, k_y[, k_z]) order
    k = np.stack([ks[d - 1 - i].ravel() for i in range(d)], axis=1)
    k2 = np.sum(k * k, axis=1)
    inside = k2 <= (P * (1.0 + SPHERE_MARGIN)) ** 2
    zero = k2 == 0.0
    kz = k.copy()
    kz[zero] = 1.0  # any nonzero vector: the k = 0 entry is replaced by its limit below
    uh = quadrature.u_hat(kz, d, kernel, axis, axis2, alpha)
    if d == 3:
        one_minus_p = -np.expm1(-np.sum(kz * kz, axis=1) / a)
    else:
        one_minus_p = 1.0 - p2(kz, r0, r1)
    M = uh * one_minus_p
    M[zero] = (1.0 / a) if (d == 3 and kernel == "coulomb") else 0.0
    M[~inside] = 0.0
    return M.reshape((n_pad,) * d)


def I1(rho: np.ndarray, M: np.ndarray) -> np.ndarray:
    """u1 = (IDFT (M DFT(rho_pad)))[:n]^d on M's n_pad grid, real part (the imaginary part is
    rounding); also returns F = DFT(rho_pad)."""
    rho = np.asarray(rho, dtype=np.float64)
    d, n = rho.ndim, rho.shape[0]
    pad = np.zeros((M.shape[0],) * d)
    pad[(slice(0, n),) * d] = rho
    F = np.fft.fftn(pad)
    v = np.fft.ifftn(M * F)
    return v[(slice(0, n),) * d].real.copy(), F


def I2_nodes(d: int, n: int, L: float, nodes2, kernel="coulomb", axis=None, axis2=None,
             alpha=0.0, a=None, r0=None, r1=None, P2=None):
    """I_2's nodes and weights: Algorithm 1's rule with radius P2, weights times p_d."""
    k, W = quadrature.nodes_weights(d, n, L, nodes2, kernel, axis, axis2, alpha, P2)
    return k, W * partition(k, d, a, r0, r1)


def alg2_eval(rho: np.ndarray, L: float, nodes2, kernel: str = "coulomb", axis=None, axis2=None,
              alpha: float = 0.0, a=None, r0=None, r1=None, P=None, P2=None, lam: float = 1.0,
              method: str = "nufft", setting: str = "parity", n_pad: int | None = None) -> dict:
    """Algorithm 2: u = I_1 + I_2 and E on the grid; also the parts and the dual energies."""
    rho = np.asarray(rho, dtype=np.float64)
    d, n = rho.ndim, rho.shape[0]
    h = L / n
    if P is None:
        P = math.pi / h
    if P2 is None or P2 > P:
        raise ValueError("P2 must be given and at most P")
    M = multiplier_I1(d, n, L, kernel, axis, axis2, alpha, a, r0, r1, P, n_pad)
    u1, F = I1(rho, M)
    npd = M.shape[0]
    k, W = I2_nodes(d, n, L, nodes2, kernel, axis, axis2, alpha, a, r0, r1, P2)
    rh = pipeline.type2(rho, L, k, method, setting)
    f = pipeline.type1(W * rh, d, n, L, k, method, setting)
    u2 = f.real.copy()
    u = u1 + u2
    # dual energies: sum_m u1_m rho_m = n_pad^{-d} sum_g M_g |F_g|^2 (rho real)
    e1 = 0.5 * lam * h ** d * float(npd) ** (-d) * math.fsum((M * np.abs(F) ** 2).ravel().tolist())
    e2 = pipeline.energy_dual(rh, W, lam)
    s1 = 0.5 * lam * h ** d * float(npd) ** (-d) * math.fsum((np.abs(M) * np.abs(F) ** 2).ravel().tolist())
    s2 = pipeline.energy_scale(rh, W, lam)
    return {
        "u": u, "u1": u1, "u2": u2,
        "E": pipeline.energy(u, rho, L, lam),
        "E_dual": e1 + e2, "E1_dual": e1, "E2_dual": e2,
        "E_scale": s1 + s2,
        "imag_max": float(np.max(np.abs(f.imag))),
        "k2": k, "W2": W, "M": M,
    }
