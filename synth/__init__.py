"""Seeded synthetic workloads shared by the oracle tests, the GPU tests and the benchmark.

This module only describes the workloads (grid, box, kernel, node counts) and samples the
densities on the grid.  It holds none of the method's arithmetic: no quadrature, no Fourier
transform, no kernel symbol, no energy.  Both sides of every parity check receive the same
arrays from here and compute everything else on their own.

Grid convention (used by every caller): a d-dimensional C-order array, last index fastest.
In 3D the array index is (i_z, i_y, i_x); in 2D it is (i_y, i_x).  Index i along an axis sits
at coordinate x = -L/2 + i*h with h = L/n, i = 0..n-1 (the right end of the box is excluded).

Seeds: 1311 for density mixtures, 4120 for dipole axes; numpy ``default_rng``.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Optional, Sequence

import numpy as np

SEED_MIX = 1311
SEED_AXIS = 4120


def grid_coords(d: int, n: int, L: float):
    """Return the d coordinate arrays (broadcastable, C-order (z,y,x) or (y,x))."""
    h = L / n
    x1 = -L / 2 + h * np.arange(n, dtype=np.float64)
    if d == 3:
        z = x1[:, None, None]
        y = x1[None, :, None]
        x = x1[None, None, :]
        return z, y, x
    if d == 2:
        y = x1[:, None]
        x = x1[None, :]
        return y, x
    raise ValueError("d must be 2 or 3")


def random_unit(rng: np.random.Generator, d: int = 3) -> np.ndarray:
    v = rng.standard_normal(d)
    return v / np.linalg.norm(v)


# --------------------------------------------------------------------------- densities
def gauss_iso(d: int, n: int, L: float, s: float = 1.0) -> np.ndarray:
    """exp(-|x|^2 / s^2) on the grid."""
    c = grid_coords(d, n, L)
    r2 = sum(ci * ci for ci in c)
    return np.exp(-r2 / (s * s))


def gauss_axes(n: int, L: float, a: Sequence[float]) -> np.ndarray:
    """3D exp(-(x^2/a_x + y^2/a_y + z^2/a_z)); ``a`` is (a_x, a_y, a_z)."""
    z, y, x = grid_coords(3, n, L)
    return np.exp(-(x * x / a[0] + y * y / a[1] + z * z / a[2]))


def mixture(d: int, n: int, L: float, centres: np.ndarray, widths: np.ndarray,
            weights: np.ndarray) -> np.ndarray:
    """sum_i w_i exp(-|x - c_i|^2 / s_i^2); centres are given in (x, y[, z]) order."""
    c = grid_coords(d, n, L)
    # c is ordered (z, y, x) / (y, x); centres are (x, y, z) / (x, y)
    axes = list(reversed(c))
    out = np.zeros((n,) * d, dtype=np.float64)
    for ci, si, wi in zip(centres, widths, weights):
        r2 = sum((axes[a] - ci[a]) ** 2 for a in range(d))
        out += wi * np.exp(-r2 / (si * si))
    return out


def mixture_params(rng: np.random.Generator, count: int, d: int, c_half: float,
                   s_lo: float, s_hi: float, w_lo: float, w_hi: float):
    centres = rng.uniform(-c_half, c_half, size=(count, d))
    widths = rng.uniform(s_lo, s_hi, size=count)
    weights = rng.uniform(w_lo, w_hi, size=count)
    return centres, widths, weights


# --------------------------------------------------------------------------- workloads
@dataclass
class Workload:
    """One density on one grid with one interaction kernel and one node set."""
    name: str
    d: int
    n: int
    L: float
    kernel: str                      # "coulomb" | "dipole"
    nodes: tuple                     # (N_r, N_theta, N_phi) in 3D, (N_r, N_phi) in 2D
    precision: str                   # "fp32" | "fp64"
    tol: float                       # relative L-inf tolerance against the oracle
    axis: Optional[np.ndarray] = None
    lam: float = 1.0
    make_rho: Callable[[], np.ndarray] = field(default=None, repr=False)
    desc: str = ""

    @property
    def h(self) -> float:
        return self.L / self.n

    @property
    def n_points(self) -> int:
        return self.n ** self.d

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.nodes))

    def rho(self) -> np.ndarray:
        return self.make_rho()


def default_nodes(d: int, n: int) -> tuple:
    """Default node counts used when a caller names only (d, n).

    3D anchors: n=32 -> 32x32x64, n=128 -> 96x96x192, n=256 -> 160x160x320; other n are
    linearly interpolated in n and rounded to a multiple of 8 (n=48 -> 40, 64 -> 56,
    96 -> 72).  2D: n=512 -> 128 x 256 and N_r = n/4, N_phi = n/2 in general.
    """
    if d == 2:
        nr = max(8, n // 4)
        return (nr, 2 * nr)
    xs = [32, 128, 256]
    ys = [32, 96, 160]
    v = float(np.interp(n, xs, ys, left=None, right=None))
    if n < 32:
        v = float(n)
    if n > 256:
        v = 160 + (n - 256) * 0.5
    nr = max(8, int(round(v / 8.0)) * 8)
    return (nr, nr, 2 * nr)


def config1() -> Workload:
    return Workload(
        name="c1", d=3, n=32, L=16.0, kernel="coulomb", nodes=(32, 32, 64),
        precision="fp64", tol=1e-10,
        make_rho=lambda: gauss_iso(3, 32, 16.0),
        desc="3D Coulomb, exp(-|x|^2) on 32^3 over [-8,8]^3, 32x32x64 nodes, FP64")


def config2() -> Workload:
    def rho():
        rng = np.random.default_rng(SEED_MIX)
        centres, widths, weights = mixture_params(rng, 8, 2, 2.0, 0.5, 1.5, 1.0, 1.0)
        y, x = grid_coords(2, 512, 32.0)
        base = np.exp(-(x * x + y * y / 4.0))
        return base + mixture(2, 512, 32.0, centres, widths, weights)
    return Workload(
        name="c2", d=2, n=512, L=32.0, kernel="coulomb", nodes=(128, 256),
        precision="fp64", tol=1e-10, make_rho=rho,
        desc="2.5D Coulomb, exp(-(x^2+y^2/4)) + 8 seeded Gaussians on 512^2 over [-16,16]^2, "
             "128x256 nodes, FP64")


def config3() -> Workload:
    axis = random_unit(np.random.default_rng(SEED_AXIS), 3)
    return Workload(
        name="c3", d=3, n=128, L=24.0, kernel="dipole", nodes=(96, 96, 192),
        precision="fp32", tol=1e-5, axis=axis,
        make_rho=lambda: gauss_axes(128, 24.0, (1.0, 1.0, 2.25)),
        desc="3D dipole (seeded axis), exp(-(x^2+y^2+z^2/2.25)) on 128^3 over [-12,12]^3, "
             "96x96x192 nodes, FP32")


def config4() -> Workload:
    def rho():
        rng = np.random.default_rng(SEED_MIX)
        centres, widths, weights = mixture_params(rng, 16, 3, 4.0, 0.6, 1.4, 0.5, 1.0)
        return mixture(3, 256, 32.0, centres, widths, weights)
    return Workload(
        name="c4", d=3, n=256, L=32.0, kernel="coulomb", nodes=(160, 160, 320),
        precision="fp32", tol=1e-5, make_rho=rho,
        desc="3D Coulomb, 16 seeded Gaussians on 256^3 over [-16,16]^3, 160x160x320 nodes, FP32")


def config5(precision: str = "fp32", count: int = 64) -> list:
    """Batch of ``count`` seeded densities on uneven cubic grids (box [-12,12]^3).

    Sizes are drawn from {32,48,64,96,128}; the first half are Coulomb, the second half
    dipolar with seeded random axes; each density is a mixture drawn like config 4's.
    """
    rng = np.random.default_rng(SEED_MIX)
    arng = np.random.default_rng(SEED_AXIS)
    sizes = rng.choice([32, 48, 64, 96, 128], size=count)
    out = []
    for i in range(count):
        n = int(sizes[i])
        kern = "coulomb" if i < count // 2 else "dipole"
        axis = random_unit(arng, 3) if kern == "dipole" else None
        centres, widths, weights = mixture_params(rng, 16, 3, 4.0, 0.6, 1.4, 0.5, 1.0)
        mk = (lambda n=n, c=centres, s=widths, w=weights: mixture(3, n, 24.0, c, s, w))
        out.append(Workload(
            name=f"c5[{i}]", d=3, n=n, L=24.0, kernel=kern, nodes=default_nodes(3, n),
            precision=precision, tol=1e-5 if precision == "fp32" else 1e-10, axis=axis,
            make_rho=mk, desc=f"batch member {i}: n={n}, {kern}"))
    return out


CONFIGS = {"c1": config1, "c2": config2, "c3": config3, "c4": config4}
