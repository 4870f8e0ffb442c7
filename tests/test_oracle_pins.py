"""Pins for the CPU oracle: each test checks the oracle against something other than itself.

quadrature   exactness of the rules, closed-form sums of the weights, node symmetry
direct (O1)  the uniform-DFT special case (numpy.fft), the grid/dual energy identity
nufft  (O2)  its FFT against numpy.fft; its type-1/type-2 sums against the direct sums
pipeline     closed-form potentials and energies (3D/2.5D Coulomb, Examples 4, 5, 7),
             total charge, and the operator's invariants
"""
import math

import numpy as np
import pytest

import synth
from oracle import closed_forms as cf
from oracle import direct, nufft, pipeline, quadrature
from conftest import read_golden


def rel_inf(a, b, mask=None):
    if mask is not None:
        a, b = a[mask], b[mask]
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# --------------------------------------------------------------------------- quadrature
def test_gauss_legendre_exact_on_polynomials():
    P = 7.3
    x, w = quadrature.gauss_legendre(12, 0.0, P)
    for deg in range(0, 24):
        assert abs(np.sum(w * x ** deg) - P ** (deg + 1) / (deg + 1)) <= 1e-12 * P ** (deg + 1)


@pytest.mark.parametrize("m", [32, 128, 320])
def test_gauss_legendre_against_high_precision_rule(m):
    # Nodes are the roots of P_m found to 40 digits; weights 2 (1 - t^2) / (m P_{m-1}(t))^2.
    # Near the ends a node is only representable to ~5e-17 absolute, which moves the exact
    # weight at that double by up to ~2e-12 relative at m = 320 (the bound used here).
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    x, w = quadrature.gauss_legendre(m, -1.0, 1.0)
    for i in (0, 1, 3, m // 3, m // 2):
        t = mp.findroot(lambda s: mp.legendre(m, s), mp.mpf(x[i]))
        wt = 2 * (1 - t ** 2) / (m ** 2 * mp.legendre(m - 1, t) ** 2)
        assert abs(float(x[i] - t)) <= 1e-16
        assert abs(float((w[i] - wt) / wt)) <= 5e-12


def test_weight_sums_closed_form_3d_2d():
    # Coulomb: |k|^{d-1} U_hat = 1, so sum_j W_j = (2 pi)^{-d} * measure of the ball in (r, angles)
    n, L = 16, 8.0
    P = math.pi / (L / n)
    k, W = quadrature.nodes_weights(3, n, L, (10, 12, 16), "coulomb")
    assert abs(W.sum() - P * 4 * math.pi / (2 * math.pi) ** 3) < 1e-13 * W.sum()
    assert np.allclose(np.linalg.norm(k, axis=1).max(), P, rtol=0.1)
    k2, W2 = quadrature.nodes_weights(2, n, L, (10, 16), "coulomb")
    assert abs(W2.sum() - P * 2 * math.pi / (2 * math.pi) ** 2) < 1e-13 * W2.sum()
    # sum_j W_j |k_j|^2 / r^2 ... moment check pins r^{d-1} and sin(theta):
    # sum W_j k_z^2 = (2pi)^-3 int r^2 cos^2(t) sin(t) = (2pi)^-3 (P^3/3)(2/3)(2 pi)
    kz = k[:, 2]
    ref = (P ** 3 / 3) * (2.0 / 3.0) * (2 * math.pi) / (2 * math.pi) ** 3
    assert abs(np.sum(W * kz ** 2) - ref) < 1e-12 * ref


def test_node_set_symmetric_under_negation():
    for d, nodes in ((3, (6, 8, 12)), (2, (6, 12))):
        k, W = quadrature.nodes_weights(d, 16, 8.0, nodes, "dipole" if d == 3 else "coulomb",
                                        axis=[0.3, -0.5, 0.8])
        # mirror of (a, b, c) is (a, N_theta-1-b, c+N_phi/2)
        idx = np.arange(k.shape[0]).reshape(nodes)
        if d == 3:
            mir = idx[:, ::-1, :]
            mir = np.roll(mir, -nodes[2] // 2, axis=2)
        else:
            mir = np.roll(idx, -nodes[1] // 2, axis=1)
        mir = mir.ravel()
        assert np.max(np.abs(k + k[mir])) < 1e-12 * np.abs(k).max()
        assert np.max(np.abs(W - W[mir])) < 1e-14 * np.abs(W).max()


def test_dipole_trace_vanishes():
    k, _ = quadrature.nodes_weights(3, 16, 8.0, (6, 8, 12))
    s = sum(quadrature.u_hat(k, 3, "dipole", axis=e) for e in np.eye(3))
    assert np.max(np.abs(s)) < 1e-13


# --------------------------------------------------------------------------- O2 FFT
@pytest.mark.parametrize("n,d", [(8, 3), (12, 3), (48, 2), (96, 2), (64, 3)])
def test_oracle_fft_matches_numpy(n, d):
    rng = np.random.default_rng(n)
    x = rng.standard_normal((n,) * d) + 1j * rng.standard_normal((n,) * d)
    ref = np.fft.fftn(x)
    s = np.max(np.abs(ref))
    assert np.max(np.abs(nufft.fft(x, -1) - ref)) < 1e-14 * s
    assert np.max(np.abs(nufft.fft(x, +1) - np.fft.ifftn(x) * n ** d)) < 1e-14 * s


# --------------------------------------------------------------------------- O1 direct
@pytest.mark.parametrize("d", [2, 3])
def test_direct_sums_reduce_to_uniform_dft(d):
    n, L = 8, 5.0
    h = L / n
    rng = np.random.default_rng(7)
    rho = rng.standard_normal((n,) * d)
    q = np.array(np.meshgrid(*[np.arange(-n // 2, n // 2)] * d, indexing="ij")).reshape(d, -1).T
    # q is in array-axis order; nodes are (k_x, k_y[, k_z]) = reversed
    k = 2 * math.pi * q[:, ::-1] / L
    got = direct.type2(rho, L, k)
    sign = (-1.0) ** q.sum(axis=1)
    ref = h ** d * sign * np.fft.fftn(rho)[tuple((q % n).T)]
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    c = rng.standard_normal(q.shape[0]) + 1j * rng.standard_normal(q.shape[0])
    f = direct.type1(c, d, n, L, k)
    C = np.zeros((n,) * d, complex)
    C[tuple((q % n).T)] = c * sign
    assert np.max(np.abs(f - np.fft.ifftn(C) * n ** d)) < 1e-12 * np.max(np.abs(f))


def test_grid_energy_equals_dual_energy():
    n, L = 10, 6.0
    rng = np.random.default_rng(3)
    rho = rng.standard_normal((n,) * 3)
    k, W = quadrature.nodes_weights(3, n, L, (6, 6, 12), "dipole", axis=[1.0, 2.0, 2.0])
    u, E, im, rh = direct.apply(rho, L, k, W, lam=1.7)
    assert abs(E - pipeline.energy_dual(rh, W, 1.7)) < 1e-12 * pipeline.energy_scale(rh, W, 1.7)
    assert im < 1e-12 * np.max(np.abs(u))


# --------------------------------------------------------------------------- O2 vs O1
# fp32ref is the reference of every FP32 parity test: measured 0.6-1.0e-8 on these cases,
# pinned at 3e-8 (three orders below the FP32 path's 1e-5 tolerance)
@pytest.mark.parametrize("setting,tol", [("parity", 3e-14), ("fine", 3e-11), ("fp32ref", 3e-8),
                                         ("paper12", 5e-11), ("paper6", 1e-5)])
@pytest.mark.parametrize("d,n,nodes", [(3, 12, (8, 8, 16)), (3, 16, (10, 10, 20)), (2, 32, (16, 32))])
def test_nufft_matches_direct_sums(setting, tol, d, n, nodes):
    L = 8.0
    rng = np.random.default_rng(n + d)
    rho = synth.gauss_iso(d, n, L) + 0.1 * rng.standard_normal((n,) * d)
    k, W = quadrature.nodes_weights(d, n, L, nodes)
    rd = direct.type2(rho, L, k)
    rn = pipeline.type2(rho, L, k, "nufft", setting)
    assert rel_inf(rn, rd) < tol
    fd = direct.type1(W * rd, d, n, L, k)
    fn = pipeline.type1(W * rd, d, n, L, k, "nufft", setting)
    assert rel_inf(fn, fd) < tol


def test_nufft_random_nodes_and_nonsquare_stencil_wrap():
    # nodes anywhere in [-pi, pi)^3, including next to the periodic seam
    rng = np.random.default_rng(11)
    n, L = 16, 8.0
    h = L / n
    t = rng.uniform(-math.pi, math.pi, size=(200, 3))
    t[:10] = math.pi * (1 - 1e-9) * np.sign(t[:10])
    c = rng.standard_normal(200) + 1j * rng.standard_normal(200)
    fd = direct.type1(c, 3, n, L, t / h)
    assert rel_inf(nufft.type1(c, t, 3, n, "parity"), fd) < 3e-14
    f = rng.standard_normal((n,) * 3) + 1j * rng.standard_normal((n,) * 3)
    ref = direct.type2(f.real, L, t / h) + 1j * direct.type2(f.imag, L, t / h)
    assert rel_inf(h ** 3 * nufft.type2(f, t, "parity"), ref) < 3e-14


# --------------------------------------------------------------------------- closed forms
def test_example7_closed_form_matches_printed_values():
    lam = 8 * math.pi / 3
    for case, gx, gz, E in read_golden("ex7_energy.txt"):
        got = cf.ex7_energy(float(gx), float(gz), lam)
        assert abs(got - float(E)) <= 2e-16 + 1e-15 * abs(float(E)), case


def test_t_integral_matches_erf_and_bessel_forms():
    z, y, x = synth.grid_coords(3, 16, 10.0)
    r = np.sqrt(x * x + y * y + z * z)
    ut = cf.aniso_gauss_potential((x, y, z), (1.0, 1.0, 1.0), kind="coulomb3d")
    assert rel_inf(ut, cf.coulomb3d_gauss(r)) < 1e-13
    yy, xx = synth.grid_coords(2, 32, 16.0)
    r2 = np.sqrt(xx * xx + yy * yy)
    ut2 = cf.aniso_gauss_potential((xx, yy), (1.3, 1.3), kind="coulomb2d")
    assert rel_inf(ut2, cf.coulomb2d_gauss(r2, 1.3)) < 1e-13


def test_pipeline_3d_coulomb_gaussian_closed_form():
    n, L = 32, 12.0
    rho = synth.gauss_iso(3, n, L)
    o = pipeline.oracle_eval(rho, L, (32, 32, 64), "coulomb")
    z, y, x = synth.grid_coords(3, n, L)
    r = np.sqrt(x * x + y * y + z * z)
    assert rel_inf(o["u"], cf.coulomb3d_gauss(r), r < 3) < 1e-8
    assert abs(o["E"] - cf.coulomb3d_gauss_energy()) < 1e-12
    assert abs(o["E"] - o["E_dual"]) < 1e-13
    assert o["imag_max"] < 1e-13
    # total charge: rho_hat at k = 0 is h^3 sum rho = pi^{3/2}
    q = pipeline.type2(rho, L, np.zeros((1, 3)), "direct")[0]
    assert abs(q - math.pi ** 1.5) < 1e-13


def test_pipeline_2d_coulomb_eq42():
    n, L, a = 64, 16.0, 1.3
    y, x = synth.grid_coords(2, n, L)
    rho = np.exp(-(x * x + y * y) / a)
    o = pipeline.oracle_eval(rho, L, (32, 64), "coulomb")
    r = np.sqrt(x * x + y * y)
    assert rel_inf(o["u"], cf.coulomb2d_gauss(r, a), r < 3) < 1e-12


def test_pipeline_example4_anisotropic_coulomb():
    n, L = 32, 12.0
    z, y, x = synth.grid_coords(3, n, L)
    o = pipeline.oracle_eval(cf.ex4_rho(x, y, z), L, (32, 32, 64), "coulomb")
    assert rel_inf(o["u"], cf.ex4_u(x, y, z), np.sqrt(x * x + y * y + z * z) < 3) < 1e-7


def test_pipeline_example5_dipole():
    n, L = 32, 12.0
    axis = np.array([-0.36589, -0.69481, 0.61916])
    z, y, x = synth.grid_coords(3, n, L)
    rho = cf.ex4_rho(x, y, z, (1.3, 1.5, 1.8))
    o = pipeline.oracle_eval(rho, L, (32, 32, 64), "dipole", axis=axis)
    assert rel_inf(o["u"], cf.ex5_u(x, y, z, axis), np.sqrt(x * x + y * y + z * z) < 3) < 1e-8


def test_pipeline_example7_energies():
    lam = 8 * math.pi / 3
    for case, gx, gz, E in read_golden("ex7_energy.txt"):
        gx, gz, E = float(gx), float(gz), float(E)
        L = 26.0 if gx < 0.5 else 12.0
        n = 64
        z, y, x = synth.grid_coords(3, n, L)
        rho = cf.ex7_rho(x, y, z, gx, gz)
        k, W = quadrature.nodes_weights(3, n, L, (32, 32, 64), "dipole", axis=[0, 0, 1])
        rh = pipeline.type2(rho, L, k)
        assert abs(pipeline.energy_dual(rh, W, lam) - E) < 1e-12, case


def test_config3_energy_closed_form_axis_dependence():
    # E(n) = E(z) P2(n_z) for a density symmetric about z (checked on a reduced grid)
    n, L = 48, 18.0
    rho = synth.gauss_axes(n, L, (1.0, 1.0, 2.25))
    axis = synth.random_unit(np.random.default_rng(synth.SEED_AXIS), 3)
    k, W = quadrature.nodes_weights(3, n, L, (32, 32, 64), "dipole", axis=axis)
    rh = pipeline.type2(rho, L, k)
    E = pipeline.energy_dual(rh, W)
    ref = cf.dipole_energy_cylindrical(axis, 1.0, 1.0 / 2.25, 1.0, scale=1.5 * math.pi ** 1.5)
    assert abs(E - ref) < 1e-9 * pipeline.energy_scale(rh, W)


# --------------------------------------------------------------------------- invariants
def _op(rho, L, nodes, kernel="coulomb", axis=None):
    return pipeline.oracle_eval(rho, L, nodes, kernel, axis=axis)


def test_invariants_linearity_symmetry_translation_sign():
    n, L, nodes = 16, 8.0, (10, 10, 20)
    rng = np.random.default_rng(5)
    r1 = rng.standard_normal((n,) * 3)
    r2 = rng.standard_normal((n,) * 3)
    u1, u2 = _op(r1, L, nodes)["u"], _op(r2, L, nodes)["u"]
    u12 = _op(2.0 * r1 - 3.0 * r2, L, nodes)["u"]
    assert rel_inf(u12, 2.0 * u1 - 3.0 * u2) < 1e-13
    assert abs(np.sum(u1 * r2) - np.sum(u2 * r1)) < 1e-12 * np.sum(np.abs(u1 * r2))
    assert _op(r1, L, nodes)["E"] > 0 and _op(r2, L, nodes)["E"] > 0
    # Toeplitz: a density supported away from the edges, shifted by whole cells
    g = np.zeros((n,) * 3)
    g[3:10, 4:11, 2:9] = rng.standard_normal((7, 7, 7))
    s = (2, 1, 3)
    gs = np.roll(g, s, axis=(0, 1, 2))
    ug, us = _op(g, L, nodes)["u"], _op(gs, L, nodes)["u"]
    assert rel_inf(us[2:, 1:, 3:], ug[:-2, :-1, :-3]) < 1e-13


def test_invariant_dipole_trace():
    n, L, nodes = 16, 8.0, (10, 10, 20)
    rho = np.random.default_rng(9).standard_normal((n,) * 3)
    us = [_op(rho, L, nodes, "dipole", axis=e)["u"] for e in np.eye(3)]
    assert np.max(np.abs(us[0] + us[1] + us[2])) < 1e-13 * np.max(np.abs(us[0]))


# --------------------------------------------------------------------------- other dipole kernels
def test_pipeline_example6_two_axis_dipole():
    a = (1.2, 1.45, 1.73)
    n = np.array([0.82778, 0.41505, -0.37751])
    m = np.array([0.31180, 0.93780, -0.15214])
    N, L = 40, 12.0
    z, y, x = synth.grid_coords(3, N, L)
    rho = cf.ex4_rho(x, y, z, a)
    o = pipeline.oracle_eval(rho, L, (40, 40, 80), "dipole", axis=n, axis2=m, setting="fine")
    ref = cf.ex6_u(x, y, z, n, m, a)
    mask = np.sqrt(x * x + y * y + z * z) < 3
    assert rel_inf(o["u"], ref, mask) < 1e-8


@pytest.mark.parametrize("ex", [2, 3])
def test_pipeline_examples_2_3_planar_dipole(ex):
    if ex == 2:
        a, n, m = 1.3, np.array([0.52460, -0.85135, 0.0]), None
    else:
        a, n, m = 1.8, np.array([-0.44404, -0.89600, 0.0]), np.array([0.85125, -0.52476, 0.0])
    N, L = 96, 24.0
    y, x = synth.grid_coords(2, N, L)
    rho = np.exp(-(x * x + y * y) / a)
    o = pipeline.oracle_eval(rho, L, (72, 144), "dipole", axis=n, axis2=m, setting="fine")
    ref = cf.ex23_u(x, y, a, n, m)
    assert rel_inf(o["u"], ref) < 1e-9


def test_planar_dipole_alpha_term_is_minus_alpha_rho():
    # the constant -alpha of the 2.5D symbol acts as -alpha times the (band-limited) density
    # (inside |x| < 6: at the box corners the phi rule with 144 nodes no longer resolves
    # exp(i k.x) for |k||x| up to ~ 140)
    N, L = 96, 24.0
    y, x = synth.grid_coords(2, N, L)
    rho = np.exp(-(x * x + y * y) / 1.3)
    n = np.array([0.3, -0.5, 0.8])
    o1 = pipeline.oracle_eval(rho, L, (72, 144), "dipole", axis=n, alpha=0.7, setting="fine")
    o0 = pipeline.oracle_eval(rho, L, (72, 144), "dipole", axis=n, alpha=0.0, setting="fine")
    mask = np.sqrt(x * x + y * y) < 6
    assert np.max(np.abs((o1["u"] - o0["u"]) + 0.7 * rho)[mask]) < 1e-10
