"""Pins of the Algorithm 2 oracle (Section 3.3, eq. 3.9): partition functions, the regular-FFT
part I_1 against brute-force sums, each part and their sum against closed forms, the reduction
to Algorithm 1 when p_d = 1, the dual energy, and planted mistakes that the pins must catch."""
import math

import numpy as np
import pytest

import synth
from oracle import alg2, closed_forms as cf, pipeline

AX = np.array([-0.36589, -0.69481, 0.61916])


# ----------------------------------------------------------------- partition functions
def test_p2_is_a_symmetric_monotone_step():
    r0, r1 = 0.75, 10.0
    c = 0.5 * (r0 + r1)
    t = np.linspace(0.0, 6.0, 61)
    up = alg2.p2(np.stack([c + t, 0 * t], 1), r0, r1)
    dn = alg2.p2(np.stack([c - t, 0 * t], 1), r0, r1)
    assert np.max(np.abs(up + dn - 1.0)) < 1e-15          # erfc(x) + erfc(-x) = 2
    assert abs(alg2.p2(np.array([[c, 0.0]]), r0, r1)[0] - 0.5) < 1e-16
    k = np.stack([np.linspace(0, 12, 200), np.zeros(200)], 1)
    v = alg2.p2(k, r0, r1)
    assert np.all(np.diff(v) <= 0) and v[0] >= 1 - 1e-16
    assert alg2.p2(np.array([[r1, 0.0]]), r0, r1)[0] < 2e-17


def test_p3_and_the_coulomb_limit_at_zero():
    a = 0.7
    assert alg2.p3(np.zeros((1, 3)), a)[0] == 1.0
    # (1 - p3) / k^2 -> 1/a - k^2/(2 a^2): the value M takes at k = 0 is the limit
    n, L = 4, 400.0                                    # first frequency dk = pi / 400
    M = alg2.multiplier_I1(3, n, L, "coulomb", a=a)
    assert M[0, 0, 0] == 1.0 / a
    dk = math.pi / L
    series = 1.0 / a - dk * dk / (2 * a * a) + dk ** 4 / (6 * a ** 3)
    assert abs(M[0, 0, 1] - series) < dk ** 6 / (24 * a ** 4) + 1e-15
    assert abs(M[0, 0, 1] - M[0, 0, 0]) < dk * dk / a ** 2   # continuous at k = 0


def test_multiplier_entries_by_hand():
    """n = 4, h = 1: DFT frequencies pi/4 * g (g = 0, 1, 2, 3, -4, -3, -2, -1), P = pi."""
    a = 0.9
    n, L = 4, 4.0
    q = math.pi / 4
    one = lambda k2: -math.expm1(-k2 / a)
    M = alg2.multiplier_I1(3, n, L, "dipole", axis=(0.0, 0.0, 1.0), a=a)
    # array axis 0 is z, axis 2 is x
    assert abs(M[1, 0, 0] - 2.0 * one(q * q)) < 1e-15          # k = (0, 0, q): -1 + 3
    assert abs(M[0, 0, 1] + one(q * q)) < 1e-15                # k = (q, 0, 0): -1
    assert abs(M[0, 4, 0] + one(math.pi ** 2)) < 1e-15         # k = (0, -pi, 0), on the sphere
    assert M[0, 4, 4] == 0.0 and M[3, 3, 3] == 0.0            # |g| > 4: outside the ball
    assert M[0, 0, 0] == 0.0                                   # dipole: limit 0
    kk = q * q * (1 + 4 + 9)                                   # g = (z 1, y 2, x 3)
    assert abs(M[1, 2, 3] - (-1 + 3 * q * q / kk) * one(kk)) < 1e-15
    M2 = alg2.multiplier_I1(2, n, L, "coulomb", r0=0.3, r1=4.0)
    assert M2[0, 0] == 0.0
    k = math.sqrt(5) * q                                        # (y 1, x 2) and (y 2, x 1)
    exp = (1.0 - 0.5 * math.erfc(12 * (k - 2.15) / 3.7)) / k
    assert abs(M2[1, 2] - exp) < 1e-15 and abs(M2[2, 1] - exp) < 1e-15


# ----------------------------------------------------------------- I_1 against brute force
def _I1_brute(rho, M):
    """u1_m = q^{-d} sum_g e^{2 pi i g.m/q} M_g sum_l rho_l e^{-2 pi i g.l/q}, q = n_pad."""
    d, n, q = rho.ndim, rho.shape[0], M.shape[0]
    g1 = np.concatenate([np.arange(0, q // 2), np.arange(-(q // 2), 0)])  # fftfreq integers
    G = np.stack([a.ravel() for a in np.meshgrid(*([g1] * d), indexing="ij")], 1)
    Lx = np.stack([a.ravel() for a in np.meshgrid(*([np.arange(n)] * d), indexing="ij")], 1)
    ph = np.exp(-2j * np.pi * (G @ Lx.T) / q)                       # (q^d, n^d)
    F = ph @ rho.ravel()
    u = (ph.conj().T @ (M.ravel() * F)) / q ** d
    return u.real.reshape((n,) * d), float(np.max(np.abs(u.imag)))


@pytest.mark.parametrize("d,n,n_pad", [(3, 6, None), (2, 10, None), (3, 5, 12), (2, 10, 24)])
def test_I1_matches_brute_force_sums(d, n, n_pad):
    L = 3.0 * n / 4
    rng = np.random.default_rng(7 + d)
    rho = rng.standard_normal((n,) * d)
    if d == 3:
        M = alg2.multiplier_I1(3, n, L, "dipole", axis=AX, a=1.3, n_pad=n_pad)
    else:
        M = alg2.multiplier_I1(2, n, L, "dipole", axis=AX, axis2=(0.2, 0.9, 0.1), alpha=0.4,
                               r0=0.2, r1=3.0, n_pad=n_pad)
    u, _ = alg2.I1(rho, M)
    ub, im = _I1_brute(rho, M)
    assert np.max(np.abs(u - ub)) < 1e-13 * np.max(np.abs(ub))
    assert im < 1e-13 * np.max(np.abs(ub))                        # the operator is real


# ----------------------------------------------------------------- closed forms
def _grid3(n, L):
    z, y, x = synth.grid_coords(3, n, L)
    return x, y, z


def _coulomb_parts_err(n=40, L=16.0, s=1.5):
    x, y, z = _grid3(n, L)
    r = np.sqrt(x * x + y * y + z * z)
    rho = np.exp(-r * r / (s * s))
    prm = alg2.default_parameters(3, n, L, "fp64")
    out = alg2.alg2_eval(rho, L, prm["nodes2"], a=prm["a"], P2=prm["P2"])
    ue = cf.coulomb3d_gauss(r, s)
    s2 = math.sqrt(s * s + 4.0 / prm["a"])                       # rho smoothed by p_3
    u2e = cf.coulomb3d_gauss(r, s2, (s / s2) ** 3)
    m = np.max(np.abs(ue))
    return (np.max(np.abs(out["u1"] - (ue - u2e))) / m, np.max(np.abs(out["u2"] - u2e)) / m,
            np.max(np.abs(out["u"] - ue)) / m, out, cf.coulomb3d_gauss_energy(s))


def test_alg2_coulomb_parts_match_closed_forms():
    e1, e2, e, out, E_ex = _coulomb_parts_err()
    assert e1 < 1e-12 and e2 < 1e-12 and e < 1e-12, (e1, e2, e)
    assert abs(out["E"] - E_ex) < 1e-12 * E_ex
    assert abs(out["E"] - out["E_dual"]) < 1e-12 * out["E_scale"]
    assert out["imag_max"] < 1e-12


def test_alg2_dipole_matches_closed_form():
    n, L, s = 40, 16.0, 1.5
    x, y, z = _grid3(n, L)
    r2 = x * x + y * y + z * z
    rho = np.exp(-r2 / (s * s))
    prm = alg2.default_parameters(3, n, L, "fp64")
    out = alg2.alg2_eval(rho, L, prm["nodes2"], "dipole", axis=AX, a=prm["a"], P2=prm["P2"])
    ue = -rho + cf.aniso_gauss_potential((x, y, z), (s * s,) * 3, kind="dipole_nn3d", axis=AX)
    s2sq = s * s + 4.0 / prm["a"]
    amp = (s * s / s2sq) ** 1.5
    u2e = amp * (-np.exp(-r2 / s2sq) + cf.aniso_gauss_potential((x, y, z), (s2sq,) * 3,
                                                                kind="dipole_nn3d", axis=AX))
    m = np.max(np.abs(ue))
    assert np.max(np.abs(out["u"] - ue)) < 1e-11 * m
    assert np.max(np.abs(out["u2"] - u2e)) < 1e-11 * m


def test_alg2_2d_matches_eq_4_2():
    n, L, a0 = 64, 16.0, 1.0
    z = synth.grid_coords(2, n, L)
    y, x = z
    r = np.sqrt((x - 1.3) ** 2 + (y + 0.7) ** 2)
    rho = np.exp(-r * r / a0)
    prm = alg2.default_parameters(2, n, L, "fp64")
    out = alg2.alg2_eval(rho, L, prm["nodes2"], r0=prm["r0"], r1=prm["r1"], P2=prm["P2"])
    ue = cf.coulomb2d_gauss(r, a0)
    assert np.max(np.abs(out["u"] - ue)) < 1e-11 * np.max(np.abs(ue))
    assert abs(out["E"] - out["E_dual"]) < 1e-12 * out["E_scale"]


# ----------------------------------------------------------------- reduction to Algorithm 1
@pytest.mark.parametrize("d", [3, 2])
def test_alg2_with_p_equal_one_is_algorithm_1(d):
    n, L = 8, 6.0
    rng = np.random.default_rng(11)
    rho = rng.standard_normal((n,) * d)
    P = math.pi / (L / n)
    if d == 3:
        nodes, kw = (6, 6, 12), {"a": 1e300}
        kern = dict(kernel="dipole", axis=AX)
    else:
        nodes, kw = (8, 16), {"r0": 1e6, "r1": 2e6}
        kern = dict(kernel="coulomb")
    out = alg2.alg2_eval(rho, L, nodes, P2=P, method="direct", **kern, **kw)
    ref = pipeline.oracle_eval(rho, L, nodes, method="direct", **kern)
    assert np.max(np.abs(out["u1"])) < 1e-290 or np.max(np.abs(out["u1"])) == 0.0
    assert np.max(np.abs(out["u"] - ref["u"])) < 1e-14 * np.max(np.abs(ref["u"]))
    assert abs(out["E"] - ref["E"]) < 1e-14 * ref["E_scale"]


# ----------------------------------------------------------------- planted mistakes
def test_dropping_one_minus_p_in_I1_is_caught(monkeypatch):
    monkeypatch.setattr(alg2, "multiplier_I1",
                        lambda d, n, L, kernel="coulomb", axis=None, axis2=None, alpha=0.0,
                        a=None, r0=None, r1=None, P=None, n_pad=None:
                        _full_symbol(d, n, L, kernel, axis, P))
    e1, _, e, _, _ = _coulomb_parts_err(n=24, L=12.0, s=1.5)
    assert e1 > 1e-6 and e > 1e-6


def _full_symbol(d, n, L, kernel, axis, P):
    """U_hat on the DFT grid without the (1 - p) factor (0 at k = 0)."""
    from oracle import quadrature
    ks = np.meshgrid(*alg2.frequencies(d, n, L), indexing="ij")
    k = np.stack([ks[d - 1 - i].ravel() for i in range(d)], 1)
    k2 = np.sum(k * k, 1)
    kz = k.copy()
    kz[k2 == 0] = 1.0
    M = quadrature.u_hat(kz, d, kernel, axis)
    M[k2 == 0] = 0.0
    P = math.pi * n / L if P is None else P
    M[k2 > (P * (1 + 1e-12)) ** 2] = 0.0
    return M.reshape((2 * n,) * d)


def test_dropping_p_in_I2_weights_is_caught(monkeypatch):
    from oracle import quadrature
    monkeypatch.setattr(alg2, "I2_nodes", lambda d, n, L, nodes2, kernel="coulomb", axis=None,
                        axis2=None, alpha=0.0, a=None, r0=None, r1=None, P2=None:
                        quadrature.nodes_weights(d, n, L, nodes2, kernel, axis, axis2, alpha, P2))
    _, e2, e, _, _ = _coulomb_parts_err(n=24, L=12.0, s=1.5)
    assert e2 > 1e-6 and e > 1e-6


def test_padding_without_oversampling_is_caught(monkeypatch):
    def bad_I1(rho, M):
        d = rho.ndim
        # circular convolution on the n-point grid (the frequencies of every other 2n bin)
        sub = M[(slice(None, None, 2),) * d]
        v = np.fft.ifftn(sub * np.fft.fftn(rho))
        return v.real.copy(), np.fft.fftn(rho)

    monkeypatch.setattr(alg2, "I1", bad_I1)
    n, L = 6, 4.5
    rho = np.random.default_rng(3).standard_normal((n,) * 3)
    M = alg2.multiplier_I1(3, n, L, "dipole", axis=AX, a=1.3)
    u, _ = alg2.I1(rho, M)
    ub, _ = _I1_brute(rho, M)
    assert np.max(np.abs(u - ub)) > 1e-3 * np.max(np.abs(ub))


def test_transposed_frequency_axes_are_caught(monkeypatch):
    from oracle import quadrature
    orig = quadrature.u_hat

    def swapped(k, d, kernel, axis=None, axis2=None, alpha=0.0):
        return orig(k[:, ::-1], d, kernel, axis, axis2, alpha)

    monkeypatch.setattr(quadrature, "u_hat", swapped)
    with pytest.raises(AssertionError):
        test_multiplier_entries_by_hand()
