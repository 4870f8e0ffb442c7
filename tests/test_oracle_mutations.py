"""Plant plausible mistakes in the oracle (CPU only) and check that a pin catches each one.

Each mutation patches one oracle function for the duration of a test; the pin it should trip
is re-run and must fail.  This shows the pins are sharp enough to see a dropped term, a wrong
sign, a transposed operand or a wrong index.
"""
import math

import numpy as np
import pytest

import synth
from oracle import closed_forms as cf
from oracle import direct, pipeline, quadrature

ORIG_NW = quadrature.nodes_weights
ORIG_UHAT = quadrature.u_hat
ORIG_T2 = pipeline.type2


def _interior_err(kernel, axis, rho_fn, u_fn, method="nufft", n=20):
    L = 10.0
    z, y, x = synth.grid_coords(3, n, L)
    o = pipeline.oracle_eval(rho_fn(x, y, z), L, (n, n, 2 * n), kernel, axis=axis,
                             method=method)
    ref = u_fn(x, y, z)
    m = np.sqrt(x * x + y * y + z * z) < 3
    return np.max(np.abs(o["u"][m] - ref[m])) / np.max(np.abs(ref[m]))


AX = np.array([-0.36589, -0.69481, 0.61916])
MIX_C = np.array([[1.5, -0.5, 0.3], [-1.0, 1.0, -0.8]])
MIX_S = np.array([1.0, 1.2])
MIX_W = np.array([1.0, 0.6])


def ex4_err():
    return _interior_err("coulomb", None, cf.ex4_rho, cf.ex4_u)


def ex5_err():
    a = (1.3, 1.5, 1.8)
    return _interior_err("dipole", AX, lambda x, y, z: cf.ex4_rho(x, y, z, a),
                         lambda x, y, z: cf.ex5_u(x, y, z, AX, a))


def mix_err(method="nufft", n=20):
    # an off-centre mixture: not even under x -> -x, so a conjugated transform shows
    return _interior_err(
        "coulomb", None,
        lambda x, y, z: sum(w * np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / s ** 2)
                            for c, s, w in zip(MIX_C, MIX_S, MIX_W)),
        lambda x, y, z: cf.coulomb3d_mixture(x, y, z, MIX_C, MIX_S, MIX_W), method, n)


def test_unmutated_baseline_passes():
    assert ex4_err() < 1e-4 and ex5_err() < 1e-4 and mix_err() < 1e-4
    assert ex2_err() < 1e-4 and ex6_err() < 1e-4


def _drop_sin(d, n, L, nodes, kernel="coulomb", axis=None, axis2=None, alpha=0.0, P=None):
    k, W = ORIG_NW(d, n, L, nodes, kernel, axis, axis2, alpha, P)
    if d == 3:
        st = np.sqrt(k[:, 0] ** 2 + k[:, 1] ** 2) / np.linalg.norm(k, axis=1)
        W = W / st
    return k, W


def _flip_dipole(k, d, kernel, axis=None, axis2=None, alpha=0.0):
    v = ORIG_UHAT(k, d, kernel, axis, axis2, alpha)
    return -v if kernel == "dipole" else v


def _transpose_nodes(d, n, L, nodes, kernel="coulomb", axis=None, axis2=None, alpha=0.0, P=None):
    k, W = ORIG_NW(d, n, L, nodes, kernel, axis, axis2, alpha, P)
    return k[:, ::-1].copy(), W


def _planar_dipole_no_half(k, d, kernel, axis=None, axis2=None, alpha=0.0):
    # drops the 1/2 of the 2.5D dipole symbol (eqs. dipkernelF2d / dipkernelF2dd)
    v = ORIG_UHAT(k, d, kernel, axis, axis2, alpha)
    return 2.0 * v if (kernel == "dipole" and d == 2) else v


def _two_axis_uses_n_twice(k, d, kernel, axis=None, axis2=None, alpha=0.0):
    # ignores the second orientation m of eq. dipkerneldF
    return ORIG_UHAT(k, d, kernel, axis, None, alpha)


def ex2_err():
    a, n = 1.3, np.array([0.52460, -0.85135, 0.0])
    y, x = synth.grid_coords(2, 64, 24.0)
    rho = np.exp(-(x * x + y * y) / a)
    o = pipeline.oracle_eval(rho, 24.0, (48, 96), "dipole", axis=n)
    ref = cf.ex23_u(x, y, a, n)
    m = np.sqrt(x * x + y * y) < 4
    return np.max(np.abs(o["u"][m] - ref[m])) / np.max(np.abs(ref[m]))


def ex6_err():
    a = (1.2, 1.45, 1.73)
    n, mm = np.array([0.82778, 0.41505, -0.37751]), np.array([0.31180, 0.93780, -0.15214])
    z, y, x = synth.grid_coords(3, 20, 10.0)
    o = pipeline.oracle_eval(cf.ex4_rho(x, y, z, a), 10.0, (20, 20, 40), "dipole", axis=n, axis2=mm)
    ref = cf.ex6_u(x, y, z, n, mm, a)
    m = np.sqrt(x * x + y * y + z * z) < 3
    return np.max(np.abs(o["u"][m] - ref[m])) / np.max(np.abs(ref[m]))


def _conj_type2(rho, L, k, method="nufft", setting="parity"):
    return np.conj(ORIG_T2(rho, L, k, method, setting))


@pytest.mark.parametrize("mutation", ["drop_sin", "flip_dipole", "transpose", "conj_type2",
                                      "grid_offset", "planar_half", "two_axis"])
def test_pins_catch_mutation(monkeypatch, mutation):
    if mutation == "drop_sin":
        monkeypatch.setattr(quadrature, "nodes_weights", _drop_sin)
        err = ex4_err()
    elif mutation == "flip_dipole":
        monkeypatch.setattr(quadrature, "u_hat", _flip_dipole)
        err = ex5_err()
    elif mutation == "transpose":
        monkeypatch.setattr(quadrature, "nodes_weights", _transpose_nodes)
        err = max(ex4_err(), ex5_err())
    elif mutation == "planar_half":
        monkeypatch.setattr(quadrature, "u_hat", _planar_dipole_no_half)
        err = ex2_err()
    elif mutation == "two_axis":
        monkeypatch.setattr(quadrature, "u_hat", _two_axis_uses_n_twice)
        err = ex6_err()
    elif mutation == "conj_type2":
        monkeypatch.setattr(pipeline, "type2", _conj_type2)
        err = mix_err()
    else:
        # type-2 sampled on a grid offset by one cell (x_i = -L/2 + (i+1) h) while type-1
        # uses the right one
        def offset_type2(rho, L, k, method="nufft", setting="parity"):
            h = L / rho.shape[0]
            return ORIG_T2(rho, L, k, method, setting) * np.exp(-1j * (k @ np.full(k.shape[1], h)))
        monkeypatch.setattr(pipeline, "type2", offset_type2)
        err = mix_err()
    assert err > 5e-2, f"{mutation} not detected (err={err:.2e})"


def test_fp32ref_pin_catches_narrow_stencil(monkeypatch):
    # The FP32 reference setting run with half its stencil (w = 8 instead of 16, tau balanced
    # for w = 8) must fail the 3e-8 pin against the direct sums (Section 2 with eqs. 3.2/3.7).
    from oracle import nufft
    orig = nufft.params

    def narrow(N, setting="parity"):
        if setting == "fp32ref":
            tau = (8 * np.pi / 2) / (2.0 * N ** 2 * np.sqrt(2.0))
            return 2 * N, 8, tau
        return orig(N, setting)

    d, n, nodes, L = 3, 12, (8, 8, 16), 8.0
    rho = synth.gauss_iso(d, n, L) + 0.1 * np.random.default_rng(n + d).standard_normal((n,) * d)
    k, W = quadrature.nodes_weights(d, n, L, nodes)
    rd = direct.type2(rho, L, k)
    ok = np.max(np.abs(pipeline.type2(rho, L, k, "nufft", "fp32ref") - rd)) / np.max(np.abs(rd))
    assert ok < 3e-8
    monkeypatch.setattr(nufft, "params", narrow)
    bad = np.max(np.abs(pipeline.type2(rho, L, k, "nufft", "fp32ref") - rd)) / np.max(np.abs(rd))
    assert bad > 3e-8, f"narrow fp32ref stencil not detected (err={bad:.2e})"
