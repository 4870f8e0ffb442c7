"""Parity of the CUDA path (through the C-ABI) with the FP64 CPU oracle.

Tolerances (relative L-inf of u against the oracle; energy error divided by the energy scale
(lambda/2) sum_j |W_j| |rho_hat_j|^2, since dipolar energies can be near zero):
  FP64 path  <= 1e-10,  FP32 path <= 1e-5.
The oracle runs its own NUFFT (Section 2, Gaussian gridding) with its own nodes; only the
seeded densities from ``synth`` are shared.
"""
import math

import numpy as np
import pytest

import synth
from oracle import direct, pipeline, quadrature

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_4120_gb300 as p
    p.load_library()
    return p


def rel_inf(a, b):
    return float(np.max(np.abs(np.asarray(a) - b)) / np.max(np.abs(b)))


def run(pkg, wl, rho, eps=None, lam=1.0, **kw):
    eps = eps if eps is not None else (1e-6 if wl.precision == "fp32" else 1e-12)
    plan = pkg.Plan(wl.d, wl.n, wl.L, wl.kernel, axis=wl.axis, eps=eps, nodes=wl.nodes,
                    precision=wl.precision, device=0, **kw)
    dt = torch.float32 if wl.precision == "fp32" else torch.float64
    r = torch.from_numpy(rho).to(device="cuda:0", dtype=dt)
    u, E = plan.eval_energy(r, lam=lam)
    torch.cuda.synchronize()
    return plan, r, u.double().cpu().numpy(), float(E.item())


def check(wl, u, E, ref, tol):
    err = rel_inf(u, ref["u"])
    eerr = abs(E - ref["E"]) / ref["E_scale"]
    assert err <= tol, f"{wl.name}: rel L-inf {err:.3e} > {tol:.1e}"
    assert eerr <= tol, f"{wl.name}: energy error {eerr:.3e} > {tol:.1e}"
    return err, eerr


# --------------------------------------------------------------------------- node set
@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_plan_nodes_and_weights_match_oracle(pkg, name):
    wl = synth.CONFIGS[name]()
    plan = pkg.Plan(wl.d, wl.n, wl.L, wl.kernel, axis=wl.axis, nodes=wl.nodes, device=0)
    k, W = plan.nodes()
    kr, Wr = quadrature.nodes_weights(wl.d, wl.n, wl.L, wl.nodes, wl.kernel, axis=wl.axis)
    assert np.max(np.abs(k - kr)) <= 1e-13 * np.max(np.abs(kr))
    assert np.max(np.abs(W - Wr)) <= 1e-13 * np.max(np.abs(Wr))


# --------------------------------------------------------------------------- full configs
def test_parity_config1_fp64(pkg):
    wl = synth.config1()
    rho = wl.rho()
    ref = pipeline.oracle_eval(rho, wl.L, wl.nodes, wl.kernel, setting="parity")
    _, _, u, E = run(pkg, wl, rho)
    check(wl, u, E, ref, 1e-10)


def test_parity_config2_fp64(pkg):
    wl = synth.config2()
    rho = wl.rho()
    ref = pipeline.oracle_eval(rho, wl.L, wl.nodes, wl.kernel, setting="parity")
    _, _, u, E = run(pkg, wl, rho)
    check(wl, u, E, ref, 1e-10)


def test_parity_config3_fp32_dipole(pkg):
    wl = synth.config3()
    rho = wl.rho()
    ref = pipeline.oracle_eval(rho, wl.L, wl.nodes, wl.kernel, axis=wl.axis, setting="fp32ref")
    _, _, u, E = run(pkg, wl, rho)
    check(wl, u, E, ref, 1e-5)


@pytest.mark.slow
def test_parity_config4_fp32_full_size(pkg):
    wl = synth.config4()
    rho = wl.rho()
    ref = pipeline.oracle_eval(rho, wl.L, wl.nodes, wl.kernel, setting="fp32ref")
    _, _, u, E = run(pkg, wl, rho)
    check(wl, u, E, ref, 1e-5)


def test_config3_fp64_path_matches_oracle(pkg):
    wl = synth.config3()
    wl.precision = "fp64"
    rho = wl.rho()
    ref = pipeline.oracle_eval(rho, wl.L, wl.nodes, wl.kernel, axis=wl.axis, setting="parity")
    _, _, u, E = run(pkg, wl, rho)
    check(wl, u, E, ref, 1e-10)


# --------------------------------------------------------------------------- small / ragged
SMALL = [
    # d, n, L, kernel, nodes, precision
    (3, 24, 10.0, "coulomb", (12, 12, 24), "fp64"),      # fine grid 48 = 16*3 (radix 3)
    (3, 36, 12.0, "dipole", (16, 14, 30), "fp32"),       # fine grid 72 (radix 8,3,3)
    (3, 48, 12.0, "coulomb", (24, 20, 40), "fp32"),      # fine grid 96
    (3, 40, 10.0, "dipole", (20, 16, 36), "fp64"),       # fine grid 80 -> 96 (sigma 2.4)
    (2, 40, 12.0, "coulomb", (20, 44), "fp64"),          # 2D, fine grid 96
    (2, 100, 20.0, "coulomb", (30, 62), "fp32"),         # 2D, fine grid 200 -> 216
    (2, 256, 16.0, "coulomb", (64, 128), "fp32"),
]


@pytest.mark.parametrize("case", SMALL)
def test_parity_small_ragged(pkg, case):
    d, n, L, kernel, nodes, prec = case
    rng = np.random.default_rng(n * 7 + d)
    axis = synth.random_unit(rng, 3) if kernel == "dipole" else None
    cen, wid, wts = synth.mixture_params(rng, 5, d, L / 6, 0.6, 1.4, 0.5, 1.0)
    rho = synth.mixture(d, n, L, cen, wid, wts) + 0.05 * rng.standard_normal((n,) * d)
    wl = synth.Workload(name=f"small{case}", d=d, n=n, L=L, kernel=kernel, nodes=nodes,
                        precision=prec, tol=1e-5 if prec == "fp32" else 1e-10, axis=axis)
    ref = pipeline.oracle_eval(rho, L, nodes, kernel, axis=axis, setting="parity", lam=0.7)
    _, _, u, E = run(pkg, wl, rho, lam=0.7)
    check(wl, u, E, ref, wl.tol)
    assert np.max(np.abs(u)) > 0


# --------------------------------------------------------------------------- stage entry points
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_type2_matches_direct_sums(pkg, prec, tol):
    d, n, L, nodes = 3, 24, 8.0, (10, 10, 20)
    rng = np.random.default_rng(1)
    rho = rng.standard_normal((n,) * 3)
    k, W = quadrature.nodes_weights(d, n, L, nodes)
    ref = direct.type2(rho, L, k)
    plan = pkg.Plan(d, n, L, nodes=nodes, precision=prec, eps=1e-12 if prec == "fp64" else 1e-6, device=0)
    dt = torch.float64 if prec == "fp64" else torch.float32
    got = plan.type2(torch.from_numpy(rho).to("cuda:0", dt)).cpu().numpy().astype(np.complex128)
    assert rel_inf(got, ref) < tol


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-5)])
def test_type1_matches_direct_sums(pkg, prec, tol):
    d, n, L, nodes = 3, 24, 8.0, (10, 10, 20)
    rng = np.random.default_rng(2)
    k, W = quadrature.nodes_weights(d, n, L, nodes)
    c = rng.standard_normal(k.shape[0]) + 1j * rng.standard_normal(k.shape[0])
    ref = direct.type1(c, d, n, L, k).real
    plan = pkg.Plan(d, n, L, nodes=nodes, precision=prec, eps=1e-12 if prec == "fp64" else 1e-6, device=0)
    ct = torch.from_numpy(c).to("cuda:0", torch.complex128 if prec == "fp64" else torch.complex64)
    got = plan.type1(ct).double().cpu().numpy()
    assert rel_inf(got, ref) < tol


def test_type1_dominant_nodes_match_direct_sums(pkg):
    # a few nodes carry most of the weight (1e4 x the rest, 1e-3 of the nodes): their FP32
    # contributions exceed the range of the fused-multiply-add rounding and take the
    # conversion path, while the other nodes of the same subproblems stay on the fast one
    d, n, L, nodes = 3, 24, 8.0, (10, 10, 20)
    rng = np.random.default_rng(3)
    k, W = quadrature.nodes_weights(d, n, L, nodes)
    M = k.shape[0]
    c = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    heavy = rng.choice(M, size=max(2, M // 1000), replace=False)
    c[heavy] *= 1e4
    for cc, tol in ((c, 1e-5), (np.where(np.isin(np.arange(M), heavy), 0, c), 1e-5)):
        ref = direct.type1(cc, d, n, L, k).real
        plan = pkg.Plan(d, n, L, nodes=nodes, precision="fp32", eps=1e-6, device=0)
        got = plan.type1(torch.from_numpy(cc).to("cuda:0", torch.complex64)).double().cpu().numpy()
        plan.close()
        assert rel_inf(got, ref) < tol


def test_energy_entry_point_and_host_path(pkg):
    wl = synth.config1()
    rho = wl.rho()
    plan, r, u, E = run(pkg, wl, rho)
    # standalone energy of the device u equals the fused one
    ut = torch.from_numpy(u).to("cuda:0")
    E2 = plan.energy(r, ut, lam=1.0)
    assert abs(E2 - E) <= 1e-14 * abs(E)
    assert abs(E2 - pipeline.energy(u, rho, wl.L)) <= 1e-14 * abs(E)
    # host-buffer path
    uh, Eh = plan.eval_host(torch.from_numpy(rho).pin_memory(), lam=1.0)
    assert rel_inf(uh.numpy(), u) < 1e-13
    assert abs(Eh - E) < 1e-13 * abs(E)


def test_repeat_evaluations_agree(pkg):
    wl = synth.config1()
    rho = wl.rho()
    plan, r, u1, E1 = run(pkg, wl, rho)
    u2, E2 = plan.eval_energy(r)
    torch.cuda.synchronize()
    # spreading adds with atomics, so the order of the additions (not the result's accuracy)
    # may change between runs: agreement to a few ulps of the largest value
    assert rel_inf(u2.cpu().numpy(), u1) < 1e-13
    assert abs(float(E2.item()) - E1) < 1e-13 * abs(E1)


def test_linearity_and_dipole_trace_on_gpu(pkg):
    n, L, nodes = 32, 12.0, (16, 16, 32)
    rng = np.random.default_rng(4)
    rho = torch.from_numpy(rng.standard_normal((n,) * 3)).to("cuda:0")
    us = []
    for e in np.eye(3):
        p = pkg.Plan(3, n, L, "dipole", axis=e, nodes=nodes, precision="fp64", eps=1e-12, device=0)
        us.append(p.eval(rho).cpu().numpy())
    assert np.max(np.abs(us[0] + us[1] + us[2])) < 1e-11 * np.max(np.abs(us[0]))


def test_bad_tensor_arguments_raise(pkg):
    plan = pkg.Plan(3, 32, 12.0, nodes=(8, 8, 16), device=0)
    with pytest.raises(ValueError):
        plan.eval(torch.zeros((32, 32, 31), device="cuda:0"))
    with pytest.raises(ValueError):
        plan.eval(torch.zeros((32, 32, 32), dtype=torch.float64, device="cuda:0"))
    with pytest.raises(TypeError):
        plan.eval(torch.zeros((32, 32, 32)))
    with pytest.raises(pkg.NlintError):
        pkg.Plan(3, 12, 6.0, eps=1e-12, device=0)   # fine grid too small for w = 13


# --------------------------------------------------------------------------- other dipole kernels
OTHER = [
    # d, n, L, nodes, precision, axis, axis2, alpha
    (3, 32, 12.0, (24, 24, 48), "fp64", (0.82778, 0.41505, -0.37751), (0.31180, 0.93780, -0.15214), 0.0),
    (3, 48, 12.0, (32, 32, 64), "fp32", (0.3, -0.5, 0.8), (-0.7, 0.1, 0.2), 0.0),
    (2, 64, 16.0, (40, 80), "fp64", (0.52460, -0.85135, 0.0), None, 0.0),
    (2, 96, 16.0, (48, 96), "fp64", (0.3, -0.5, 0.8), (0.85125, -0.52476, 0.1), 0.7),
    (2, 128, 20.0, (64, 128), "fp32", (-0.44404, -0.89600, 0.0), (0.85125, -0.52476, 0.0), -0.3),
]


@pytest.mark.parametrize("case", OTHER)
def test_parity_two_axis_and_planar_dipoles(pkg, case):
    d, n, L, nodes, prec, axis, axis2, alpha = case
    rng = np.random.default_rng(n + 3 * d)
    cen, wid, wts = synth.mixture_params(rng, 4, d, L / 8, 0.7, 1.3, 0.5, 1.0)
    rho = synth.mixture(d, n, L, cen, wid, wts)
    tol = 1e-5 if prec == "fp32" else 1e-10
    plan = pkg.Plan(d, n, L, "dipole", axis=axis, axis2=axis2, alpha=alpha, nodes=nodes,
                    precision=prec, eps=1e-6 if prec == "fp32" else 1e-12, device=0)
    k, W = plan.nodes()
    kr, Wr = quadrature.nodes_weights(d, n, L, nodes, "dipole", axis=axis, axis2=axis2, alpha=alpha)
    assert np.max(np.abs(W - Wr)) <= 1e-13 * np.max(np.abs(Wr))
    dt = torch.float32 if prec == "fp32" else torch.float64
    u, E = plan.eval_energy(torch.from_numpy(rho).to("cuda:0", dt), lam=1.3)
    torch.cuda.synchronize()
    ref = pipeline.oracle_eval(rho, L, nodes, "dipole", axis=axis, axis2=axis2, alpha=alpha,
                               lam=1.3, setting="parity")
    err = rel_inf(u.double().cpu().numpy(), ref["u"])
    assert err <= tol, f"rel L-inf {err:.3e}"
    assert abs(float(E.item()) - ref["E"]) <= tol * ref["E_scale"]


# --------------------------------------------------------------------------- energy-only path
@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_energy_only_matches_oracle_dual_energy(pkg, name):
    wl = synth.CONFIGS[name]()
    rho = wl.rho()
    setting = "fp32ref" if wl.precision == "fp32" else "parity"
    ref = pipeline.oracle_eval(rho, wl.L, wl.nodes, wl.kernel, axis=wl.axis, setting=setting, lam=1.7)
    plan = pkg.Plan(wl.d, wl.n, wl.L, wl.kernel, axis=wl.axis, nodes=wl.nodes, precision=wl.precision,
                    eps=1e-6 if wl.precision == "fp32" else 1e-12, device=0)
    dt = torch.float32 if wl.precision == "fp32" else torch.float64
    r = torch.from_numpy(rho).to("cuda:0", dt)
    E = float(plan.energy_only(r, lam=1.7).item())
    _, E2 = plan.eval_energy(r, lam=1.7)
    torch.cuda.synchronize()
    tol = wl.tol
    assert abs(E - ref["E_dual"]) <= tol * ref["E_scale"], (E, ref["E_dual"])
    assert abs(E - float(E2.item())) <= tol * ref["E_scale"]


# --------------------------------------------------------------------------- Toeplitz form
@pytest.mark.parametrize("name", ["c1", "c2", "c3"])
def test_toeplitz_form_matches_oracle_and_nufft_path(pkg, name):
    wl = synth.CONFIGS[name]()
    rho = wl.rho()
    setting = "fp32ref" if wl.precision == "fp32" else "parity"
    ref = pipeline.oracle_eval(rho, wl.L, wl.nodes, wl.kernel, axis=wl.axis, setting=setting, lam=0.8)
    plan = pkg.Plan(wl.d, wl.n, wl.L, wl.kernel, axis=wl.axis, nodes=wl.nodes, precision=wl.precision,
                    eps=1e-6 if wl.precision == "fp32" else 1e-12, device=0)
    dt = torch.float32 if wl.precision == "fp32" else torch.float64
    r = torch.from_numpy(rho).to("cuda:0", dt)
    plan.toeplitz()
    ut, Et = plan.eval_toeplitz(r, lam=0.8)
    un, En = plan.eval_energy(r, lam=0.8)
    torch.cuda.synchronize()
    ut = ut.double().cpu().numpy()
    assert rel_inf(ut, ref["u"]) <= wl.tol
    assert rel_inf(ut, un.double().cpu().numpy()) <= wl.tol
    assert abs(float(Et.item()) - ref["E"]) <= wl.tol * ref["E_scale"]


@pytest.mark.parametrize("case", SMALL[:4] + [SMALL[5]])
def test_toeplitz_small_ragged(pkg, case):
    d, n, L, kernel, nodes, prec = case
    rng = np.random.default_rng(n * 11 + d)
    axis = synth.random_unit(rng, 3) if kernel == "dipole" else None
    cen, wid, wts = synth.mixture_params(rng, 5, d, L / 6, 0.6, 1.4, 0.5, 1.0)
    rho = synth.mixture(d, n, L, cen, wid, wts) + 0.05 * rng.standard_normal((n,) * d)
    tol = 1e-5 if prec == "fp32" else 1e-10
    ref = pipeline.oracle_eval(rho, L, nodes, kernel, axis=axis, setting="parity")
    plan = pkg.Plan(d, n, L, kernel, axis=axis, nodes=nodes, precision=prec,
                    eps=1e-6 if prec == "fp32" else 1e-12, device=0)
    plan.toeplitz()
    dt = torch.float32 if prec == "fp32" else torch.float64
    u, E = plan.eval_toeplitz(torch.from_numpy(rho).to("cuda:0", dt))
    torch.cuda.synchronize()
    assert rel_inf(u.double().cpu().numpy(), ref["u"]) <= tol
    assert abs(float(E.item()) - ref["E"]) <= tol * ref["E_scale"]


def test_toeplitz_requires_precompute(pkg):
    plan = pkg.Plan(3, 32, 12.0, nodes=(8, 8, 16), device=0)
    with pytest.raises(pkg.NlintError):
        plan.eval_toeplitz(torch.zeros((32, 32, 32), device="cuda:0"))
