"""GPU parity of Algorithm 2 (Section 3.3, eq. 3.9) against the FP64 oracle (oracle.alg2) on the
plan's own parameters (fine-grid size for I_1's padding, a / R0, R1, P2, I_2's nodes), and at
the 256^3 benchmark size against the analytic potential and the Algorithm 1 path."""
import numpy as np
import pytest

import synth
from oracle import alg2, closed_forms as cf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
AX = (-0.36589, -0.69481, 0.61916)


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_4120_gb300 as p
    p.load_library()
    return p


def _oracle_for(plan, rho, kernel, axis=None, axis2=None, alpha=0.0, lam=1.0):
    inf = plan.info
    nodes = (inf["n_r"], inf["n_theta"], inf["n_phi"]) if inf["d"] == 3 else (inf["n_r"], inf["n_phi"])
    kw = dict(a=inf["pu_a"]) if inf["d"] == 3 else dict(r0=inf["pu_r0"], r1=inf["pu_r1"])
    return alg2.alg2_eval(rho, inf["L"], nodes, kernel, axis=axis, axis2=axis2, alpha=alpha,
                          P=inf["P"], P2=inf["P2"], lam=lam, n_pad=inf["n_fine"], **kw)


CASES = [
    # d, n, L, kernel, precision, extra
    (3, 32, 16.0, "coulomb", "fp64", {}),
    (3, 36, 12.0, "dipole", "fp32", {"axis": AX}),                   # fine grid 72, ragged tiles
    (3, 24, 10.0, "dipole", "fp64", {"axis": AX, "axis2": (0.3118, 0.9378, -0.1521)}),
    (2, 64, 16.0, "coulomb", "fp64", {}),
    (2, 100, 20.0, "dipole", "fp32", {"axis": (0.5246, -0.85135, 0.0), "alpha": 0.7}),
    # grids wide enough for I_2's frequency window (windowed I_2 passes)
    (3, 48, 16.0, "dipole", "fp32", {"axis": AX}),
    (3, 64, 16.0, "coulomb", "fp64", {}),
    (2, 128, 16.0, "coulomb", "fp64", {}),
]


@pytest.mark.parametrize("case", CASES)
def test_alg2_matches_oracle(pkg, case):
    d, n, L, kernel, prec, extra = case
    rng = np.random.default_rng(1311 + n)
    c, s, w = synth.mixture_params(rng, 4, d, L / 8, 0.8, 1.4, 0.5, 1.0)
    rho = synth.mixture(d, n, L, c, s, w)
    plan = pkg.Plan(d, n, L, kernel, precision=prec, eps=1e-6 if prec == "fp32" else 1e-12,
                    algorithm=2, device=0, **extra)
    assert plan.info["algorithm"] == 2
    dt = torch.float32 if prec == "fp32" else torch.float64
    u, E = plan.eval_energy(torch.from_numpy(rho).to("cuda:0", dt), lam=1.0)
    torch.cuda.synchronize()
    ref = _oracle_for(plan, rho, kernel, extra.get("axis"), extra.get("axis2"), extra.get("alpha", 0.0))
    tol = 1e-5 if prec == "fp32" else 1e-10
    got = u.double().cpu().numpy()
    err = np.max(np.abs(got - ref["u"])) / np.max(np.abs(ref["u"]))
    assert err <= tol, err
    assert abs(E.item() - ref["E"]) <= tol * ref["E_scale"], (E.item(), ref["E"])


def test_alg2_eval_equals_eval_energy_and_host_path(pkg):
    n, L = 32, 12.0
    rng = np.random.default_rng(4)
    rho = rng.standard_normal((n,) * 3)
    plan = pkg.Plan(3, n, L, "coulomb", precision="fp64", eps=1e-12, algorithm=2, device=0)
    r = torch.from_numpy(rho).to("cuda:0")
    u0 = plan.eval(r)
    u1, E1 = plan.eval_energy(r)
    uh, Eh = plan.eval_host(rho)
    uh = uh.numpy()
    torch.cuda.synchronize()
    assert torch.max(torch.abs(u0 - u1)).item() <= 1e-13 * torch.max(torch.abs(u1)).item()
    assert np.max(np.abs(uh - u1.cpu().numpy())) <= 1e-13 * np.max(np.abs(uh))
    assert abs(Eh - E1.item()) <= 1e-12 * abs(E1.item())


def test_alg2_plan_refuses_the_other_forms(pkg):
    plan = pkg.Plan(3, 32, 12.0, precision="fp32", algorithm=2, device=0)
    rho = torch.zeros((32,) * 3, device="cuda:0")
    for call in (lambda: plan.toeplitz(), lambda: plan.energy_only(rho)):
        with pytest.raises(pkg.NlintError) as ei:
            call()
        assert ei.value.code == -5


def test_alg2_at_benchmark_size_matches_analytic_and_algorithm_1(pkg):
    """256^3 over [-16, 16]^3, the 16-Gaussian mixture: FP32 Algorithm 2 against the closed form
    at sampled points (interior and box corners), and against the FP32 Algorithm 1 path in the
    interior |x| < 8 (Algorithm 1's 160x160x320 nodes do not resolve the box corners to 1e-5:
    the phase P |x| reaches 700 there; Algorithm 2's I_2 nodes only see |k| <= P2)."""
    wl = synth.CONFIGS["c4"]()
    rho_np = wl.rho()
    rho = torch.from_numpy(rho_np).to("cuda:0", torch.float32)
    p2 = pkg.Plan(3, wl.n, wl.L, "coulomb", precision="fp32", eps=1e-6, algorithm=2, device=0)
    u2, E2 = p2.eval_energy(rho)
    p1 = pkg.Plan(3, wl.n, wl.L, "coulomb", nodes=wl.nodes, precision="fp32", eps=1e-6, device=0)
    u1, E1 = p1.eval_energy(rho)
    torch.cuda.synchronize()
    a2 = u2.double().cpu().numpy()
    a1 = u1.double().cpu().numpy()
    umax = np.max(np.abs(a1))
    z, y, x = synth.grid_coords(3, wl.n, wl.L)
    inner = (x * x + y * y + z * z) < 64.0
    assert np.max(np.abs(a2 - a1)[inner]) <= 1e-5 * umax
    rng = np.random.default_rng(9)
    idx = [tuple(rng.integers(0, wl.n, 3)) for _ in range(400)] + [(0, 0, 0), (0, wl.n - 1, 5)]
    x1 = -wl.L / 2 + (wl.L / wl.n) * np.arange(wl.n)
    pts = np.array([[x1[i[2]], x1[i[1]], x1[i[0]]] for i in idx])   # arrays are (z, y, x)
    c, s, w = synth.mixture_params(np.random.default_rng(synth.SEED_MIX), 16, 3, 4.0, 0.6, 1.4,
                                   0.5, 1.0)                       # the c4 recipe
    ue = cf.coulomb3d_mixture(pts[:, 0], pts[:, 1], pts[:, 2], c, s, w)
    got = np.array([a2[i] for i in idx])
    assert np.max(np.abs(got - ue)) <= 1e-5 * umax, np.max(np.abs(got - ue)) / umax
    E_ex = cf.coulomb3d_mixture_energy(c, s, w)
    assert abs(E2.item() - E_ex) <= 1e-5 * E_ex
