"""Degenerate inputs on the GPU path: a zero density (u and E exactly zero), a density at one grid
point (the operator's kernel itself, at a corner of the box and inside it) against the direct
sums of the oracle, and a NaN in the density, which must reach every u and E as NaN (no fixed
point accumulation may turn it into a finite value), for Algorithms 1 and 2."""
import numpy as np
import pytest

from oracle import pipeline

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


@pytest.mark.parametrize("prec,alg", [("fp32", 1), ("fp64", 1), ("fp32", 2)])
def test_zero_density_gives_exact_zeros(pkg, prec, alg):
    n = 48
    plan = pkg.Plan(3, n, 12.0, "dipole", axis=AX, precision=prec,
                    eps=1e-6 if prec == "fp32" else 1e-12, algorithm=alg, device=0)
    rho = torch.zeros((n,) * 3, dtype=plan.dtype, device="cuda:0")
    u, E = plan.eval_energy(rho)
    torch.cuda.synchronize()
    assert torch.count_nonzero(u).item() == 0 and E.item() == 0.0


@pytest.mark.parametrize("d,where", [(3, "corner"), (3, "inside"), (2, "corner"), (2, "inside")])
def test_single_point_density_matches_direct_sums(pkg, d, where):
    n, L = 16, 8.0
    nodes = (12, 12, 24) if d == 3 else (16, 32)
    rho = np.zeros((n,) * d)
    rho[(0,) * d if where == "corner" else (5, 11, 7)[:d]] = 1.0
    kern = dict(kernel="dipole", axis=AX) if d == 3 else dict(kernel="coulomb")
    plan = pkg.Plan(d, n, L, precision="fp64", eps=1e-12, nodes=nodes, device=0, **kern)
    u, E = plan.eval_energy(torch.from_numpy(rho).to("cuda:0"))
    torch.cuda.synchronize()
    ref = pipeline.oracle_eval(rho, L, nodes, method="direct", **kern)
    got = u.cpu().numpy()
    assert np.max(np.abs(got - ref["u"])) <= 1e-10 * np.max(np.abs(ref["u"]))
    assert abs(E.item() - ref["E"]) <= 1e-10 * ref["E_scale"]


@pytest.mark.parametrize("prec,alg", [("fp32", 1), ("fp64", 1), ("fp32", 2)])
def test_nan_in_the_density_reaches_every_output(pkg, prec, alg):
    n = 48
    plan = pkg.Plan(3, n, 12.0, "coulomb", precision=prec, eps=1e-6 if prec == "fp32" else 1e-12,
                    algorithm=alg, device=0)
    rho = torch.rand((n,) * 3, dtype=plan.dtype, device="cuda:0",
                     generator=torch.Generator(device="cuda:0").manual_seed(3))
    rho[17, 3, 40] = float("nan")
    u, E = plan.eval_energy(rho)
    torch.cuda.synchronize()
    assert torch.isnan(u).all().item() and np.isnan(E.item())
