"""Every FFT pass schedule (nlint_params.fft_sched: the two-stage radix schedule of the column,
row, fold and packed real-data passes, FP32) computes the same operator: each
schedule mask agrees with the default one to FP32 rounding and with the oracle (eqs. 3.2 and
3.7 by Section 2's NUFFT at its FP32 reference setting) to the FP32 tolerance, on grids whose
fine lines have two schedules (2^a points) and on grids whose lines have one (3 * 2^a), for
Algorithm 1, the Toeplitz form and Algorithm 2, in 2D and 3D.  FP64 plans ignore the mask."""
import numpy as np
import pytest

import synth
from oracle import pipeline

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_4120_gb300 as p
    p.load_library()
    return p


def _rho(d, n, L, seed):
    rng = np.random.default_rng(seed)
    cen, wid, wts = synth.mixture_params(rng, 6, d, L / 6, 0.6, 1.4, 0.5, 1.0)
    return synth.mixture(d, n, L, cen, wid, wts)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# (d, n, L, kernel, nodes): fine grids of 128 (2^a) and 96 (3 * 2^a) points in 3D, 256 in 2D
CASES = [(3, 64, 16.0, "dipole", (48, 48, 96)), (3, 48, 16.0, "coulomb", (36, 36, 72)),
         (2, 128, 16.0, "coulomb", (64, 128))]


@pytest.mark.parametrize("case", CASES, ids=["3d-128", "3d-96", "2d-256"])
def test_every_schedule_mask_gives_the_same_potential(pkg, case):
    d, n, L, kern, nodes = case
    axis = (0.3, -0.5, 0.8) if kern == "dipole" else None
    rho = _rho(d, n, L, 11 + d + n)
    ref = pipeline.oracle_eval(rho, L, nodes, kern, axis=axis, setting="fp32ref", lam=1.0)
    r = torch.from_numpy(rho).to("cuda:0", torch.float32)
    base = None
    for mask in (0, 1, 2, 4, 8, 15):
        plan = pkg.Plan(d, n, L, kern, axis=axis, nodes=nodes, precision="fp32", eps=1e-6,
                        fft_sched=mask, device=0)
        assert plan.info["fft_sched"] == mask
        u, E = plan.eval_energy(r, lam=1.0)
        u = u.double().cpu().numpy()
        E = float(E.item())
        plan.close()
        assert _rel(u, ref["u"]) <= 1e-5, (mask, _rel(u, ref["u"]))
        assert abs(E - ref["E"]) <= 1e-5 * ref["E_scale"]
        if base is None:
            base = u
        else:  # the same operator: only the FP32 rounding of the transforms differs
            assert _rel(u, base) <= 2e-6, (mask, _rel(u, base))


def test_schedules_in_the_toeplitz_form_and_algorithm_2(pkg):
    n, L = 64, 16.0
    rho = _rho(3, n, L, 5)
    r = torch.from_numpy(rho).to("cuda:0", torch.float32)
    out = {}
    for mask in (0, 15):
        p1 = pkg.Plan(3, n, L, "coulomb", precision="fp32", eps=1e-6, fft_sched=mask, device=0)
        p1.toeplitz()
        ut, _ = p1.eval_toeplitz(r, lam=1.0)
        un, _ = p1.eval_energy(r, lam=1.0)
        p2 = pkg.Plan(3, n, L, "coulomb", precision="fp32", eps=1e-6, algorithm=2, fft_sched=mask,
                      device=0)
        u2, _ = p2.eval_energy(r, lam=1.0)
        out[mask] = [x.double().cpu().numpy() for x in (ut, un, u2)]
        p1.close()
        p2.close()
    for a, b in zip(out[0], out[15]):
        assert _rel(b, a) <= 2e-6
    assert _rel(out[15][0], out[15][1]) <= 1e-5  # Toeplitz vs NUFFT form of one operator


def test_fp64_plans_ignore_the_mask(pkg):
    p = pkg.Plan(3, 32, 12.0, "coulomb", precision="fp64", eps=1e-12, fft_sched=15, device=0)
    assert p.info["fft_sched"] == 0
    p.close()


def test_staged_and_register_loads_of_the_real_data_passes_agree(pkg):
    # the first z pass stages its input by 16-byte copies when the density is 16-byte aligned;
    # a density 4 bytes into a buffer takes the register loads instead: the same transform
    n, L = 64, 16.0
    rho = _rho(3, n, L, 9).astype(np.float32)
    plan = pkg.Plan(3, n, L, "coulomb", precision="fp32", eps=1e-6, device=0)
    aligned = torch.from_numpy(rho).to("cuda:0")
    assert aligned.data_ptr() % 16 == 0
    buf = torch.zeros(rho.size + 4, dtype=torch.float32, device="cuda:0")
    shifted = buf[1:1 + rho.size].view(rho.shape)
    shifted.copy_(aligned)
    assert shifted.data_ptr() % 16 == 4
    ua, Ea = plan.eval_energy(aligned, lam=1.0)
    us, Es = plan.eval_energy(shifted, lam=1.0)
    ua, us = ua.double().cpu().numpy(), us.double().cpu().numpy()
    plan.close()
    assert _rel(us, ua) <= 2e-6
    assert abs(float(Es.item()) - float(Ea.item())) <= 2e-6 * abs(float(Ea.item()))
