"""nlint_energy_noalloc: the energy entry point for callers that cannot allocate device memory.

It is checked through the C-ABI against the oracle's energy (the trapezoidal sum of the
energy Remark after Algorithm 2, summed exactly with math.fsum) and against the plan-based
nlint_energy on the same arrays, on calls in a row with different data: a large grid that
fills thousands of partial sums, then a smaller one that must not see the larger call's
partial sums, which stay in the library's scratch array.  This file is named to be collected
last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_4120_gb300 as pkg
    return pkg, pkg.load_library()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_energy_matches_plan_energy_twice(lib, prec):
    pkg, L_ = lib
    d, n, L, lam = 3, 48, 12.0, 0.8
    plan = pkg.Plan(d, n, L, "coulomb", nodes=(8, 8, 16), precision=prec,
                    eps=1e-6 if prec == "fp32" else 1e-12, device=0)
    dt = torch.float32 if prec == "fp32" else torch.float64
    code = pkg.NLINT_FP32 if prec == "fp32" else pkg.NLINT_FP64
    rng = np.random.default_rng(17)
    E_dev = torch.zeros((), dtype=torch.float64, device="cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        rho = torch.from_numpy(rng.standard_normal((n,) * d) + call).to("cuda:0", dt)
        u = torch.from_numpy(rng.standard_normal((n,) * d) * (1 + call)).to("cuda:0", dt)
        ref = plan.energy(rho, u, lam=lam)
        rc = L_.nlint_energy_noalloc(d, n, L, code, ctypes.c_void_p(rho.data_ptr()),
                                     ctypes.c_void_p(u.data_ptr()), lam,
                                     ctypes.c_void_p(E_dev.data_ptr()), ctypes.c_void_p(stream))
        assert rc == 0, L_.nlint_last_error()
        torch.cuda.synchronize()
        got = float(E_dev.item())
        scale = 0.5 * lam * (L / n) ** d * float((rho.double() * u.double()).abs().sum())
        assert abs(got - ref) <= 1e-13 * scale, (call, got, ref)
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_energy_matches_oracle_large_then_small(lib, prec):
    # 256^3 (4096 partial sums, folded by the final kernel) followed by 48^3 (27 partial
    # sums): the second call must use only its own partials, not the first call's leftovers
    from oracle import pipeline
    pkg, L_ = lib
    dt = torch.float32 if prec == "fp32" else torch.float64
    npdt = np.float32 if prec == "fp32" else np.float64
    code = pkg.NLINT_FP32 if prec == "fp32" else pkg.NLINT_FP64
    rng = np.random.default_rng(1311)
    E_dev = torch.zeros((), dtype=torch.float64, device="cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    for d, n, L, lam in ((3, 256, 32.0, 1.0), (3, 48, 12.0, 0.8), (2, 40, 9.0, 1.3)):
        rho_h = (rng.standard_normal((n,) * d) + 0.25).astype(npdt)
        u_h = rng.standard_normal((n,) * d).astype(npdt)
        rho = torch.from_numpy(rho_h).to("cuda:0")
        u = torch.from_numpy(u_h).to("cuda:0")
        rc = L_.nlint_energy_noalloc(d, n, L, code, ctypes.c_void_p(rho.data_ptr()),
                                     ctypes.c_void_p(u.data_ptr()), lam,
                                     ctypes.c_void_p(E_dev.data_ptr()), ctypes.c_void_p(stream))
        assert rc == 0, L_.nlint_last_error()
        torch.cuda.synchronize()
        got = float(E_dev.item())
        ref = pipeline.energy(u_h, rho_h, L, lam)
        scale = 0.5 * lam * (L / n) ** d * float(np.abs(rho_h.astype(np.float64) * u_h).sum())
        assert abs(got - ref) <= 1e-13 * scale, (n, got, ref)


def test_noalloc_energy_rejects_oversized_grids(lib):
    pkg, L_ = lib
    E_dev = torch.zeros((), dtype=torch.float64, device="cuda:0")
    x = torch.zeros(8, device="cuda:0")
    rc = L_.nlint_energy_noalloc(3, 1024, 1.0, pkg.NLINT_FP32, ctypes.c_void_p(x.data_ptr()),
                                 ctypes.c_void_p(x.data_ptr()), 1.0,
                                 ctypes.c_void_p(E_dev.data_ptr()), None)
    assert rc == -1
    assert b"too large" in L_.nlint_last_error()
