"""Stream ordering of a plan's evaluation: an Algorithm 1 plan clears its spreading grid on an
internal stream forked from the caller's stream (before the interpolation) and joined back
before the spreading.  Each result must equal a fresh plan's result for the same input, whatever
ran on the plan before, on the current stream, on another torch stream, and when the evaluation
is captured into a CUDA graph and replayed with new data.  The streaming host entry point
(copies on two plan-owned streams, overlapped with the evaluations) must give each density
what the device entry point gives it."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
TOL = 1e-6  # FP32: the same operator, only the order of the spreading's global atomics differs


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_4120_gb300 as p
    p.load_library()
    return p


def _plan(pkg):
    return pkg.Plan(3, 48, 12.0, "coulomb", precision="fp32", eps=1e-6, nodes=(24, 24, 48), device=0)


def _densities(n, count):
    rng = np.random.default_rng(77)
    out = []
    for _ in range(count):
        c, s, w = synth.mixture_params(rng, 4, 3, 2.0, 0.6, 1.2, 0.5, 1.0)
        out.append(torch.from_numpy(synth.mixture(3, n, 12.0, c, s, w)).to("cuda:0", torch.float32))
    return out


def _rel(a, b):
    return (torch.max(torch.abs(a - b)) / torch.max(torch.abs(b))).item()


def test_evaluations_with_other_densities_in_between_agree(pkg):
    ra, rb = _densities(48, 2)
    ub_fresh, Eb_fresh = _plan(pkg).eval_energy(rb)
    plan = _plan(pkg)
    for _ in range(3):
        plan.eval_energy(ra)
        ub, Eb = plan.eval_energy(rb)
    torch.cuda.synchronize()
    assert _rel(ub, ub_fresh) <= TOL
    assert abs(Eb.item() - Eb_fresh.item()) <= TOL * abs(Eb_fresh.item())


def test_type1_after_an_evaluation_matches_a_fresh_plan(pkg):
    ra, rb = _densities(48, 2)
    fresh = _plan(pkg)
    c = fresh.type2(ra)
    u_fresh = fresh.type1(c)
    plan = _plan(pkg)
    plan.eval_energy(rb)
    u = plan.type1(c)
    torch.cuda.synchronize()
    assert _rel(u, u_fresh) <= TOL


def test_evaluation_on_another_torch_stream(pkg):
    ra, rb = _densities(48, 2)
    ub_fresh = _plan(pkg).eval(rb)
    plan = _plan(pkg)
    plan.eval(ra)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        ub = plan.eval(rb, stream=st)
    torch.cuda.current_stream().wait_stream(st)
    torch.cuda.synchronize()
    assert _rel(ub, ub_fresh) <= TOL


def test_evaluation_captured_in_a_cuda_graph(pkg):
    ra, rb, rc = _densities(48, 3)
    refs = [_plan(pkg).eval_energy(r) for r in (rb, rc)]
    plan = _plan(pkg)
    rho = ra.clone()
    u = torch.empty_like(rho)
    E = torch.empty((), dtype=torch.float64, device="cuda:0")
    plan.eval_energy(rho, out=u, E_out=E)  # first use outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        plan.eval_energy(rho, out=u, E_out=E)
    for r, (u_ref, E_ref) in zip((rb, rc), refs):
        rho.copy_(r)
        g.replay()
        torch.cuda.synchronize()
        assert _rel(u, u_ref) <= TOL
        assert abs(E.item() - E_ref.item()) <= TOL * abs(E_ref.item())


@pytest.mark.parametrize("count", [1, 2, 5])
def test_streaming_host_entry_point_matches_device_evaluations(pkg, count):
    rhos = _densities(48, count)
    ref = _plan(pkg)
    refs = [ref.eval_energy(r) for r in rhos]
    plan = _plan(pkg)
    rh = [r.cpu().pin_memory() for r in rhos]
    uh = [torch.empty_like(r).pin_memory() for r in rh]
    for _ in range(2):  # the second call reuses the staging buffers and events
        us, Es = plan.eval_host_many(rh, us_host=uh)
    torch.cuda.synchronize()
    for u, E, (u_ref, E_ref) in zip(us, Es, refs):
        assert _rel(u, u_ref.cpu()) <= TOL
        assert abs(E - E_ref.item()) <= TOL * abs(E_ref.item())
    us2, none = plan.eval_host_many([r.cpu() for r in rhos], energies=False)  # pageable memory
    assert none is None
    for u, (u_ref, _) in zip(us2, refs):
        assert _rel(u, u_ref.cpu()) <= TOL


@pytest.mark.parametrize("d,prec,alg", [(2, "fp64", 1), (3, "fp64", 1), (3, "fp32", 2)])
def test_streaming_host_entry_point_other_plans(pkg, d, prec, alg):
    n, L = (64, 16.0) if d == 2 else (32, 12.0)
    plan = pkg.Plan(d, n, L, "coulomb", precision=prec, eps=1e-6 if prec == "fp32" else 1e-12,
                    algorithm=alg, device=0)
    dt = torch.float32 if prec == "fp32" else torch.float64
    rng = np.random.default_rng(5 + d)
    rh = [torch.from_numpy(rng.standard_normal((n,) * d)).to(dt).pin_memory() for _ in range(3)]
    us, Es = plan.eval_host_many(rh)
    tol = 1e-6 if prec == "fp32" else 1e-12
    for r, u, E in zip(rh, us, Es):
        u_ref, E_ref = plan.eval_energy(r.to("cuda:0"))
        torch.cuda.synchronize()
        assert _rel(u, u_ref.cpu()) <= tol
        assert abs(E - E_ref.item()) <= tol * abs(E_ref.item())


def test_streaming_host_entry_point_rejects_bad_arguments(pkg):
    plan = _plan(pkg)
    with pytest.raises(ValueError):
        plan.eval_host_many([])
    assert plan._lib.nlint_eval_host_many(plan._h, 0, None, None, 1.0, None, None) == -1
    null2 = (ctypes.c_void_p * 2)(None, None)
    assert plan._lib.nlint_eval_host_many(plan._h, 2, null2, null2, 1.0, None, None) == -1
