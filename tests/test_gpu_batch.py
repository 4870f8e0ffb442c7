"""Batched evaluation (one CUDA graph over many plans) against the same plans evaluated one at
a time, and against the oracle for a few members of the mixed-size workload."""
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


def _members(precision, count=10):
    # a reduced mixed-size batch with the recipe of the 64-density workload (sizes <= 64 so that
    # the oracle stays fast)
    rng = np.random.default_rng(synth.SEED_MIX + 7)
    arng = np.random.default_rng(synth.SEED_AXIS + 7)
    out = []
    for i in range(count):
        n = int(rng.choice([24, 32, 48, 64]))
        kern = "coulomb" if i % 2 == 0 else "dipole"
        axis = synth.random_unit(arng, 3) if kern == "dipole" else None
        c, s, w = synth.mixture_params(rng, 6, 3, 3.0, 0.6, 1.4, 0.5, 1.0)
        rho = synth.mixture(3, n, 16.0, c, s, w)
        nodes = synth.default_nodes(3, n)
        out.append((n, kern, axis, nodes, rho))
    return out


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_equals_single_plans_and_replays(pkg, precision):
    members = _members(precision)
    eps = 1e-6 if precision == "fp32" else 1e-12
    dt = torch.float32 if precision == "fp32" else torch.float64
    plans = [pkg.Plan(3, n, 16.0, k, axis=a, nodes=nd, precision=precision, eps=eps, device=0)
             for n, k, a, nd, _ in members]
    rhos = [torch.from_numpy(r).to("cuda:0", dt) for *_, r in members]
    singles = []
    for p, r in zip(plans, rhos):
        u, E = p.eval_energy(r, lam=0.9)
        singles.append((u.double().cpu().numpy(), float(E.item())))
    batch = pkg.Batch(plans, branches=4)
    for rep in range(2):  # second call replays the captured graph
        us, Es = batch.eval(rhos, lam=0.9)
        torch.cuda.synchronize()
        Es = Es.cpu().numpy()
        for i, (u, E) in enumerate(singles):
            ub = us[i].double().cpu().numpy()
            tol = 1e-5 if precision == "fp32" else 1e-12
            assert np.max(np.abs(ub - u)) <= tol * np.max(np.abs(u)), (rep, i)
            assert abs(Es[i] - E) <= tol * abs(E) + 1e-14, (rep, i)
    info = batch.info()
    assert info["count"] == len(plans) and info["kernels_per_eval"] >= 9 * len(plans)
    # new contents in the same tensors: the replayed graph reads them
    for r in rhos:
        r.mul_(2.0)
    us, Es = batch.eval(rhos, lam=0.9)
    torch.cuda.synchronize()
    for i, (u, E) in enumerate(singles):
        ub = us[i].double().cpu().numpy()
        tol = 1e-5 if precision == "fp32" else 1e-12
        assert np.max(np.abs(ub - 2 * u)) <= tol * 2 * np.max(np.abs(u))
        assert abs(float(Es[i]) - 4 * E) <= tol * 4 * abs(E) + 1e-14
    batch.close()


def test_batch_members_match_oracle(pkg):
    members = _members("fp32", count=4)
    plans = [pkg.Plan(3, n, 16.0, k, axis=a, nodes=nd, precision="fp32", eps=1e-6, device=0)
             for n, k, a, nd, _ in members]
    rhos = [torch.from_numpy(r).to("cuda:0", torch.float32) for *_, r in members]
    batch = pkg.Batch(plans)
    us, Es = batch.eval(rhos, lam=1.0)
    torch.cuda.synchronize()
    for i, (n, k, a, nd, rho) in enumerate(members):
        ref = pipeline.oracle_eval(rho, 16.0, nd, k, axis=a, setting="fp32ref")
        err = np.max(np.abs(us[i].double().cpu().numpy() - ref["u"])) / np.max(np.abs(ref["u"]))
        assert err <= 1e-5, (i, err)
        assert abs(float(Es[i]) - ref["E"]) <= 1e-5 * ref["E_scale"]
    batch.close()


def test_batch_rejects_bad_arguments(pkg):
    with pytest.raises(pkg.NlintError):
        pkg.Batch([])


def test_batch_rejects_a_plan_listed_twice(pkg):
    # one plan owns one set of workspaces, so two of its evaluations cannot run side by side
    # on the graph's branches: the batch refuses the duplicate instead of corrupting both
    p = pkg.Plan(3, 24, 16.0, "coulomb", nodes=(16, 16, 32), precision="fp32", eps=1e-6, device=0)
    q = pkg.Plan(3, 32, 16.0, "coulomb", nodes=(16, 16, 32), precision="fp32", eps=1e-6, device=0)
    with pytest.raises(pkg.NlintError, match="more than once"):
        pkg.Batch([p, q, p], branches=2)
    b = pkg.Batch([p, q], branches=2)  # the same plans once each are accepted
    b.close()
    p.close()
    q.close()


def test_batch_uses_each_plans_form(pkg):
    """Plans with a precomputed Toeplitz kernel run in that form inside the batch graph, the
    others by the NUFFT path (and an Algorithm 2 plan by its own path): each member equals
    the same plan evaluated alone in its form."""
    members = _members("fp32", count=8)
    plans, rhos, singles = [], [], []
    for i, (n, k, a, nd, rho) in enumerate(members):
        alg = 2 if i == 5 else 1
        p = pkg.Plan(3, n, 16.0, k, axis=a, nodes=None if alg == 2 else nd, precision="fp32",
                     eps=1e-6, algorithm=alg, device=0)
        if i % 2 == 0:
            p.toeplitz()
        r = torch.from_numpy(rho).to("cuda:0", torch.float32)
        u, E = p.eval_toeplitz(r, lam=1.1) if i % 2 == 0 else p.eval_energy(r, lam=1.1)
        singles.append((u.double().cpu().numpy(), float(E.item())))
        plans.append(p)
        rhos.append(r)
    batch = pkg.Batch(plans, branches=3)
    us, Es = batch.eval(rhos, lam=1.1)
    torch.cuda.synchronize()
    Es = Es.cpu().numpy()
    for i, (u, E) in enumerate(singles):
        ub = us[i].double().cpu().numpy()
        assert np.max(np.abs(ub - u)) <= 1e-5 * np.max(np.abs(u)), i
        assert abs(Es[i] - E) <= 1e-5 * abs(E), i
    batch.close()


def test_batch_large_members_of_the_64_density_set_match_oracle(pkg, tmp_path):
    """The 96^3 and 128^3 members of the 64-density workload (its own seeded densities, axes
    and node counts), on autotuned plans inside a batch graph, against the oracle."""
    import bench
    members = synth.config5("fp32")
    pick = []
    for n in (96, 128):
        for kern in ("coulomb", "dipole"):
            m = next((m for m in members if m.n == n and m.kernel == kern), None)
            if m is not None:
                pick.append(m)
    assert any(m.n == 96 for m in pick) and any(m.n == 128 for m in pick)
    import os
    os.environ["NLINT_TUNE_CACHE"] = str(tmp_path / "tune.jsonl")
    try:
        prms, reps = bench.tuned_member_params(pkg, pick, "fp32", torch.device("cuda", 0))
    finally:
        del os.environ["NLINT_TUNE_CACHE"]
    plans = [pkg.Plan(3, m.n, m.L, params=q, device=0) for m, q in zip(pick, prms)]
    rhos = [torch.from_numpy(m.rho()).to("cuda:0", torch.float32) for m in pick]
    batch = pkg.Batch(plans)
    us, Es = batch.eval(rhos, lam=1.0)
    torch.cuda.synchronize()
    for i, m in enumerate(pick):
        ref = pipeline.oracle_eval(m.rho(), m.L, m.nodes, m.kernel, axis=m.axis, setting="fp32ref")
        err = np.max(np.abs(us[i].double().cpu().numpy() - ref["u"])) / np.max(np.abs(ref["u"]))
        assert err <= 1e-5, (m.n, m.kernel, err)
        assert abs(float(Es[i]) - ref["E"]) <= 1e-5 * ref["E_scale"], (m.n, m.kernel)
    batch.close()
