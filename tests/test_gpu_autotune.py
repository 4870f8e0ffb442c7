"""The autotuner picks the faster of the smallest stencil width that meets a tolerance (measured
against an FP64 plan) and the next one, the fastest bin shape and subproblem size, caches the
choice, and the tuned plan meets the tolerance against the oracle; the batch tuner keeps the
faster of two decompositions of a whole batch."""
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


def test_autotune_meets_tolerance_and_caches(pkg, tmp_path):
    n, L, nodes = 64, 16.0, (48, 48, 96)
    axis = (0.3, -0.5, 0.8)
    prm = pkg.make_params(3, n, L, "dipole", axis=axis, nodes=nodes, precision="fp32", device=0)
    cache = str(tmp_path / "tune.jsonl")
    tuned, rep = pkg.autotune(prm, 1e-5, cache)
    assert rep["from_cache"] == 0 and 2 <= rep["w"] <= 16 and rep["err"] <= 0.5e-5
    assert rep["max_sub"] in (256, 512, 1024, 2048)
    assert rep["bin_shape"] in (1, 3, 4)  # the FP32 3D shapes
    assert tuned.w == rep["w"] and tuned.max_sub == rep["max_sub"]
    assert tuned.bin_shape == rep["bin_shape"]
    # the FFT pass schedules: a mask of the four pass classes, carried into the tuned parameters
    assert 0 <= rep["fft_sched"] <= 15 and tuned.fft_sched == rep["fft_sched"]
    # the other width timed, if any, is a neighbour that also meets the tolerance
    assert rep["w_alt"] == 0 or (abs(rep["w_alt"] - rep["w"]) == 1 and rep["err_alt"] <= 0.5e-5)
    # a tighter tolerance: the chosen width (the smallest qualifying one or the next, whichever
    # is faster) meets the tighter bound, and is at least the loose bound's smallest width
    _, rep2 = pkg.autotune(prm, 3e-6, cache)
    assert rep2["w"] >= rep["w"] - 1 and rep2["err"] <= 1.5e-6
    # beyond FP32 rounding: no width qualifies, and the tuner says so
    with pytest.raises(pkg.NlintError):
        pkg.autotune(prm, 1e-8, cache)
    # cache hit
    tuned3, rep3 = pkg.autotune(prm, 1e-5, cache)
    assert rep3["from_cache"] == 1 and tuned3.w == tuned.w and tuned3.max_sub == tuned.max_sub
    assert tuned3.bin_shape == tuned.bin_shape
    # the tuned plan against the oracle on a benchmark-like density
    rng = np.random.default_rng(5)
    cen, wid, wts = synth.mixture_params(rng, 8, 3, 3.0, 0.6, 1.4, 0.5, 1.0)
    rho = synth.mixture(3, n, L, cen, wid, wts)
    plan = pkg.Plan(3, n, L, params=tuned, device=0)
    assert plan.info["bin_shape"] == tuned.bin_shape
    u, E = plan.eval_energy(torch.from_numpy(rho).to("cuda:0", torch.float32))
    torch.cuda.synchronize()
    ref = pipeline.oracle_eval(rho, L, nodes, "dipole", axis=axis, setting="fp32ref")
    err = np.max(np.abs(u.double().cpu().numpy() - ref["u"])) / np.max(np.abs(ref["u"]))
    assert err <= 1e-5, err


def test_autotune_fp64_picks_an_fp64_shape(pkg, tmp_path):
    prm = pkg.make_params(3, 24, 12.0, "coulomb", nodes=(16, 16, 32), precision="fp64", device=0)
    tuned, rep = pkg.autotune(prm, 1e-10, str(tmp_path / "t64.jsonl"))
    assert rep["bin_shape"] in (1, 2) and tuned.bin_shape == rep["bin_shape"]


def test_autotune_batch_keeps_the_faster_decomposition(pkg, tmp_path):
    # six members of the 64-density workload: three classes (32^3 and 48^3 Coulomb, 32^3 dipoles
    # with two different axes: one class)
    members = synth.config5("fp32")
    pick = []
    for n, kern in ((32, "coulomb"), (48, "coulomb"), (32, "dipole")):
        pick += [m for m in members if m.n == n and m.kernel == kern][:2]
    assert len(pick) == 6
    prm = [pkg.make_params(3, m.n, m.L, m.kernel, axis=m.axis, nodes=m.nodes, precision="fp32",
                           device=0) for m in pick]
    out, reps, brep = pkg.autotune_batch(prm, 1e-5, str(tmp_path / "tune.jsonl"))
    assert brep["classes"] == 3 and brep["choice"] in (0, 1, 2)
    timed = [t for t in brep["ms"] if t > 0]
    assert brep["ms"][0] > 0 and brep["ms"][1] > 0
    assert brep["ms"][brep["choice"]] == min(timed)  # the fastest set is kept
    for m, q, r in zip(pick, out, reps):
        assert q.n == m.n and q.w == r["w"] and 2 <= q.w <= 16 and r["err"] <= 0.5e-5
        assert r["w_alt"] == 0 or (abs(r["w_alt"] - r["w"]) == 1 and r["err_alt"] <= 0.5e-5)
        assert (q.bin_shape, q.max_sub) == ((0, 0) if brep["choice"] else (r["bin_shape"], r["max_sub"]))
        assert tuple(q.axis) == tuple(m.axis) if m.axis is not None else True
    # members of one class share their width; the tuned plans evaluate within the tolerance
    assert out[0].w == out[1].w and out[4].w == out[5].w
    for m, q in zip(pick[::2], out[::2]):
        plan = pkg.Plan(3, m.n, m.L, params=q, device=0)
        u, E = plan.eval_energy(torch.from_numpy(m.rho()).to("cuda:0", torch.float32), lam=1.0)
        ref = pipeline.oracle_eval(m.rho(), m.L, m.nodes, m.kernel, axis=m.axis, setting="fp32ref")
        err = np.max(np.abs(u.double().cpu().numpy() - ref["u"])) / np.max(np.abs(ref["u"]))
        assert err <= 1e-5, (m.n, m.kernel, err)
        plan.close()
