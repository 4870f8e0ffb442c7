"""The autotuner picks the smallest stencil width that meets a tolerance (measured against an
FP64 plan), the fastest bin shape and subproblem size, caches the choice, and the tuned plan
meets the tolerance against the oracle."""
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
    # a tighter tolerance never picks a narrower stencil
    _, rep2 = pkg.autotune(prm, 3e-6, cache)
    assert rep2["w"] >= rep["w"] and rep2["err"] <= 1.5e-6
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
