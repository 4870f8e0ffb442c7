"""FP32 node kernels for every bin shape and for widths that take each lane layout.

The FP32 kernels evaluate the spreading function from each node's fractional offsets.  The 3D
interpolation gives each node a lane (half-groups of bank-disjoint origins; tiles staged by
TMA where they do not wrap, by plain loads where they do); the spreading, and the 2D kernels,
exchange the values by warp shuffles, with a lane layout that depends on the width (32 lanes
per node with one or two values per lane: w = 7, 11; 16 lanes per node, two nodes per warp,
with one, two or three values per lane: w = 4, 6, 12).  After each evaluation the plan's status
word must show that no bounded device-side wait ran out.  Each case is checked

  * against the FP64 oracle (eqs. 3.2 and 3.7 by Section 2's NUFFT at its parity setting), to
    the accuracy the width allows (the exponential-of-semicircle error at sigma = 2, about
    1e-5 relative at w = 5 and 1e-6 at w = 7, with FP32 rounding beside it), and
  * against the FP64 GPU path with the same width and nodes: both approximate the operator
    with the same stencil, so they differ only by FP32 rounding (<= 1e-5 relative).
"""
import numpy as np
import pytest

import synth
from oracle import pipeline

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# oracle tolerance by width (the width's own NUFFT error with a margin, never below 1e-5)
TOL_W = {4: 3e-3, 6: 1e-4, 7: 1e-5, 11: 1e-5, 12: 1e-5}


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_4120_gb300 as p
    p.load_library()
    return p


def _case(d):
    if d == 3:
        n, L, nodes = 32, 12.0, (20, 16, 36)
    else:
        n, L, nodes = 96, 16.0, (40, 72)
    rng = np.random.default_rng(4120 + d)
    cen, wid, wts = synth.mixture_params(rng, 5, d, L / 6, 0.6, 1.4, 0.5, 1.0)
    rho = synth.mixture(d, n, L, cen, wid, wts) + 0.05 * rng.standard_normal((n,) * d)
    axis = synth.random_unit(rng, 3)
    return n, L, nodes, rho, axis


@pytest.fixture(scope="module")
def refs():
    out = {}
    for d in (2, 3):
        n, L, nodes, rho, axis = _case(d)
        kern = "dipole" if d == 3 else "coulomb"
        out[d] = pipeline.oracle_eval(rho, L, nodes, kern, axis=axis if d == 3 else None,
                                      setting="parity", lam=0.9)
    return out


def _eval(pkg, d, prec, w, bin_shape):
    n, L, nodes, rho, axis = _case(d)
    kern = "dipole" if d == 3 else "coulomb"
    plan = pkg.Plan(d, n, L, kern, axis=axis if d == 3 else None, nodes=nodes, precision=prec,
                    w=w, bin_shape=bin_shape, device=0)
    assert plan.info["bin_shape"] == bin_shape and plan.info["w"] == w
    dt = torch.float32 if prec == "fp32" else torch.float64
    u, E = plan.eval_energy(torch.from_numpy(rho).to("cuda:0", dt), lam=0.9)
    torch.cuda.synchronize()
    res = u.double().cpu().numpy(), float(E.item())
    plan.check()  # no bounded device-side wait (the interpolation's TMA tile load) ran out
    plan.close()
    return res


@pytest.mark.parametrize("bin_shape", [1, 3, 4])
@pytest.mark.parametrize("w", [4, 6, 7, 11, 12])
def test_fp32_node_kernels_each_shape_and_width(pkg, refs, bin_shape, w):
    ref = refs[3]
    u, E = _eval(pkg, 3, "fp32", w, bin_shape)
    err = np.max(np.abs(u - ref["u"])) / np.max(np.abs(ref["u"]))
    eerr = abs(E - ref["E"]) / ref["E_scale"]
    assert err <= TOL_W[w] and eerr <= TOL_W[w], (err, eerr)
    u64, E64 = _eval(pkg, 3, "fp64", w, 1 if w < 10 else 2)
    assert np.max(np.abs(u - u64)) <= 1e-5 * np.max(np.abs(u64))
    assert abs(E - E64) <= 1e-5 * ref["E_scale"]


@pytest.mark.parametrize("w", [4, 6, 7])
def test_fp32_node_kernels_2d(pkg, refs, w):
    ref = refs[2]
    u, E = _eval(pkg, 2, "fp32", w, 1)
    err = np.max(np.abs(u - ref["u"])) / np.max(np.abs(ref["u"]))
    assert err <= TOL_W[w], err
    assert abs(E - ref["E"]) / ref["E_scale"] <= TOL_W[w]
    u64, _ = _eval(pkg, 2, "fp64", w, 1)
    assert np.max(np.abs(u - u64)) <= 1e-5 * np.max(np.abs(u64))


def test_bin_shape_validation(pkg):
    # shapes outside the compiled set are refused; an automatic choice always builds
    with pytest.raises(pkg.NlintError):
        pkg.Plan(3, 32, 12.0, "coulomb", nodes=(8, 8, 16), precision="fp32", bin_shape=2, device=0)
    with pytest.raises(pkg.NlintError):
        pkg.Plan(3, 32, 12.0, "coulomb", nodes=(8, 8, 16), precision="fp64", bin_shape=3, device=0)
    with pytest.raises(pkg.NlintError):  # 31^3 tile of 8-byte cells: beyond shared memory
        pkg.Plan(3, 32, 12.0, "coulomb", nodes=(8, 8, 16), precision="fp32", w=16, bin_shape=4,
                 device=0)
    p = pkg.Plan(3, 32, 12.0, "coulomb", nodes=(8, 8, 16), precision="fp32", w=16, device=0)
    assert p.info["bin_shape"] in (1, 3)
    p.close()
