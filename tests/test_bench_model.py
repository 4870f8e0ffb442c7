"""The bench's algorithmic models at the 256^3 workload (FP32, w = 7; FP64, w = 13) equal the
figures the measurement documentation divides by: the whole-path bytes s (51.4 N^3 + 2 N_f),
the spreading kernel's bytes (the fine-grid ball plus the node stream) and the node kernels'
8 w^d flops per half node."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

C4 = {"precision": 0, "n": 256, "n_fine": 512, "n_nodes": 160 * 160 * 320,
      "n_half_nodes": 160 * 160 * 320 // 2, "w": 7, "d": 3}


def test_path_bytes():
    assert bench.path_bytes(C4) == pytest.approx(4 * (51.4 * 256 ** 3 + 2 * 8192000))
    assert bench.path_bytes(C4) == pytest.approx(3.515e9, rel=1e-3)
    assert bench.path_bytes(dict(C4, precision=1)) == pytest.approx(2 * bench.path_bytes(C4))


def test_spread_and_interp_bytes():
    # the half ball (pi/12) 512^3 complex floats plus two values per half node:
    # 281.1 MB + 32.8 MB = 313.9 MB per node kernel at the 256^3 workload
    ball = (3.141592653589793 / 12) * 512 ** 3 * 8
    assert ball == pytest.approx(281.1e6, rel=1e-3)
    for st in ("spread", "interp"):
        assert bench.stage_bytes(C4, st) == pytest.approx(ball + 4096000 * 8)
        assert bench.stage_bytes(C4, st) == pytest.approx(313.9e6, rel=1e-3)
    # the per-stage models add up to the whole-path model (which rounds n/2 + 1 stored planes
    # to n/2 and the per-cell coefficient to 51.4)
    stages = ("fwd_fft_z", "fwd_fft_y", "fwd_fft_x", "interp", "spread", "inv_fft_x",
              "inv_fft_y", "inv_fft_z")
    tot = sum(bench.stage_bytes(C4, st) for st in stages)
    assert tot == pytest.approx(bench.path_bytes(C4), rel=5e-3)
    # the stored records: FP32 16-byte origin/offset record, W and c for the interpolation;
    # FP64: packed origin and 3 w stencil values
    assert bench.layout_bytes(C4, "interp") == pytest.approx(ball + 4096000 * (16 + 4 + 8))
    c4_64 = dict(C4, precision=1, w=13)
    ball64 = 2 * ball
    assert bench.layout_bytes(c4_64, "spread") == pytest.approx(ball64 + 4096000 * (4 + 39 * 8 + 16))


def test_node_flops():
    assert bench.node_flops(C4) == 8 * 7 ** 3 * 4096000
    assert bench.node_flops(dict(C4, w=13)) == pytest.approx(7.2e10, rel=1e-2)


def test_job_rate_of_replicas():
    assert bench.job_rate(16777216 * 10, 4, 0.0307) == pytest.approx(4 * 16777216 * 10 / 0.0307)
