"""The arithmetic facts the spreading kernels' fixed-point accumulation relies on, checked on
the CPU in numpy:

* FP64 contributions are rounded to integers by adding 1.5 * 2^52 (one fused multiply-add on
  the GPU): for |v| < 2^51 the sum lies in [2^52, 2^53), where doubles are spaced by 1, so its
  bit pattern minus that of 1.5 * 2^52 is v rounded to the nearest integer (ties to even).
* FP32 3D contributions of nodes with S |c_j| <= 2^22 are rounded the same way in single
  precision: v + 1.5 * 2^23 lies in [2^23, 2^24] for |v| <= 2^22, where floats are spaced by 1
  (and 2^24 is exact), so the bit pattern's excess over that of 1.5 * 2^23 is v rounded to the
  nearest integer; beyond 2^22 that fails, which is why heavier nodes take another path.
* The scale S = 2^(E - ilogb(B) - 1) keeps S * B below 2^E, so every contribution and every
  cell sum of a subproblem stays inside the range above (E = 50) and inside int32 (E = 29,
  with the 4x headroom the kernels leave for rounding in B).
"""
import math

import numpy as np

MAGIC = 6755399441055744.0  # 1.5 * 2^52


def _magic_round(v):
    s = np.asarray(v, dtype=np.float64) + MAGIC
    return s.view(np.int64) - np.float64(MAGIC).view(np.int64)


def test_magic_number_rounding_matches_round_half_even():
    rng = np.random.default_rng(52)
    mags = 2.0 ** rng.uniform(-3, 50.9, 200000)
    v = mags * rng.choice([-1.0, 1.0], mags.size)
    assert np.array_equal(_magic_round(v), np.rint(v).astype(np.int64))


def test_magic_number_rounding_at_ties_and_edges():
    v = np.array([0.5, 1.5, 2.5, -0.5, -1.5, -2.5, 0.0, -0.0, 2.0 ** 51 - 1, -(2.0 ** 51 - 1),
                  2.0 ** 50 + 0.5, -(2.0 ** 50) - 0.5])
    assert np.array_equal(_magic_round(v), np.rint(v).astype(np.int64))


def test_scale_keeps_contributions_in_range():
    rng = np.random.default_rng(29)
    # E, the range a contribution (and, for int32, a cell sum) must stay in, and the relative
    # rounding of the computed B that the headroom below that range must absorb (B is summed in
    # the plan precision over at most 1024 terms)
    for E, limit, slack in ((29, 2 ** 31, 1e-4), (50, 2 ** 51, 1e-12)):
        for B in 10.0 ** rng.uniform(-30, 30, 2000):
            ex = E - math.frexp(B)[1]  # frexp exponent = ilogb(B) + 1
            S = math.ldexp(1.0, ex)
            assert S * B <= 2.0 ** E
            assert S * B * (1 + slack) < limit


MAGIC32 = np.float32(12582912.0)  # 1.5 * 2^23


def _magic_round32(v):
    s = np.asarray(v, dtype=np.float32) + MAGIC32  # one rounding of the float sum
    return s.view(np.int32).astype(np.int64) - int(MAGIC32.view(np.int32))


def test_single_precision_magic_rounding_within_2_22():
    rng = np.random.default_rng(23)
    mags = (2.0 ** rng.uniform(-3, 22, 200000)).astype(np.float32)
    v = mags * rng.choice(np.array([-1.0, 1.0], dtype=np.float32), mags.size)
    v = v[np.abs(v) <= 2.0 ** 22]
    assert np.array_equal(_magic_round32(v), np.rint(v.astype(np.float64)).astype(np.int64))
    edges = np.array([0.5, 1.5, 2.5, -0.5, -1.5, -2.5, 0.0, 2.0 ** 22, -(2.0 ** 22),
                      2.0 ** 22 - 0.5, -(2.0 ** 22) + 0.5, 2.0 ** 21 + 0.5], dtype=np.float32)
    assert np.array_equal(_magic_round32(edges), np.rint(edges.astype(np.float64)).astype(np.int64))


def test_single_precision_magic_rounding_fails_beyond_2_22():
    # the reason for the range check: past 2^22 the sum leaves [2^23, 2^24] and the bit
    # pattern no longer counts units
    v = np.array([2.0 ** 22 + 2.0, 2.0 ** 23, -(2.0 ** 22) - 2.0], dtype=np.float32)
    assert not np.array_equal(_magic_round32(v), np.rint(v.astype(np.float64)).astype(np.int64))
