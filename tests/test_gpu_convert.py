"""The mixed path's FP64 <-> FP32 conversions, which run on the integer pipe (on GB300 the
hardware conversions issue to the FP64 pipe, the bound of the update kernel), against
numpy's IEEE casts bit for bit: FP64 -> FP32 rounds to nearest, ties to even, over random bit
patterns, random magnitudes across the float range and exact ties; FP32 -> FP64 widens
exactly.  The one documented departure: results below the smallest normal float (and
subnormal floats widened) become signed zeros."""
import numpy as np
import pytest

from paper_1502_02935_gb300 import mhd

pytestmark = pytest.mark.gpu


def _doubles(rng, n):
    bits = rng.integers(0, 2 ** 63, n, dtype=np.int64).view(np.uint64) | (rng.integers(0, 2, n).astype(np.uint64) << 63)
    mags = rng.uniform(-1, 1, n) * np.exp2(rng.integers(-140, 140, n).astype(np.float64))
    # exact ties between two floats, and values just beside them
    base = rng.uniform(-1, 1, n).astype(np.float32).astype(np.float64)
    ulp = np.abs(np.spacing(base.astype(np.float32)).astype(np.float64))
    ties = base + 0.5 * ulp * rng.choice([-1.0, 1.0, 1.0 + 2.0 ** -30, 1.0 - 2.0 ** -30], n)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 3.4028235677973366e38, 3.4028235677973367e38,
                        1.1754943508222875e-38, 1.1754942e-38, 5e-324, -1e300, 1e-300])
    return np.concatenate([bits.view(np.float64), mags, ties, special])


def test_fp64_to_fp32_matches_ieee_round_to_nearest_even():
    rng = np.random.default_rng(41)
    d = _doubles(rng, 1 << 20)
    got, _ = mhd.convert_fp(d, np.zeros(d.size, np.float32))
    with np.errstate(over="ignore", under="ignore", invalid="ignore"):
        want = d.astype(np.float32)
    normal = np.isfinite(want) & (np.abs(want) >= np.finfo(np.float32).tiny)
    assert np.array_equal(got[normal].view(np.uint32), want[normal].view(np.uint32))
    inf = np.isinf(want) & ~np.isnan(d)
    assert np.array_equal(got[inf], want[inf])
    tiny = ~normal & ~np.isinf(want) & ~np.isnan(d)
    assert np.all(got[tiny] == 0.0) and np.array_equal(np.signbit(got[tiny]), np.signbit(d[tiny]))
    assert np.all(np.isnan(got[np.isnan(d)]))
    assert normal.sum() > 2_000_000 // 2


def test_fp32_to_fp64_is_exact():
    rng = np.random.default_rng(42)
    f = np.concatenate([rng.integers(0, 2 ** 32, 1 << 21, dtype=np.uint64).astype(np.uint32).view(np.float32),
                        np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-40], np.float32)])
    _, got = mhd.convert_fp(np.zeros(f.size), f)
    with np.errstate(invalid="ignore"):  # the random bit patterns include signalling NaNs
        want = f.astype(np.float64)
    normal = np.isfinite(f) & (np.abs(f) >= np.finfo(np.float32).tiny)
    assert np.array_equal(got[normal].view(np.uint64), want[normal].view(np.uint64))
    assert np.array_equal(got[np.isinf(f)], want[np.isinf(f)])
    sub = np.isfinite(f) & ~normal
    assert np.all(got[sub] == 0.0) and np.array_equal(np.signbit(got[sub]), np.signbit(f[sub]))
    assert np.all(np.isnan(got[np.isnan(f)]))
