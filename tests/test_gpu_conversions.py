"""The float64 <-> float32 format conversions that the mixed-precision kernels
form with integer operations on the IEEE 754 bit fields, against numpy's
IEEE 754 conversions (round to nearest, ties to even): edge cases of the
rounding and of the exponent range, then random bit patterns."""
import numpy as np
import pytest

from paper_1411_3019_gb300 import md

pytestmark = pytest.mark.gpu


def _edge_values():
    two = np.float64(2.0)
    fmax = float(np.finfo(np.float32).max)
    vals = [0.0, -0.0, 1.0, -1.0, 0.1, 1.0 / 3.0, np.pi, 250.0, -149.42, 1e-3, 1e30, -1e-30,
            fmax, -fmax,
            fmax + two ** 103,            # halfway between max and 2^128: ties to even -> inf
            fmax + two ** 103 - two ** 75,  # one float64 ulp below halfway -> max
            two ** 128, -two ** 128, 1e300, -1e300,
            two ** -126, -two ** -126,     # smallest normal
            two ** -126 * (1 - two ** -24),  # rounds up into the normal range
            two ** -127, two ** -149, two ** -150, two ** -150 * 1.5, two ** -151, 5e-324, -5e-324,
            1 + two ** -24, 1 + 3 * two ** -24, 1 + two ** -24 + two ** -52,  # ties and just above
            2 - two ** -24, 2 - two ** -25,  # carry into the exponent
            np.inf, -np.inf, np.nan]
    return np.array(vals, dtype=np.float64)


def _check(values):
    f, d = md.md_check_conversions(values)
    with np.errstate(over="ignore"):
        ref = values.astype(np.float32)
    nan = np.isnan(values)
    assert np.array_equal(np.isnan(f), nan)
    assert np.array_equal(f[~nan].view(np.uint32), ref[~nan].view(np.uint32))
    back = f.astype(np.float64)
    assert np.array_equal(np.isnan(d), nan)
    assert np.array_equal(d[~nan].view(np.uint64), back[~nan].view(np.uint64))


def test_edge_cases_round_like_ieee754():
    _check(_edge_values())


def test_random_values_across_the_float32_range():
    g = np.random.default_rng(11)
    m = g.uniform(1.0, 2.0, 400_000) * g.choice([-1.0, 1.0], 400_000)
    e = g.integers(-152, 130, 400_000)
    _check(np.ldexp(m, e))


def test_random_bit_patterns_and_exact_ties():
    g = np.random.default_rng(12)
    bits = g.integers(0, 2 ** 63, 400_000, dtype=np.uint64) | (g.integers(0, 2, 400_000, dtype=np.uint64) << 63)
    _check(bits.view(np.float64))
    # values exactly halfway between two float32 neighbours
    f = (g.uniform(1e-30, 1e30, 100_000)).astype(np.float32)
    up = np.nextafter(f, np.float32(np.inf))
    _check((f.astype(np.float64) + up.astype(np.float64)) / 2)


def test_empty_and_bad_arguments():
    f, d = md.md_check_conversions(np.zeros(0))
    assert f.size == 0 and d.size == 0
    assert md.lib().md_check_conversions(None, 5, None, None) == md.MD_ERR_INVALID_ARG
