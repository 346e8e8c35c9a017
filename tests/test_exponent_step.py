"""The FP64 monotonised-central slope (grmhd.cuh, mc_slope_d) halves |q_{i+1} - q_{i-1}|
and doubles min(|dl|, |dr|) on their bit patterns instead of with FP64 products:
an exponent step, or for the subnormal range a shift (rounded to even when
halving). These are the same integer formulas, checked bit for bit against
IEEE products over random doubles spanning every binade, the subnormals and the
binade boundaries, so the slope is unchanged to the last bit."""
import numpy as np

MAG = np.int64(0x7FFFFFFFFFFFFFFF)


def _bits(x):
    return np.asarray(x, dtype=np.float64).view(np.int64)


def _half(b):  # |x|/2 with the sign of x, from the bits b of x
    mag = b & MAG
    h = np.where(mag >= (1 << 53), mag - (1 << 52), (mag >> 1) + (mag & (mag >> 1) & 1))
    return h | (b & ~MAG)


def _double(mag):  # 2|x| from the magnitude bits of a finite x below 2^1023
    return np.where(mag < (1 << 52), mag << 1, mag + (1 << 52))


def _samples():
    rng = np.random.default_rng(1912)
    n = 400_000
    x = np.ldexp(rng.random(n) + 0.5, rng.integers(-1080, 1020, n)) * rng.choice([-1.0, 1.0], n)
    edge = [0.0, -0.0, 5e-324, -5e-324, 1e-323, 2.2250738585072009e-308, 2.2250738585072014e-308,
            4.450147717014402e-308, 4.4501477170144023e-308, 1.0, 0.75, -3.0]
    return np.concatenate([x, edge])


def test_halving_matches_the_product():
    x = _samples()
    assert np.array_equal(_half(_bits(x)), _bits(0.5 * x))
    assert (np.abs(x) < 4.5e-308).sum() > 1000  # the subnormal-result range is exercised


def test_doubling_matches_the_product():
    x = np.abs(_samples())
    x = x[x < 8.9e307]
    assert np.array_equal(_double(_bits(x)), _bits(2.0 * x))
