"""CPU check of the per-product error model the tensor-core tests use
(test_gpu_tc.py): a TF32 input keeps 10 stored mantissa bits, so
|x - tf32(x)| <= 2^-10 |x| whether the conversion truncates or rounds; the
split form x = x_hi + x_lo (x_hi = x with its 13 low mantissa bits cleared)
forms x_hi y_hi + x_hi tf32(y_lo) + tf32(x_lo) y_hi, whose error is at most
3 * 2^-20 |x y|. The products are formed exactly in float64 here, so only the
input rounding is measured."""
import numpy as np
import pytest


def _trunc(x):
    """tf32 by truncation: clear the 13 low mantissa bits of each float32."""
    return (np.asarray(x, np.float32).view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)


def _round(x):
    """tf32 by round-to-nearest-even on the 13 dropped bits (finite inputs)."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 13) & 1
    u = (u + 0xFFF + lsb) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32)


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(n) * np.exp2(rng.integers(-20, 20, n))
    return x.astype(np.float32)


@pytest.mark.parametrize("conv", [_trunc, _round])
def test_tf32_product_error(conv):
    x, y = _inputs(200000, 1), _inputs(200000, 2)
    exact = x.astype(np.float64) * y.astype(np.float64)
    got = conv(x).astype(np.float64) * conv(y).astype(np.float64)
    rel = np.abs(got - exact) / np.abs(exact)
    assert np.max(rel) <= 2 * 2.0 ** -10 + 2.0 ** -20
    assert np.max(rel) > 2.0 ** -12   # the bound is not vacuous: TF32 is this coarse


@pytest.mark.parametrize("conv", [_trunc, _round])
def test_split_tf32_product_error(conv):
    x, y = _inputs(200000, 3), _inputs(200000, 4)
    xh, yh = _trunc(x), _trunc(y)            # exactly representable in TF32
    xl = (x.astype(np.float64) - xh).astype(np.float32)   # exact in float32
    yl = (y.astype(np.float64) - yh).astype(np.float32)
    assert np.array_equal(xh.astype(np.float64) + xl, x.astype(np.float64))
    assert np.all(np.abs(xl) <= 2.0 ** -10 * np.abs(x))
    exact = x.astype(np.float64) * y.astype(np.float64)
    got = (xh.astype(np.float64) * yh + xh.astype(np.float64) * conv(yl)
           + conv(xl).astype(np.float64) * yh)
    rel = np.abs(got - exact) / np.abs(exact)
    assert np.max(rel) <= 3 * 2.0 ** -20
    # and a dropped cross term would break it: x_hi y_hi alone is TF32-coarse
    rel_hi = np.abs(xh.astype(np.float64) * yh - exact) / np.abs(exact)
    assert np.max(rel_hi) > 3 * 2.0 ** -20
