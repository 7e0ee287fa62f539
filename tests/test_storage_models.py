"""The oracle's models of reduced map storage (host): the FP16 scale puts a
map's largest magnitude in [2^14, 2^15), inside half precision's normal range
below its largest finite value, and the FP16 rounding keeps 11 significant
bits (relative error at most 2^-11) and leaves stored values unchanged."""
import math

import numpy as np
import pytest

from oracle.coefficients import f16_scale, to_f16


@pytest.mark.parametrize("mx", [3.0, 2.5e9, 4.2e-9, 1.0, 65504.0, 1e-30])
def test_scale_puts_the_largest_value_in_range(mx):
    vals = np.array([mx, -0.5 * mx, 0.1 * mx, 0.0])
    s = f16_scale(vals)
    assert math.log2(s) == int(math.log2(s))                  # a power of two
    assert 2.0 ** 14 <= mx / s < 2.0 ** 15
    assert np.isfinite(to_f16(vals, s)).all()


def test_rounding_error_and_idempotence():
    rng = np.random.default_rng(0)
    v = rng.uniform(1e3, 3e3, 1000) * rng.choice([-1, 1], 1000)
    s = f16_scale(v)
    r = to_f16(v, s)
    assert np.max(np.abs(r - v) / np.abs(v)) <= 2.0 ** -11
    np.testing.assert_array_equal(to_f16(r, s), r)
    # a plain half rounding (no scale) of values in range agrees
    np.testing.assert_array_equal(to_f16(v, 1.0), v.astype(np.float16).astype(np.float64))


def test_empty_and_zero_maps_take_unit_scale():
    assert f16_scale(np.zeros(5)) == 1.0
    assert f16_scale(np.zeros(0)) == 1.0
