"""The FP32 form's format changes on the GPU (rpba_check_formats), pinned to
IEEE-754 bit patterns computed by numpy: a double split into a 24-bit
truncated hi word and a rounded lo word, their FP64 sum, and the widening
of floats to doubles built from integer operations."""

import numpy as np
import pytest

from paper_1910_08138_gb300 import rpba

pytestmark = pytest.mark.gpu


def _truncate24(x):
    """x with the low 29 of its 52 fraction bits cleared (24 significant bits)."""
    u = x.view(np.uint64) & ~np.uint64((1 << 29) - 1)
    return u.view(np.float64)


def test_double_to_float_pair_and_float_to_double():
    rng = np.random.default_rng(3)
    n = 4000
    x = rng.normal(size=n) * 10.0 ** rng.uniform(-25, 35, n)
    x = np.concatenate([x, [0.0, -0.0, 1.0, -1.5, 2.0 ** -74, -(2.0 ** -74), 1234.5678, -np.pi * 1e6,
                            2.0 ** 127 * 1.999, 2.0 ** -75, 1e-30, 3e38, 2.0 ** 128 * 1.5]])
    f = (rng.normal(size=x.size) * 10.0 ** rng.uniform(-37, 38, x.size)).astype(np.float32)
    specials = np.array([0.0, -0.0, 1e-45, -1e-45, 1.17549435e-38, 3.4028235e38, np.inf, -np.inf, 1.0, -2.5],
                        dtype=np.float32)
    f[:specials.size] = specials
    hi, lo, back, fd = rpba.rpba_check_formats(x, f)

    mag = np.abs(x)
    fast = (mag >= 2.0 ** -74) & (mag < 2.0 ** 128)
    # fast path: hi is the 24-bit truncation, lo the rest rounded to float
    t = _truncate24(x[fast])
    np.testing.assert_array_equal(hi[fast], t.astype(np.float32))
    np.testing.assert_array_equal(lo[fast], (x[fast] - t).astype(np.float32))
    # other magnitudes: the FP64 conversion (round to nearest, then the remainder)
    slow = ~fast & (mag < 3.4e38)
    h = x[slow].astype(np.float32)
    np.testing.assert_array_equal(hi[slow], h)
    np.testing.assert_array_equal(lo[slow], (x[slow] - h.astype(np.float64)).astype(np.float32))
    # the pair sums back exactly in FP64 and keeps 2^-48 of x
    normal_lo = (lo == 0) | (np.abs(lo) >= np.float32(1.17549435e-38))  # the sum widens lo like fd below
    np.testing.assert_array_equal(back[normal_lo], hi[normal_lo].astype(np.float64) + lo[normal_lo].astype(np.float64))
    ok = fast & (mag > 0)
    assert np.all(np.abs(back[ok] - x[ok]) <= 2.0 ** -48 * mag[ok])
    assert hi[x == 0].tolist() == [0.0] * int((x == 0).sum()) and np.all(lo[x == 0] == 0)

    # float -> double: exact, subnormal floats flush to a zero of the same sign
    sub = (f != 0) & (np.abs(f) < np.float32(1.17549435e-38))
    want = f.astype(np.float64)
    want[sub] = np.copysign(0.0, f[sub].astype(np.float64))
    np.testing.assert_array_equal(fd, want)
    assert np.array_equal(np.signbit(fd), np.signbit(want))
