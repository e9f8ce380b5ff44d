"""The seeded input generator: designs are reproducible and independent
random starts differ only in the movable cells."""
import numpy as np

from paper_2402_18311_gb300 import synth


def test_random_start_redraws_movable_cells_only():
    d = synth.tiny_1k(0)
    n = d.n_movable
    x1, y1 = synth.random_start(d, 3)
    x2, y2 = synth.random_start(d, 3)
    x3, _ = synth.random_start(d, 4)
    np.testing.assert_array_equal(x1, x2)
    np.testing.assert_array_equal(y1, y2)
    assert not np.array_equal(x1[:n], x3[:n])
    np.testing.assert_array_equal(x1[n:], d.x[n:])
    np.testing.assert_array_equal(y1[n:], d.y[n:])
    xl, yl, xh, yh = d.die
    assert np.all(x1[:n] >= xl) and np.all(x1[:n] + d.w[:n] <= xh)
    assert np.all(y1[:n] >= yl) and np.all(y1[:n] + d.h[:n] <= yh)
    # centred: within a few sigma (1e-3 of the extent) of the die centre
    cx = x1[:n] + 0.5 * d.w[:n]
    assert abs(float(np.mean(cx)) - 0.5 * (xl + xh)) < 0.01 * (xh - xl)


def test_designs_are_reproducible():
    a, b = synth.tiny_1k(0), synth.tiny_1k(0)
    for f in ("w", "h", "x", "y", "net_ptr", "pin_cell", "pin_dx", "pin_dy"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


def test_medium_mixed_has_movable_macros_inside_the_die():
    base, d = synth.medium_210k(0), synth.medium_mixed_210k(0)
    n = d.n_movable
    mac = np.nonzero(d.is_macro[:n])[0]
    assert mac.size == 32
    assert np.all((d.w[mac] >= 16) & (d.w[mac] <= 64) & (d.h[mac] >= 16) & (d.h[mac] <= 64))
    xl, yl, xh, yh = d.die
    assert np.all(d.x[mac] >= xl) and np.all(d.x[mac] + d.w[mac] <= xh)
    assert np.all(d.y[mac] >= yl) and np.all(d.y[mac] + d.h[mac] <= yh)
    # everything else is the medium design, and the fixed macros stay flagged
    other = np.setdiff1d(np.arange(d.n_cells), mac)
    for f in ("w", "h", "x", "y"):
        np.testing.assert_array_equal(getattr(d, f)[other], getattr(base, f)[other])
    np.testing.assert_array_equal(d.is_macro[n:], base.is_macro[n:])
    np.testing.assert_array_equal(d.pin_cell, base.pin_cell)
