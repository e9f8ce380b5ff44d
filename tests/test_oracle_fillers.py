"""Pins of the oracle's filler cells (ePlace whitespace fillers, cited by the
paper through the density penalty of Eq. 2) and of the placer with them."""
import math

import numpy as np
import pytest

from oracle import density as dens
from oracle import fillers as fil
from oracle import placer as pl
from paper_2402_18311_gb300 import synth


def test_size_is_the_rounded_mean_of_the_movable_standard_cells():
    # widths 1, 2, 4 units and a macro of 10 at F = 2: mean of 4, 8, 16 -> 9.33 -> 9
    Wq = np.array([4, 8, 16, 40, 99], np.int64)
    Hq = np.array([4, 4, 4, 40, 99], np.int64)
    macro = np.array([0, 0, 0, 1, 0], np.uint8)
    assert fil.size(Wq, Hq, 4, macro) == (9, 4)
    # ties round to even: mean 2.5 -> 2, mean 3.5 -> 4
    assert fil.size(np.array([2, 3]), np.array([3, 4]), 2, None) == (2, 4)
    assert fil.size(np.array([5]), np.array([5]), 0, None) == (0, 0)


def test_count_fills_the_whitespace_at_the_target_density():
    # die 16 x 16, fixed area 16 inside, movable area 40, t = 0.5:
    # 0.5 (256 - 16) - 40 = 80 -> 80 / (2 x 1) = 40 fillers
    F = 3
    s2 = 2 ** (2 * F)
    assert fil.count((0, 0, 16, 16), 0.5, 16 * s2, 40 * s2, F, 2 * 8, 1 * 8) == 40
    # one unit of area short of 41
    assert fil.count((0, 0, 16, 16), 0.5, 16 * s2, 41 * s2, F, 2 * 8, 1 * 8) == 39
    # no whitespace left at the target density: none
    assert fil.count((0, 0, 16, 16), 0.5, 16 * s2, 120 * s2, F, 16, 8) == 0


def test_start_positions_are_inside_the_die_and_uniform():
    n = 4000
    x, y = fil.start(n, (-8.0, 4.0, 56.0, 36.0), 2.5, 1.0)
    assert x.dtype == np.float32 and x.shape == (n,)
    assert np.all(x >= -8.0) and np.all(x + 2.5 <= 56.0)
    assert np.all(y >= 4.0) and np.all(y + 1.0 <= 36.0)
    # uniform: 10 equal slices in each axis, chi-square with 9 dof well below 30
    for v, lo, hi in ((x, -8.0, 56.0 - 2.5), (y, 4.0, 36.0 - 1.0)):
        counts, _ = np.histogram(v, bins=10, range=(lo, hi))
        chi2 = float(np.sum((counts - n / 10) ** 2 / (n / 10)))
        assert chi2 < 30, chi2
    # the same stream from the same seed; another seed moves them
    x2, _ = fil.start(n, (-8.0, 4.0, 56.0, 36.0), 2.5, 1.0)
    np.testing.assert_array_equal(x, x2)
    x3, _ = fil.start(n, (-8.0, 4.0, 56.0, 36.0), 2.5, 1.0, seed=5)
    assert not np.array_equal(x, x3)


def _placers(d, iters, **kw):
    a = pl.Placer(d, pl.Params(tau_stop=-1.0, max_iters=10 ** 6, **kw))
    b = pl.Placer(d, pl.Params(tau_stop=-1.0, max_iters=10 ** 6, fillers=True, **kw))
    a.run(iters)
    b.run(iters)
    return a, b


def test_placer_with_fillers_keeps_them_out_of_wirelength_and_overflow():
    d = synth.tiny_1k(0)
    p = pl.Placer(d, pl.Params(tau_stop=-1.0, max_iters=100, fillers=True))
    n, nf = p.n, p.nf
    # tiny_1k: t = 1, die 256^2, 16 pads, movable area 1000 cells: the count
    Wf, Hf = fil.size(p.W, p.H, n, d.is_macro)
    assert nf == math.floor((1.0 * (256.0 ** 2 - 16.0) - p.mov_area_q * 2.0 ** (-2 * p.F))
                            / (Wf * Hf * 2.0 ** (-2 * p.F)))
    assert nf > 10 * n
    # the field map holds movable and filler area; the overflow's map only movable
    Mf = p.field_map(p.vx, p.vy)
    M = p.density_map(p.vx, p.vy)
    assert int(Mf.sum()) == p.mov_area_q + nf * Wf * Hf
    assert int(M.sum()) == p.mov_area_q
    # no pins on fillers: zero WA gradient; positions and HPWL of real cells only
    _, gx, gy = p.wirelength(p.vx, p.vy, 4.0)
    assert gx.shape == (n + nf,) and not np.any(gx[n:]) and not np.any(gy[n:])
    fx, fy = p.positions()
    assert fx.shape == (d.n_cells,)
    # one step: fillers move under the density force alone, real cells too
    x0, y0 = p.vx.copy(), p.vy.copy()
    p.step()
    assert np.any(p.vx[n:] != x0[n:]) and np.any(p.vx[:n] != x0[:n])
    # their preconditioner is max(1, lambda area_f): g = lambda gD / P there
    assert p.pins[n:].sum() == 0 and np.all(p.area[n:] == p.area[n])


def test_fillers_hold_the_cells_together():
    # Without fillers the real cells spread until the whole die holds them;
    # with fillers the density force balances at the target density: placed
    # to the same overflow, the real cells stay closer together and their
    # wirelength is lower.
    d = synth.tiny_1k(0)
    a = pl.Placer(d, pl.Params(tau_stop=0.07, max_iters=1000))
    b = pl.Placer(d, pl.Params(tau_stop=0.07, max_iters=1000, fillers=True))
    a.run()
    b.run()
    assert a.converged and b.converged
    n = d.n_movable

    def spread(p):
        return float(np.std(p.vx[:n]) + np.std(p.vy[:n]))
    assert spread(b) < 0.8 * spread(a), (spread(a), spread(b))
    assert b.hpwl(b.vx, b.vy) < 0.9 * a.hpwl(a.vx, a.vy)


def test_no_whitespace_means_no_fillers():
    d = synth.tiny_1k(0)
    d.target_density = 0.038  # t (A_die - A_fixed) below the movable area
    a, b = _placers(d, 20)
    assert b.nf == 0
    np.testing.assert_array_equal(a.vx, b.vx)
    assert a.history == b.history


def test_reset_keeps_the_fillers_in_place():
    d = synth.tiny_1k(0)
    p = pl.Placer(d, pl.Params(tau_stop=-1.0, max_iters=100, fillers=True))
    p.run(30)
    fx, fy = p.vx[p.n:].copy(), p.vy[p.n:].copy()
    p.reset(d.x[:p.n], d.y[:p.n])
    np.testing.assert_array_equal(p.vx[p.n:], np.maximum(0.0, np.minimum(fx, 256.0 - p.wo[p.n:])))
    np.testing.assert_array_equal(p.vy[p.n:], fy)
    assert p.k == 0
