"""Pins of the oracle's HPWL (Eq. 1) and WA wirelength (Eq. 3) against facts
fixed by the mathematics: the 2-pin closed form, finite differences,
bounds, the gamma -> 0 limit and translation invariance."""
import math

import numpy as np
import pytest

from oracle import wirelength as wlm


def small_netlist(seed=1, n_cells=30, n_nets=25, max_deg=9):
    rng = np.random.default_rng(seed)
    deg = rng.integers(1, max_deg + 1, n_nets)
    ptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int32)
    cells = np.concatenate([rng.choice(n_cells, d, replace=False) for d in deg]).astype(np.int32)
    dx = rng.random(cells.size).astype(np.float32)
    dy = rng.random(cells.size).astype(np.float32)
    x = (rng.random(n_cells) * 50).astype(np.float32)
    y = (rng.random(n_cells) * 50).astype(np.float32)
    return ptr, cells, dx, dy, x, y


def test_two_pin_closed_form():
    # Two pins at 0 and d: WL = d tanh(d / 2g); dWL/dd = tanh(d/2g) + (d/2g) sech^2(d/2g).
    for d, g in [(3.0, 1.0), (0.25, 2.0), (40.0, 3.5), (1e-3, 1.0)]:
        ptr = np.array([0, 2])
        wl, gp = wlm.wa_axis(ptr, np.array([0.0, d]), g)
        s = d / (2 * g)
        assert wl[0] == pytest.approx(d * math.tanh(s), rel=1e-13, abs=1e-15)
        dd = math.tanh(s) + s / math.cosh(s) ** 2
        assert gp[1] == pytest.approx(dd, rel=1e-12)
        assert gp[0] == pytest.approx(-dd, rel=1e-12)


def test_hpwl_bruteforce():
    ptr, cells, dx, dy, x, y = small_netlist()
    tot = 0.0
    for e in range(len(ptr) - 1):
        xs = [float(x[cells[j]]) + float(dx[j]) for j in range(ptr[e], ptr[e + 1])]
        ys = [float(y[cells[j]]) + float(dy[j]) for j in range(ptr[e], ptr[e + 1])]
        tot += (max(xs) - min(xs)) + (max(ys) - min(ys))
    assert wlm.hpwl(ptr, cells, dx, dy, x, y) == pytest.approx(tot, rel=1e-14)


def test_hpwl_empty_and_single_pin_nets():
    ptr = np.array([0, 0, 1, 1, 3])
    cells = np.array([0, 1, 2])
    z = np.zeros(3, np.float32)
    x = np.array([5, 1, 4], np.float32)
    y = np.array([0, 2, 7], np.float32)
    per = wlm.hpwl_per_net(ptr, cells, z, z, x, y)
    assert per.tolist() == [0.0, 0.0, 0.0, 3.0 + 5.0]


def test_wa_gradient_matches_central_differences():
    ptr, cells, dx, dy, x, y = small_netlist(seed=3)
    n_mov = 24  # the last 6 cells are fixed
    g = 2.5
    x = x.astype(np.float64); y = y.astype(np.float64)
    _, gx, gy = wlm.wa_wirelength(ptr, cells, dx, dy, x, y, g, n_mov)
    h = 1e-4 * g
    for i in range(n_mov):
        for arr, grad in ((x, gx), (y, gy)):
            old = arr[i]
            arr[i] = old + h
            fp, _, _ = wlm.wa_wirelength(ptr, cells, dx, dy, x, y, g, n_mov)
            arr[i] = old - h
            fm, _, _ = wlm.wa_wirelength(ptr, cells, dx, dy, x, y, g, n_mov)
            arr[i] = old
            fd = (fp - fm) / (2 * h)
            assert grad[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_wa_bounded_by_hpwl_and_tends_to_it():
    ptr, cells, dx, dy, x, y = small_netlist(seed=5)
    px, _ = wlm.pin_positions(cells, dx, dy, x, y)
    z = np.zeros_like(dy)
    hp = wlm.hpwl_per_net(ptr, cells, dx, z, x, np.zeros_like(y))  # x part only
    for g in [100.0, 10.0, 1.0]:
        wl, _ = wlm.wa_axis(ptr, px, g)
        assert np.all(wl >= -1e-12) and np.all(wl <= hp + 1e-9)
    # gamma = 1e-4 bin widths (bin width 4): the WA value is within 1e-6 of HPWL
    wl, _ = wlm.wa_axis(ptr, px, 4e-4)
    assert np.sum(wl) == pytest.approx(np.sum(hp), rel=1e-6)


def test_wa_translation_invariance():
    ptr, cells, dx, dy, x, y = small_netlist(seed=7)
    px, _ = wlm.pin_positions(cells, dx, dy, x, y)
    wl, gp = wlm.wa_axis(ptr, px, 3.0)
    wl2, _ = wlm.wa_axis(ptr, px + 1234.5, 3.0)
    np.testing.assert_allclose(wl, wl2, rtol=1e-9, atol=1e-9)
    sums = np.add.reduceat(gp, ptr[:-1].astype(np.int64))
    np.testing.assert_allclose(sums, 0.0, atol=1e-12)


def test_net_weights_scale_value_and_gradient():
    ptr, cells, dx, dy, x, y = small_netlist(seed=9)
    w = np.linspace(0.5, 2.0, len(ptr) - 1)
    a, gx, gy = wlm.wa_wirelength(ptr, cells, dx, dy, x, y, 2.0, 30)
    b, hx, hy = wlm.wa_wirelength(ptr, cells, dx, dy, x, y, 2.0, 30, net_w=2 * np.ones_like(w))
    assert b == pytest.approx(2 * a, rel=1e-14)
    np.testing.assert_allclose(hx, 2 * gx, rtol=1e-14, atol=1e-15)
