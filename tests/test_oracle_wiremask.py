"""Pins of the oracle's WireMask perturbation (Section 4.2).

The wire mask is pinned against the oracle's Eq. 1 HPWL (itself pinned by
brute force in test_oracle_wirelength.py).  For every macro and every
candidate, the total HPWL of the design with the macro moved there, minus
the mask, is one constant.  The chosen candidate minimises the total HPWL
over the free candidates, which are found here by a separate rectangle
test.
"""
import numpy as np

from oracle import hybro
from oracle import wiremask as wm
from oracle.wirelength import hpwl
from paper_2402_18311_gb300 import synth


def _design(cells, nets, n_movable, die, nx, ny, macros):
    """cells: [(w, h, x, y)]; nets: [[(cell, dx, dy), ...]]."""
    w = np.array([c[0] for c in cells], np.float32)
    h = np.array([c[1] for c in cells], np.float32)
    x = np.array([c[2] for c in cells], np.float32)
    y = np.array([c[3] for c in cells], np.float32)
    ptr = np.cumsum([0] + [len(n) for n in nets]).astype(np.int32)
    pc = np.array([p[0] for n in nets for p in n], np.int32)
    pdx = np.array([p[1] for n in nets for p in n], np.float32)
    pdy = np.array([p[2] for n in nets for p in n], np.float32)
    mac = np.zeros(len(cells), np.uint8)
    mac[list(macros)] = 1
    return synth.Design("hand", n_movable, w, h, x, y, ptr, pc, pdx, pdy, die, nx, ny, 1.0, mac)


def _apply(d, trace=None):
    return wm.wiremask(d.x, d.y, d.w, d.h, d.net_ptr, d.pin_cell, d.pin_dx, d.pin_dy,
                       d.n_movable, d.is_macro, d.die, d.nx, d.ny, trace=trace)


def test_hand_example():
    # Die 8 x 8, 1 x 1 bins, a fixed 1 x 1 pad at (7, 7) with its pin at its
    # centre (7.5, 7.5).  A (2 x 2, pin at (1, 1)) and B (1 x 2, pin at
    # (0.5, 0.5)) are each wired to the pad; A (area 4) moves first.
    # A: mask |X - 6.5| + |Y - 6.5|, least at (6, 6) (7 leaves the die), which
    # overlaps the pad.  (6, 5) and (5, 6) tie at 2, both at distance 11 from
    # (0, 0); the smaller row wins: A -> (6, 5), covering [6,8) x [5,7).
    # B: mask |X - 7| + |Y - 7| with X <= 7, Y <= 6.  (7, 6) at 1 hits the pad
    # and A; (6, 6) and (7, 5) at 2 hit A; at 3 only (5, 6) is free
    # ((6, 5) and (7, 4) hit A): B -> (5, 6).
    d = _design([(2, 2, 0, 0), (1, 2, 0, 0), (1, 1, 7, 7)],
                [[(0, 1.0, 1.0), (2, 0.5, 0.5)], [(1, 0.5, 0.5), (2, 0.5, 0.5)]],
                n_movable=2, die=(0.0, 0.0, 8.0, 8.0), nx=8, ny=8, macros=[0, 1])
    assert wm.macro_order(d.w, d.h, d.is_macro, d.n_movable) == [0, 1]
    x, y = _apply(d)
    assert (x[0], y[0]) == (6.0, 5.0)
    assert (x[1], y[1]) == (5.0, 6.0)
    assert (x[2], y[2]) == (7.0, 7.0)


def test_unmoved_macro_pins_count_at_their_current_place():
    # A is wired to the pad and to B, which still sits at (7, 0) (pin at
    # (7.5, 0.5)) when A moves.  In x both nets pull the same way,
    # 2 |X + 1 - 7.5|, so X = 6; in y they pull apart,
    # |Y + 1 - 7.5| + |Y + 1 - 0.5| = 7 on [0, 6], and the distance from (0, 0)
    # picks Y = 0: A -> (6, 0).
    d = _design([(2, 2, 0, 0), (1, 2, 7, 0), (1, 1, 7, 7)],
                [[(0, 1.0, 1.0), (2, 0.5, 0.5)], [(0, 1.0, 1.0), (1, 0.5, 0.5)]],
                n_movable=2, die=(0.0, 0.0, 8.0, 8.0), nx=8, ny=8, macros=[0, 1])
    trace = []
    x, y = _apply(d, trace)
    assert (x[0], y[0]) == (6.0, 0.0)
    np.testing.assert_array_equal(trace[0][2][:7], np.full(7, 7.0))


def test_macro_without_nets_goes_to_nearest_free_corner():
    d = _design([(2, 2, 3.3, 4.6), (1, 1, 0, 0)], [[(1, 0.5, 0.5)]], n_movable=1,
                die=(0.0, 0.0, 8.0, 8.0), nx=8, ny=8, macros=[0])
    x, y = _apply(d)
    # L1 distances from (3.3, 4.6): (3, 5) 0.7, (3, 4) 0.9, (4, 5) 1.1
    assert (x[0], y[0]) == (3.0, 5.0)


def test_no_free_candidate_keeps_position():
    # a fixed block covers the die: the macro cannot go anywhere
    d = _design([(2, 2, 1.25, 2.5), (8, 8, 0, 0)], [[(0, 1, 1), (1, 4, 4)]], n_movable=1,
                die=(0.0, 0.0, 8.0, 8.0), nx=8, ny=8, macros=[0])
    trace = []
    x, y = _apply(d, trace)
    assert (x[0], y[0]) == (np.float32(1.25), np.float32(2.5))
    assert trace[0][3] is None


def test_no_movable_macros_is_identity():
    d = synth.tiny_1k(0)
    x, y = _apply(d)
    assert np.array_equal(x, d.x) and np.array_equal(y, d.y)


def _free(d, x, y, m, obstacles, X, Y):
    xl, yl, xh, yh = d.die
    free = []
    for j, yy in enumerate(Y):
        for i, xx in enumerate(X):
            if xx + float(d.w[m]) > xh or yy + float(d.h[m]) > yh:
                continue
            hit = False
            for o in obstacles:
                ox0, ox1 = float(x[o]), float(x[o]) + float(d.w[o])
                oy0, oy1 = float(y[o]), float(y[o]) + float(d.h[o])
                if min(ox1, xx + float(d.w[m])) > max(ox0, xx) and \
                        min(oy1, yy + float(d.h[m])) > max(oy0, yy):
                    hit = True
                    break
            if not hit:
                free.append((i, j))
    return free


def test_mask_is_total_hpwl_up_to_a_constant_and_choice_is_least():
    d = synth.make_design(n_movable=150, die=(0, 0, 64, 64), nx=16, ny=16, n_nets=170,
                          n_pads=8, target_density=1.0, seed=5, name="wm_small")
    rng = np.random.default_rng(3)
    mac = rng.choice(d.n_movable, 6, replace=False)
    d.w[mac] = rng.integers(5, 13, 6).astype(np.float32)
    d.h[mac] = rng.integers(5, 13, 6).astype(np.float32)
    d.x[mac] = np.minimum(d.x[mac], 64 - d.w[mac]).astype(np.float32)
    d.y[mac] = np.minimum(d.y[mac], 64 - d.h[mac]).astype(np.float32)
    d.is_macro[:] = 0
    d.is_macro[mac] = 1
    trace = []
    xf, yf = _apply(d, trace)
    X = wm.grid_corners(d.die[0], d.die[2], d.nx)
    Y = wm.grid_corners(d.die[1], d.die[3], d.ny)
    x, y = d.x.copy(), d.y.copy()
    obstacles = [i for i in range(d.n_movable, d.n_cells) if d.w[i] > 0 and d.h[i] > 0]
    assert [t[0] for t in trace] == wm.macro_order(d.w, d.h, d.is_macro, d.n_movable)
    for m, fx, fy, chosen in trace:
        free = _free(d, x, y, m, obstacles, X, Y)
        assert chosen is not None and free
        tot = {}
        for (i, j) in free:
            xx, yy = x.copy(), y.copy()
            xx[m], yy[m] = X[i], Y[j]
            tot[(i, j)] = hpwl(d.net_ptr, d.pin_cell, d.pin_dx, d.pin_dy, xx, yy)
        diff = np.array([tot[k] - (fx[k[0]] + fy[k[1]]) for k in free])
        assert np.ptp(diff) <= 1e-9 * max(tot.values())
        assert chosen in tot
        assert tot[chosen] <= min(tot.values()) + 1e-9 * max(tot.values())
        x[m], y[m] = X[chosen[0]], Y[chosen[1]]
        obstacles.append(m)
    assert np.array_equal(x, xf) and np.array_equal(y, yf)


def test_invariants_on_mixed_size_design():
    d = synth.mixed_size_1k(0)
    x, y = _apply(d)
    mac = np.nonzero(d.is_macro[:d.n_movable])[0]
    other = np.setdiff1d(np.arange(d.n_cells), mac)
    assert np.array_equal(x[other], d.x[other]) and np.array_equal(y[other], d.y[other])
    X = wm.grid_corners(d.die[0], d.die[2], d.nx)
    Y = wm.grid_corners(d.die[1], d.die[3], d.ny)
    assert np.isin(x[mac], X.astype(np.float32)).all() and np.isin(y[mac], Y.astype(np.float32)).all()
    assert (x[mac] + d.w[mac] <= d.die[2]).all() and (y[mac] + d.h[mac] <= d.die[3]).all()
    blocks = list(mac) + [i for i in range(d.n_movable, d.n_cells) if d.w[i] > 0]
    for a in range(len(blocks)):
        for b in range(a + 1, len(blocks)):
            p, q = blocks[a], blocks[b]
            ox = min(x[p] + d.w[p], x[q] + d.w[q]) - max(x[p], x[q])
            oy = min(y[p] + d.h[p], y[q] + d.h[q]) - max(y[p], y[q])
            assert not (ox > 0 and oy > 0), (p, q)


def test_hybro_loop_runs_wiremask():
    d = synth.mixed_size_1k(0)
    from oracle import placer as pl
    prm = pl.Params(max_iters=20, tau_stop=0.0)
    best, rounds = hybro.run(d, prm, 1, op=hybro.WIREMASK)
    assert len(rounds) == 2 and best in (0, 1)


def test_weighted_mask_is_weighted_total_hpwl_up_to_a_constant():
    # with net weights the mask is the weighted Eq. 1 HPWL up to a constant
    d = synth.make_design(n_movable=120, die=(0, 0, 64, 64), nx=16, ny=16, n_nets=140,
                          n_pads=8, target_density=1.0, seed=9, name="wm_weighted")
    rng = np.random.default_rng(4)
    mac = rng.choice(d.n_movable, 4, replace=False)
    d.w[mac] = rng.integers(5, 11, 4).astype(np.float32)
    d.h[mac] = rng.integers(5, 11, 4).astype(np.float32)
    d.is_macro[:] = 0
    d.is_macro[mac] = 1
    net_w = rng.uniform(0.5, 2.0, d.n_nets).astype(np.float32)
    trace = []
    wm.wiremask(d.x, d.y, d.w, d.h, d.net_ptr, d.pin_cell, d.pin_dx, d.pin_dy, d.n_movable,
                d.is_macro, d.die, d.nx, d.ny, net_w=net_w, trace=trace)
    X = wm.grid_corners(d.die[0], d.die[2], d.nx)
    Y = wm.grid_corners(d.die[1], d.die[3], d.ny)
    x, y = d.x.copy(), d.y.copy()
    m, fx, fy, chosen = trace[0]
    diffs = []
    for j in range(0, d.ny, 3):
        for i in range(0, d.nx, 3):
            xx, yy = x.copy(), y.copy()
            xx[m], yy[m] = X[i], Y[j]
            tot = hpwl(d.net_ptr, d.pin_cell, d.pin_dx, d.pin_dy, xx, yy, net_w=net_w)
            diffs.append(tot - (fx[i] + fy[j]))
    assert np.ptp(diffs) <= 1e-9 * abs(max(diffs, key=abs))


def test_nets_of_lists_each_net_of_a_cell_once_in_order():
    # nets: 0 = {0, 1}, 1 = {2, 3}, 2 = {1, 1, 4} (cell 1 twice), 3 = {1}
    net_ptr = [0, 2, 4, 7, 8]
    pin_cell = [0, 1, 2, 3, 1, 1, 4, 1]
    assert wm.nets_of(net_ptr, pin_cell, 1) == [0, 2, 3]
    assert wm.nets_of(net_ptr, pin_cell, 2) == [1]
    assert wm.nets_of(net_ptr, pin_cell, 5) == []


def test_axis_mask_is_each_nets_extent_with_the_macro_at_the_corner():
    # one axis, macro m = 0 with pins at offsets 1 and 3; net 0 joins it to
    # cells at 10 and 4 (offsets 0.5, 0); net 1 to nothing else; net 2 is
    # another cell's only (weight 2 for net 0 checks the weighting)
    net_ptr = [0, 4, 5]
    pin_cell = [0, 1, 0, 2, 0]
    pin_d = np.array([1.0, 0.5, 3.0, 0.0, 2.0])
    pos = np.array([0.0, 10.0, 4.0])
    corners = np.array([0.0, 2.0, 8.0, 20.0])
    got = wm.axis_mask(corners, [0, 1], net_ptr, pin_cell, pin_d, pos, 0, np.array([2.0, 1.0]))
    want = []
    for c in corners:
        # net 0: points c+1, c+3 (macro), 10.5, 4; net 1: the single point c+2
        pts = [c + 1, c + 3, 10.5, 4.0]
        want.append(2.0 * (max(pts) - min(pts)) + 0.0)
    np.testing.assert_array_equal(got, np.array(want))
