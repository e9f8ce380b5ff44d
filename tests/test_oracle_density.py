"""Pins of the oracle's density map, overflow and field gather: exact mass,
brute force on tiny cases, hand-computed 2x2 grids and rounding rules."""
import numpy as np
import pytest

from oracle import density as dens


def grid(nx=2, ny=2, die=(0, 0, 2, 2), F=4):
    return dens.Grid(die, nx, ny, F)


def test_quantize_rounds_half_to_even():
    F = 3
    s = 2.0 ** -F
    v = np.array([0.5 * s, 1.5 * s, 2.5 * s, -0.5 * s, 3.25 * s], np.float32)
    assert dens.quantize(v, F).tolist() == [0, 2, 2, 0, 3]


def test_frac_bits_examples():
    # die 256: 256 * 2^21 = 2^29 < 2^30 but 2^30 is not; area 2516 * 2^42 < 2^62
    assert dens.frac_bits((0, 0, 256, 256), 2516.0) == 21
    assert dens.frac_bits((0, 0, 4096, 4096), 1.1e7) == 17
    # area bound binds: 2^40 * 2^(2F) < 2^62 -> F = 10
    assert dens.frac_bits((0, 0, 8, 8), 2.0 ** 40) == 10
    # a die across the origin: the extent, 1200, sets F (600 alone would
    # allow 20), so that bin-relative coordinates stay below 2^30
    assert dens.frac_bits((-600, -600, 600, 600), 1.0) == 19
    assert dens.frac_bits((-600, 0, 0, 600), 1.0) == 20


def test_hand_computed_2x2():
    # bins of 1x1 on a 2x2 die, F = 4 (1 unit = 16).
    g = grid()
    # cell 1.5 x 0.5 at (0.75, 0.25): bin (0,0) gets 0.25*0.5, bin (1,0) gets 1.0*0.5
    X, Y = dens.quantize([0.75], 4), dens.quantize([0.25], 4)
    W, H = dens.quantize([1.5], 4), dens.quantize([0.5], 4)
    M = dens.overlap_map(X, Y, W, H, g)
    u = 16 * 16
    assert M.tolist() == [[int(0.125 * u), 0], [int(0.5 * u), 0]]


def test_overflow_hand_computed():
    g = grid()
    u = 256
    M = np.array([[2 * u, 0], [u // 2, 0]], np.int64)      # 2.0 and 0.5 units of area
    Fm = np.array([[0, 0], [u // 2, 0]], np.int64)         # half of bin (1,0) fixed
    # t = 1: excess bin(0,0) = 2 - 1 = 1; bin(1,0) = 0.5 - (1 - 0.5) = 0 -> tau = 1 / 2.5
    assert dens.overflow(M, Fm, 1.0, g, int(2.5 * u)) == pytest.approx(0.4, rel=1e-15)
    # t = 0.5: bin(0,0) 2 - 0.5 = 1.5; bin(1,0) 0.5 - 0.25 = 0.25 -> tau = 1.75 / 2.5
    assert dens.overflow(M, Fm, 0.5, g, int(2.5 * u)) == pytest.approx(0.7, rel=1e-15)
    rho = dens.bin_density(M, Fm, 0.5, g)
    assert rho.tolist() == [[2.0, 0.0], [0.75, 0.0]]


def test_mass_is_exact_and_matches_bruteforce():
    rng = np.random.default_rng(0)
    g = dens.Grid((0, 0, 40, 24), 10, 6, 8)
    n = 60
    w = rng.integers(1, 9, n).astype(np.float32)
    h = rng.integers(1, 5, n).astype(np.float32)
    x = (rng.random(n) * (40 - w)).astype(np.float32)
    y = (rng.random(n) * (24 - h)).astype(np.float32)
    X, Y = dens.quantize(x, 8), dens.quantize(y, 8)
    W, H = dens.quantize(w, 8), dens.quantize(h, 8)
    M = dens.overlap_map(X, Y, W, H, g)
    assert int(M.sum()) == int(np.sum(W * H))
    for k in (1, 2, 3):
        np.testing.assert_array_equal(dens.overlap_map(X[:k], Y[:k], W[:k], H[:k], g),
                                      dens.overlap_map_bruteforce(X[:k], Y[:k], W[:k], H[:k], g))
    np.testing.assert_array_equal(M, dens.overlap_map_bruteforce(X, Y, W, H, g))


def test_cell_outside_die_is_clipped():
    g = grid()
    # a 1x1 cell hanging half off the right edge keeps only the inside half
    M = dens.overlap_map(dens.quantize([1.5], 4), dens.quantize([0.0], 4),
                         dens.quantize([1.0], 4), dens.quantize([1.0], 4), g)
    assert int(M.sum()) == 128


def test_gather_single_cell_inside_one_bin():
    g = dens.Grid((0, 0, 8, 8), 4, 4, 6)
    ex = np.arange(16, dtype=np.float64).reshape(4, 4)
    ey = -2.0 * ex
    # 1.5 x 0.75 cell inside bin (2, 1) = [4,6) x [2,4)
    X, Y = dens.quantize([4.25], 6), dens.quantize([2.5], 6)
    W, H = dens.quantize([1.5], 6), dens.quantize([0.75], 6)
    gx, gy = dens.field_gather(X, Y, W, H, g, ex, ey)
    area = 1.5 * 0.75
    assert gx[0] == pytest.approx(-area * ex[2, 1], rel=1e-15)
    assert gy[0] == pytest.approx(-area * ey[2, 1], rel=1e-15)


def test_gather_is_overlap_weighted():
    g = grid()
    ex = np.array([[1.0, 10.0], [100.0, 1000.0]])
    ey = np.zeros((2, 2))
    # unit cell centred on the grid corner overlaps each bin by 1/4
    gx, _ = dens.field_gather(dens.quantize([0.5], 4), dens.quantize([0.5], 4),
                              dens.quantize([1.0], 4), dens.quantize([1.0], 4), g, ex, ey)
    assert gx[0] == pytest.approx(-0.25 * 1111.0, rel=1e-15)


def test_stretch_axis_widens_narrow_cells_about_their_centre():
    # BW = 100: sqrt(2) * 100 = 141.42... -> 141
    Xs, Ws = dens.stretch_axis([1000, 1000, 1000, 5], [40, 141, 300, 41], 100)
    assert Ws.tolist() == [141, 141, 300, 141]
    # growth 101 -> 50 to the left (floor), 51 to the right; unchanged cells stay
    assert Xs.tolist() == [950, 1000, 1000, -45]
    # the centre moves by at most half a unit
    for x, w, xs, ws in zip([1000, 1000, 1000, 5], [40, 141, 300, 41], Xs, Ws):
        assert abs((2 * xs + ws) - (2 * x + w)) <= 1


def test_stretch_scale_is_the_floored_area_ratio():
    R = dens.stretch_scale([40, 300], [10, 300], [141, 300], [141, 300])
    assert R[0] == (40 * 10 << 31) // (141 * 141) and R[1] == 1 << 31


def test_scaled_map_keeps_each_cells_charge():
    # cells inside the die: the stretched, scaled map sums to the cells' areas
    # up to one unit per (cell, bin) term lost to the floor; a cell that is
    # not stretched contributes its exact overlaps
    g = dens.Grid((0.0, 0.0, 64.0, 64.0), 8, 8, 4)
    rng = np.random.default_rng(5)
    n = 40
    W = rng.integers(1, 200, n); H = rng.integers(1, 200, n)
    X = rng.integers(300, 600, n); Y = rng.integers(300, 600, n)
    Xs, Ys, Ws, Hs, R, wgt = dens.stretched(X, Y, W, H, g)
    M = dens.overlap_map_scaled(Xs, Ys, Ws, Hs, R, g)
    terms = sum(len(range((x - g.XL) // g.BW, (x + w - 1 - g.XL) // g.BW + 1)) *
                len(range((y - g.YL) // g.BH, (y + h - 1 - g.YL) // g.BH + 1))
                for x, y, w, h in zip(Xs, Ys, Ws, Hs))
    area = int(np.sum(W * H))
    assert area - terms <= int(M.sum()) <= area
    # R = 2^31 (no stretch in either axis) reproduces the exact map
    big = (W >= 181) & (H >= 181)
    np.testing.assert_array_equal(
        dens.overlap_map_scaled(X[big], Y[big], W[big], H[big], np.full(big.sum(), 1 << 31), g),
        dens.overlap_map(X[big], Y[big], W[big], H[big], g))


def test_scaled_map_against_brute_force():
    g = dens.Grid((0.0, 0.0, 16.0, 16.0), 4, 4, 3)
    X = np.array([5, 40, 70]); Y = np.array([9, 33, 100]); W = np.array([7, 30, 2]); H = np.array([3, 30, 50])
    Xs, Ys, Ws, Hs, R, _ = dens.stretched(X, Y, W, H, g)
    M = np.zeros((4, 4), np.int64)
    for i in range(3):
        for kx in range(4):
            ox = max(0, min(int(Xs[i] + Ws[i]), (kx + 1) * g.BW) - max(int(Xs[i]), kx * g.BW))
            for ky in range(4):
                oy = max(0, min(int(Ys[i] + Hs[i]), (ky + 1) * g.BH) - max(int(Ys[i]), ky * g.BH))
                M[kx, ky] += (ox * oy * int(R[i])) >> 31
    np.testing.assert_array_equal(dens.overlap_map_scaled(Xs, Ys, Ws, Hs, R, g), M)


def test_stretched_gradient_in_a_uniform_field_is_minus_area_times_field():
    # the gradient weight restores the charge: r * sum_b a'_ib E = W H E
    g = dens.Grid((0.0, 0.0, 64.0, 64.0), 8, 8, 4)
    X = np.array([400, 520]); Y = np.array([410, 300]); W = np.array([20, 37]); H = np.array([16, 90])
    Xs, Ys, Ws, Hs, R, wgt = dens.stretched(X, Y, W, H, g)
    Ex = np.full((8, 8), 0.75); Ey = np.full((8, 8), -2.0)
    gx, gy = dens.field_gather(Xs, Ys, Ws, Hs, g, Ex, Ey)
    area = (W * H).astype(np.float64) * 2.0 ** (-2 * g.F)
    np.testing.assert_allclose(wgt * gx, -0.75 * area, rtol=1e-12)
    np.testing.assert_allclose(wgt * gy, 2.0 * area, rtol=1e-12)


def test_scaled_term_is_the_exact_floored_product():
    # floor(ov R / 2^31) against Python's unbounded integers, at the edges
    # of its range and on random values
    rng = np.random.default_rng(5)
    ov = [0, 1, (1 << 31) - 1, 1 << 31, (1 << 62) - 1, (1 << 40) + 12345]
    R = [0, 1, (1 << 31) - 1, 1 << 31, 1 << 30, 3]
    ov += [int(v) for v in rng.integers(0, 1 << 62, 200, dtype=np.int64)]
    R += [int(v) for v in rng.integers(0, (1 << 31) + 1, 200, dtype=np.int64)]
    for a in ov:
        for r in (R[:6] if a not in ov[:6] else R):
            assert int(dens.scaled_term(a, r)) == (a * r) >> 31, (a, r)
    # R = 2^31 leaves every term whole, R = 0 removes it
    assert int(dens.scaled_term((1 << 62) - 1, 1 << 31)) == (1 << 62) - 1
    assert int(dens.scaled_term((1 << 62) - 1, 0)) == 0
