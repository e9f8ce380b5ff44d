"""Pins of the oracle's Nesterov/Lipschitz optimiser and its placement loop."""
import math

import numpy as np
import pytest

from oracle import placer as pl
from paper_2402_18311_gb300 import synth


def _noclamp(*a):
    return tuple(a)


def test_lipschitz_step_on_quadratic_is_inverse_curvature():
    # f(x) = c/2 |x|^2 -> g = c x, so |dv| / |dg| = 1 / c exactly
    rng = np.random.default_rng(0)
    for c in (0.5, 3.0, 40.0):
        v = (rng.standard_normal(7), rng.standard_normal(7))
        vp = (rng.standard_normal(7), rng.standard_normal(7))
        g = tuple(c * a for a in v)
        gp = tuple(c * a for a in vp)
        assert pl.lipschitz_step(v, vp, g, gp, 0.0) == pytest.approx(1.0 / c, rel=1e-14)
    # equal gradients keep the previous step
    assert pl.lipschitz_step(v, vp, v, v, 0.25) == 0.25


def test_nesterov_momentum_sequence():
    a = 1.0
    seq = []
    for _ in range(4):
        _, _, a = pl.nesterov_update((np.zeros(1),), (np.zeros(1),), (np.zeros(1),), a, 0.1, _noclamp)
        seq.append(a)
    ref = [1.0]
    for _ in range(4):
        ref.append((1 + math.sqrt(4 * ref[-1] ** 2 + 1)) / 2)
    assert seq == pytest.approx(ref[1:], rel=1e-15)
    assert seq[0] == pytest.approx((1 + math.sqrt(5)) / 2, rel=1e-15)


def test_nesterov_converges_on_convex_quadratic():
    # f = 1/2 sum d_i x_i^2 with curvatures in [1, 50]; Lipschitz-step Nesterov
    # with fixed step 1/L converges like O(1/k^2)
    rng = np.random.default_rng(1)
    d = rng.uniform(1, 50, 40)
    x0 = rng.standard_normal(40) * 10
    v = u = (x0.copy(),)
    a = 1.0
    f0 = 0.5 * np.sum(d * x0 ** 2)
    for _ in range(300):
        g = (d * v[0],)
        u, v, a = pl.nesterov_update(v, u, g, a, 1.0 / 50.0, _noclamp)
    f = 0.5 * np.sum(d * u[0] ** 2)
    assert f < 1e-6 * f0


def test_first_step_is_plain_gradient_step_and_clamped():
    def clamp(x):
        return (np.clip(x, 0.0, 1.0),)
    u, v, a = pl.nesterov_update((np.array([0.5, 0.5]),), (np.array([0.5, 0.5]),),
                                 (np.array([1.0, -10.0]),), 1.0, 0.1, clamp)
    # a_0 = 1 gives zero momentum on the first step
    assert u[0].tolist() == [0.4, 1.0]
    assert v[0].tolist() == [0.4, 1.0]


def test_tiny_design_spreads_and_wirelength_grows_smoothly():
    d = synth.tiny_1k(0)
    p = pl.Placer(d, pl.Params(tau_stop=-1.0, max_iters=300))
    tau0 = p.tau
    p.run()
    assert p.k == 300
    assert tau0 > 0.9 and p.tau < 0.1
    # gamma follows the overflow-driven schedule
    k, hp, tau, gamma, lam = p.history[-1]
    tau_prev = p.history[-2][2]
    assert gamma == pytest.approx(4.0 * 4.0 * 10 ** ((20 / 9) * tau_prev - 11 / 9), rel=1e-12)


def test_stop_test_leaves_solution_at_reference_point():
    d = synth.tiny_1k(0)
    p = pl.Placer(d, pl.Params(tau_stop=0.5, max_iters=300))
    p.run()
    assert p.converged and p.tau <= 0.5
    M = p.density_map(p.vx, p.vy)
    assert p.overflow(M) == p.tau


def test_lambda_multiplier_special_cases():
    m = lambda d: pl.lambda_multiplier(d, 100.0, 1.1, 0.95, 1.05)
    assert m(0.0) == 1.05                      # flat wirelength: clamped growth
    assert m(100.0) == 1.0                     # rising by dref: unchanged
    assert m(50.0) == pytest.approx(1.1 ** 0.5, rel=1e-15)   # inside the clamp
    assert m(200.0) == 0.95                    # rising fast: clamped shrink
    assert m(-500.0) == 1.05


def test_lambda_schedule_follows_hpwl_in_placer():
    d = synth.tiny_1k(0)
    p = pl.Placer(d, pl.Params(tau_stop=-1.0, max_iters=6))
    p.run()
    h = p.history
    for k in range(2, 6):
        dh = h[k - 1][1] - h[k - 2][1]
        mu = pl.lambda_multiplier(dh, p.dref, 1.1, 0.95, 1.05)
        assert h[k][4] == pytest.approx(h[k - 1][4] * mu, rel=1e-14)
    assert h[1][4] > 0 and h[0][4] == 0.0


def test_backtrack_decision_special_cases():
    assert not pl.backtrack(0.1, 1.0, 0, 0)           # off
    assert pl.backtrack(0.1, 1.0, 0, 1)
    assert not pl.backtrack(0.1, 1.0, 1, 1)           # cap reached
    assert not pl.backtrack(0.95, 1.0, 0, 3)          # exactly at the ratio: accept
    assert pl.backtrack(0.95 - 1e-12, 1.0, 0, 3)
    assert not pl.backtrack(2.0, 1.0, 0, 3)           # longer estimates never reject


def test_backtracking_on_a_quadratic_redoes_the_first_step_once():
    # f = c/2 |x|^2, g = c x: every step-length estimate is 1/c exactly.  A
    # first step of 3/c is too long; the estimate at the point it reaches
    # rejects it, and the redone step of 1/c lands on the minimum.
    c = 7.0
    v0 = (np.array([1.0, -2.0, 0.5]),)
    u, v, a, alpha = v0, v0, 1.0, 3.0 / c
    g = (c * v[0],)
    u1, v1, a1 = pl.nesterov_update(v, u, g, a, alpha, _noclamp)
    g1 = (c * v1[0],)
    alpha_hat = pl.lipschitz_step(v1, v, g1, g, alpha)
    assert alpha_hat == pytest.approx(1.0 / c, rel=1e-14)
    assert pl.backtrack(alpha_hat, alpha, 0, 4)
    u1, v1, a1 = pl.nesterov_update(v, u, g, a, alpha_hat, _noclamp)
    np.testing.assert_allclose(u1[0], 0.0, atol=1e-15)
    np.testing.assert_allclose(v1[0], 0.0, atol=1e-15)   # a_0 = 1: no momentum yet


def test_placer_backtracking_invariants():
    d = synth.tiny_1k(0)
    base = pl.Placer(d, pl.Params(tau_stop=-1.0, max_iters=120))
    base.run(120)
    off = pl.Placer(d, pl.Params(tau_stop=-1.0, max_iters=120, max_backtracks=0))
    off.run(120)
    assert off.history == base.history and off.n_back_total == 0
    on = pl.Placer(d, pl.Params(tau_stop=-1.0, max_iters=120, max_backtracks=2))
    alphas, backs = [], []
    for _ in range(200):
        k, nb = on.k, on.n_back
        if not on.step():
            break
        alphas.append((k, on.k, on.alpha, nb, on.n_back))
    assert on.evals == on.k + on.n_back_total and on.n_back_total > 0
    for (k0, k1, a, nb0, nb1), (k0n, k1n, an, _, nbn) in zip(alphas, alphas[1:]):
        if k1n == k1 + 1 and k1 >= 1:
            # accepted: its estimate passed the test, or the cap was reached
            assert an >= 0.95 * a or nb1 == 2
        if k1n == k1:
            # a redone step: shorter, counted, at most twice in a row
            assert an < 0.95 * a and nbn == nb1 + 1 <= 2


def _hand_design():
    """Four movable cells and one fixed pad on an 8 x 8 die with 2 x 2 bins of
    4 x 4; every movable cell lies inside one bin, and every net has two pins.

    cell  corner   size     bin     pins
    0     (1, 1)   1 x 1    (0, 0)  2 (nets A, B)
    1     (5, 1)   2 x 1    (1, 0)  1 (net A)
    2     (1, 4)   1 x 3    (0, 1)  0
    3     (5, 5)   .5 x .5  (1, 1)  0
    4     (6, 6)   1 x 1    (1, 1)  fixed pad, 1 (net B)

    Net A: cell 0 at offset (.5, .5), cell 1 at (1, .5): pins (1.5, 1.5) and
    (6, 1.5).  Net B: cell 0 at (.5, .5), pad at (.5, .5): pins (1.5, 1.5) and
    (6.5, 6.5)."""
    f32 = lambda v: np.array(v, np.float32)
    return synth.Design(
        name="hand", n_movable=4,
        w=f32([1, 2, 1, 0.5, 1]), h=f32([1, 1, 3, 0.5, 1]),
        x=f32([1, 5, 1, 5, 6]), y=f32([1, 1, 4, 5, 6]),
        net_ptr=np.array([0, 2, 4], np.int32), pin_cell=np.array([0, 1, 0, 4], np.int32),
        pin_dx=f32([0.5, 1.0, 0.5, 0.5]), pin_dy=f32([0.5, 0.5, 0.5, 0.5]),
        die=(0.0, 0.0, 8.0, 8.0), nx=2, ny=2, target_density=1.0)


@pytest.mark.parametrize("kappa", [1.0, 4.0])
def test_first_step_composition_worked_by_hand(kappa):
    """The placer's first iteration assembled from quantities worked out in
    closed form, none of them through the oracle's own WA, density or Poisson
    code: the two-pin WA gradient d tanh(d / 2g) differentiated, the 2 x 2
    cosine series of the field written out term by term, the gather of a cell
    inside one bin (-area E_b), then lambda_0, the preconditioner
    max(1, pins_i + lambda area_i), alpha_0 and the first Nesterov step.  A
    preconditioner that counted the pad's pin, dropped lambda area_i or the
    floor at 1, or a step length normalised over n instead of 2n coordinates,
    fails here.  With kappa != 1, cell 2 is a movable macro and its charge in
    the preconditioner is weighted by kappa."""
    d = _hand_design()
    if kappa != 1.0:
        d.is_macro = np.array([0, 0, 1, 0, 0], np.uint8)
    eta, alpha0 = 0.25, 0.05
    p = pl.Placer(d, pl.Params(tau_stop=-1.0, max_iters=10, lambda_eta=eta, alpha0=alpha0,
                               macro_precond=kappa))
    x0, y0 = p.vx.copy(), p.vy.copy()
    assert p.step()

    # gamma_0 from tau_{-1} = 0 (no bin holds more than it may): w_bin = 4
    w_bin = 4.0
    gamma = 4.0 * w_bin * 10.0 ** (-11.0 / 9.0)
    assert p.history[0][3] == pytest.approx(gamma, rel=1e-14)
    assert p.history[0][2] == 0.0

    # WA gradient of a two-pin net along one axis, pins a < b, d = b - a:
    # dWL/db = tanh(d/2g) + (d/2g) sech^2(d/2g) = -dWL/da
    def fp(dist):
        z = dist / (2.0 * gamma)
        return math.tanh(z) + z / math.cosh(z) ** 2
    gwl_x = np.array([-fp(4.5) - fp(5.0), fp(4.5), 0.0, 0.0])
    gwl_y = np.array([-fp(5.0), 0.0, 0.0, 0.0])   # net A is flat in y

    # rho = (M + t F) / A_bin per bin (x-major), A_bin = 16
    r00, r10, r01, r11 = 1.0 / 16, 2.0 / 16, 3.0 / 16, (0.25 + 1.0) / 16
    s = math.sqrt(0.5)               # cos and sin of pi/4; cos(3 pi/4) = -s
    w1 = math.pi / 8.0               # pi u / (M h) for u = 1, M = 2, h = 4
    a10 = 0.5 * s * ((r00 + r01) - (r10 + r11))
    a01 = 0.5 * s * ((r00 + r10) - (r01 + r11))
    a11 = 0.5 * (r00 - r01 - r10 + r11)
    # Ex = a10/w1 sin(w1 X) + a11 w1/(2 w1^2) sin(w1 X) cos(w1 Y); sin(w1 X) = s
    # at both bin centres, cos(w1 Y) = +s (y = 0) or -s (y = 1)
    ex = {(ix, iy): s * a10 / w1 + s * (s if iy == 0 else -s) * a11 / (2 * w1)
          for ix in (0, 1) for iy in (0, 1)}
    ey = {(ix, iy): s * a01 / w1 + s * (s if ix == 0 else -s) * a11 / (2 * w1)
          for ix in (0, 1) for iy in (0, 1)}
    bins = [(0, 0), (1, 0), (0, 1), (1, 1)]
    area = np.array([1.0, 2.0, 3.0, 0.25])
    gd_x = np.array([-area[i] * ex[b] for i, b in enumerate(bins)])
    gd_y = np.array([-area[i] * ey[b] for i, b in enumerate(bins)])

    lam = eta * (np.abs(gwl_x).sum() + np.abs(gwl_y).sum()) / (np.abs(gd_x).sum() + np.abs(gd_y).sum())
    pins = np.array([2.0, 1.0, 0.0, 0.0])
    P = np.maximum(1.0, pins + lam * area * np.array([1.0, 1.0, kappa, 1.0]))
    assert P[3] == 1.0 and P[2] > 1.0 and P[0] > pins[0]   # every branch of the preconditioner
    gx = (gwl_x + lam * gd_x) / P
    gy = (gwl_y + lam * gd_y) / P
    alpha = alpha0 * w_bin / math.sqrt((np.sum(gx ** 2) + np.sum(gy ** 2)) / (2 * 4))
    ux = np.clip(x0 - alpha * gx, 0.0, 8.0 - np.array([1, 2, 1, 0.5]))
    uy = np.clip(y0 - alpha * gy, 0.0, 8.0 - np.array([1, 1, 3, 0.5]))

    assert p.lam == pytest.approx(lam, rel=1e-12)
    assert p.alpha == pytest.approx(alpha, rel=1e-12)
    np.testing.assert_allclose(p.gpx, gx, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(p.gpy, gy, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(p.ux, ux, rtol=1e-13, atol=0)
    np.testing.assert_allclose(p.uy, uy, rtol=1e-13, atol=0)
    # a_0 = 1: no momentum on the first step, v_1 = u_1; a_1 = golden ratio
    np.testing.assert_allclose(p.vx, ux, rtol=1e-13, atol=0)
    np.testing.assert_allclose(p.vy, uy, rtol=1e-13, atol=0)
    assert p.a == pytest.approx((1 + math.sqrt(5)) / 2, rel=1e-15)
    np.testing.assert_array_equal(p.vpx, x0)
    assert p.k == 1
