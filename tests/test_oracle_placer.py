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
