"""The electrostatic global-placement iteration (Eq. 2 minimised by Nesterov's
method with a Lipschitz step estimate), float64.

Test infrastructure only (see ``oracle/__init__.py``).

Algorithm 1 runs a DREAMPlace global placement to convergence in every
round; Eq. 2 is the objective sum_e WL_e + lambda D, with lambda small
at the start (Section 3.1).  The optimiser, the schedules and the stop test are
cited (ePlace, "... Nesterov's method") but not restated.  The reading below is
the one the CUDA library implements; every constant is a field of ``Params``.

Iteration k at reference point v_k (movable lower-left corners):

    gamma_k = gamma_base * w_bin * 10^((20/9) tau_{k-1} - 11/9)
    WL, gWL  = weighted-average wirelength and gradient at v_k (Eq. 3)
    M_k, tau_k = density map and overflow at v_k; stop here if tau_k <= tau_stop
    rho -> (psi, E); gD = field gather at v_k
    k == 0:  lambda = eta * |gWL|_1 / |gD|_1
    P_i = max(1, pins_i + lambda * k_i * area_i)  (k_i = macro_precond for a
                                                   movable macro, 1 otherwise)
    g_k = (gWL + lambda gD) / P
    alpha_k = alpha0 * w_bin / rms(g_0)                       (k == 0)
            = |v_k - v_{k-1}|_2 / |g_k - g_{k-1}|_2           (k >= 1)
    u_{k+1} = clamp(v_k - alpha_k g_k)
    a_{k+1} = (1 + sqrt(4 a_k^2 + 1)) / 2
    v_{k+1} = clamp(u_{k+1} + (a_k - 1)/a_{k+1} (u_{k+1} - u_k))
    k >= 1:  lambda *= clamp(mu_base^(1 - (HPWL_k - HPWL_{k-1}) / dref), mu_lo, mu_hi)

with a_0 = 1, u_0 = v_0 = the start, tau_{-1} = tau(v_0),
dref = hpwl_ref * n_nets * w_bin, w_bin = sqrt(bin_w * bin_h), and clamp
keeping each cell inside the die (x in [xl, xh - w]).

Optional backtracking (``max_backtracks`` > 0; the step-length prediction
with backtracking of ePlace's Nesterov method, which the paper cites but does
not restate).  At k >= 1 the estimate alpha_k above is also a test of the
step that led to v_k.  If alpha_k < 0.95 alpha_{k-1}, that step was too long.
At most ``max_backtracks`` times in a row, v_k is rejected:
* alpha_{k-1} := alpha_k;
* u_k and v_k are recomputed from v_{k-1}, u_{k-1}, g_{k-1}, a_{k-1};
* v_k is evaluated again.
lambda, gamma, the HPWL and overflow references and k advance only when v_k
is accepted.  The overflow stop test applies at every evaluated point.

Optional density stretching (``stretch``; oracle.density): the field and the
density gradient come from the stretched cells; the overflow, the stop test
and gamma keep the exact unstretched map.

Optional filler cells (``fillers``; oracle.fillers): pinless movable cells
appended after the real movable ones in the optimiser's vectors (positions,
gradients, preconditioner, every norm).  They enter the density that drives
the field and the density gradient, never the HPWL, the WA model or the
overflow.  A reset from new movable positions keeps the fillers where they
are.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import density as dens
from . import fillers as fil
from . import poisson as pois
from . import wirelength as wlm


def lipschitz_step(v, v_prev, g, g_prev, alpha_prev):
    """Inverse-Lipschitz step estimate |v - v_prev|_2 / |g - g_prev|_2 over
    all coordinates; keeps the previous step when the gradients coincide."""
    num = math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(v, v_prev)))
    den = math.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(g, g_prev)))
    return num / den if den > 0 else alpha_prev


def nesterov_update(v, u, g, a, alpha, clamp):
    """One Nesterov step from reference point v with major point u:
    u' = clamp(v - alpha g), a' = (1 + sqrt(4a^2 + 1))/2,
    v' = clamp(u' + (a - 1)/a' (u' - u)).  v, u, g are tuples of arrays."""
    u_new = clamp(*[vi - alpha * gi for vi, gi in zip(v, g)])
    a_new = (1.0 + math.sqrt(4.0 * a * a + 1.0)) / 2.0
    coef = (a - 1.0) / a_new
    v_new = clamp(*[un + coef * (un - uo) for un, uo in zip(u_new, u)])
    return u_new, v_new, a_new


BACKTRACK_RATIO = 0.95


def backtrack(alpha_hat, alpha_used, n_back, max_back, ratio=BACKTRACK_RATIO):
    """True when the step of length alpha_used that led to the current point
    is to be redone with alpha_hat: the step length estimated at the point
    is below ratio * alpha_used, and fewer than max_back steps have been
    redone in a row."""
    return max_back > 0 and n_back < max_back and alpha_hat < ratio * alpha_used


def lambda_multiplier(d_hpwl, dref, mu_base, mu_lo, mu_hi):
    """Density-weight growth factor mu = clamp(mu_base^(1 - dHPWL/dref),
    mu_lo, mu_hi): lambda grows fastest while the wirelength is flat and
    shrinks when the wirelength rises faster than dref per iteration."""
    mu = mu_base ** (1.0 - d_hpwl / dref)
    return min(max(mu, mu_lo), mu_hi)


@dataclasses.dataclass
class Params:
    gamma_base: float = 4.0
    lambda_eta: float = 1e-3
    alpha0: float = 0.05
    hpwl_ref: float = 0.3
    mu_base: float = 1.1
    mu_lo: float = 0.95
    mu_hi: float = 1.05
    tau_stop: float = 0.07
    max_iters: int = 1000
    constant_gamma: float = 0.0  # > 0: use this gamma every iteration
    max_backtracks: int = 0      # > 0: redo a too-long step at most this often in a row
    stretch: bool = False        # ePlace density stretching for the field
    fillers: bool = False        # ePlace filler cells in the whitespace
    macro_precond: float = 1.0   # weight of a movable macro's charge in its preconditioner


class Placer:
    """FP64 placer state for one design."""

    def __init__(self, design, params: Params | None = None):
        self.d = design
        self.p = params or Params()
        d = design
        self.n = d.n_movable
        self.w = d.w.astype(np.float64)
        self.h = d.h.astype(np.float64)
        total_area = float(np.sum(self.w * self.h))
        self.F = dens.frac_bits(d.die, total_area)
        self.g = dens.Grid(d.die, d.nx, d.ny, self.F)
        self.t = float(np.float32(d.target_density))
        self.W = dens.quantize(d.w, self.F)
        self.H = dens.quantize(d.h, self.F)
        fx = dens.quantize(d.x[self.n:], self.F)
        fy = dens.quantize(d.y[self.n:], self.F)
        self.Fmap = dens.overlap_map(fx, fy, self.W[self.n:], self.H[self.n:], self.g)
        self.mov_area_q = int(np.sum(self.W[:self.n] * self.H[:self.n]))
        self.fixed_x = d.x[self.n:].astype(np.float64)
        self.fixed_y = d.y[self.n:].astype(np.float64)
        pc = d.pin_cell.astype(np.int64)
        pins = np.bincount(pc[pc < self.n], minlength=self.n).astype(np.float64)
        # the optimiser's cells: the movable cells, then the fillers
        self.nf = 0
        fx0 = fy0 = np.zeros(0)
        wo, ho = self.w[:self.n], self.h[:self.n]
        Wo, Ho = self.W[:self.n], self.H[:self.n]
        if self.p.fillers:
            Wf, Hf = fil.size(self.W, self.H, self.n, d.is_macro)
            self.nf = fil.count(d.die, self.t, int(np.sum(self.Fmap)), self.mov_area_q, self.F,
                                Wf, Hf)
            wf, hf = Wf * 2.0 ** -self.F, Hf * 2.0 ** -self.F
            fx0, fy0 = fil.start(self.nf, d.die, wf, hf)
            wo = np.concatenate([wo, np.full(self.nf, wf)])
            ho = np.concatenate([ho, np.full(self.nf, hf)])
            Wo = np.concatenate([Wo, np.full(self.nf, Wf, np.int64)])
            Ho = np.concatenate([Ho, np.full(self.nf, Hf, np.int64)])
        self.wo, self.ho, self.Wo, self.Ho = wo, ho, Wo, Ho
        self.pins = np.concatenate([pins, np.zeros(self.nf)])
        # the charge term of the preconditioner, a movable macro's weighted
        kappa = np.ones(self.n + self.nf)
        if d.is_macro is not None:
            kappa[:self.n][np.asarray(d.is_macro[:self.n]) != 0] = self.p.macro_precond
        self.area = wo * ho * kappa
        self.w_bin = math.sqrt(self.g.bin_w * self.g.bin_h)
        self.dref = self.p.hpwl_ref * d.n_nets * self.w_bin
        self.reset(np.concatenate([d.x[:self.n], fx0]), np.concatenate([d.y[:self.n], fy0]))

    # -- helpers -----------------------------------------------------------
    def clamp(self, x, y):
        xl, yl, xh, yh = self.g.die
        x = np.maximum(xl, np.minimum(x, xh - self.wo))
        y = np.maximum(yl, np.minimum(y, yh - self.ho))
        return x, y

    def full(self, x, y):
        """All real cells (movable, then fixed) from optimiser or movable
        vectors; fillers are not cells of the design."""
        n = self.n
        return (np.concatenate([x[:n], self.fixed_x]), np.concatenate([y[:n], self.fixed_y]))

    def density_map(self, x, y):
        """Map of the real movable cells: the overflow's."""
        X = dens.quantize(x[:self.n], self.F)
        Y = dens.quantize(y[:self.n], self.F)
        return dens.overlap_map(X, Y, self.W[:self.n], self.H[:self.n], self.g)

    def field_map(self, x, y):
        """Map that drives the field: the movable cells and the fillers
        (stretched when ``stretch`` is set)."""
        X = dens.quantize(x, self.F)
        Y = dens.quantize(y, self.F)
        if self.p.stretch:
            Xs, Ys, Ws, Hs, R, _ = dens.stretched(X, Y, self.Wo, self.Ho, self.g)
            return dens.overlap_map_scaled(Xs, Ys, Ws, Hs, R, self.g)
        return dens.overlap_map(X, Y, self.Wo, self.Ho, self.g)

    def stretched_map(self, x, y):
        """Map of the stretched cells (oracle.density), which drives the field
        when ``stretch`` is set."""
        X = dens.quantize(x, self.F)
        Y = dens.quantize(y, self.F)
        Xs, Ys, Ws, Hs, R, _ = dens.stretched(X, Y, self.Wo, self.Ho, self.g)
        return dens.overlap_map_scaled(Xs, Ys, Ws, Hs, R, self.g)

    def overflow(self, M):
        return dens.overflow(M, self.Fmap, self.t, self.g, self.mov_area_q)

    def hpwl(self, x, y):
        fx, fy = self.full(x, y)
        d = self.d
        return wlm.hpwl(d.net_ptr, d.pin_cell, d.pin_dx, d.pin_dy, fx, fy)

    def gamma(self, tau):
        if self.p.constant_gamma > 0:
            return self.p.constant_gamma
        return self.p.gamma_base * self.w_bin * 10.0 ** ((20.0 / 9.0) * tau - 11.0 / 9.0)

    def field(self, M):
        rho = dens.bin_density(M, self.Fmap, self.t, self.g)
        return pois.poisson(rho, self.g.bin_w, self.g.bin_h)

    def wirelength(self, x, y, gamma):
        """WA value and gradient over the optimiser's cells (fillers: 0)."""
        fx, fy = self.full(x, y)
        d = self.d
        wl, gx, gy = wlm.wa_wirelength(d.net_ptr, d.pin_cell, d.pin_dx, d.pin_dy, fx, fy,
                                       gamma, self.n)
        z = np.zeros(self.nf)
        return wl, np.concatenate([gx, z]), np.concatenate([gy, z])

    def density_grad(self, x, y, ex, ey):
        X = dens.quantize(x, self.F)
        Y = dens.quantize(y, self.F)
        W, H = self.Wo, self.Ho
        if self.p.stretch:
            X, Y, W, H, _, wgt = dens.stretched(X, Y, W, H, self.g)
            gx, gy = dens.field_gather(X, Y, W, H, self.g, ex, ey)
            return wgt * gx, wgt * gy
        return dens.field_gather(X, Y, W, H, self.g, ex, ey)

    # -- optimiser ------------------------------------------------------------
    def reset(self, x, y):
        """Restart the optimiser from movable positions (x, y).  Given only
        the real movable cells, the fillers stay where they are."""
        x = np.asarray(x, np.float64).copy()
        y = np.asarray(y, np.float64).copy()
        if x.shape[0] == self.n and self.nf:
            x = np.concatenate([x, self.vx[self.n:]])
            y = np.concatenate([y, self.vy[self.n:]])
        x, y = self.clamp(x, y)
        self.ux, self.uy = x.copy(), y.copy()
        self.vx, self.vy = x.copy(), y.copy()
        self.a = 1.0
        self.k = 0
        self.lam = 0.0
        self.alpha = 0.0
        self.vpx = self.vpy = self.gpx = self.gpy = None
        self.upx = self.upy = None
        self.a_prev = 1.0
        self.n_back = 0          # steps redone in a row
        self.n_back_total = 0
        self.evals = 0
        self.hpwl_prev = 0.0
        self.tau_prev = self.overflow(self.density_map(x, y))
        self.tau = self.tau_prev
        self.converged = False
        self.stopped = False
        self.history = []

    def step(self):
        """One evaluation at the current point: an iteration, or with
        backtracking a redone step.  Returns False once stopped."""
        if self.stopped:
            return False
        if self.k >= self.p.max_iters:
            self.stopped = True
            return False
        p = self.p
        self.evals += 1
        gamma = self.gamma(self.tau_prev)
        vx, vy = self.vx, self.vy
        wl, gwx, gwy = self.wirelength(vx, vy, gamma)
        hp = self.hpwl(vx, vy)
        M = self.density_map(vx, vy)
        tau = self.overflow(M)
        self.tau = tau
        self.history.append((self.k, hp, tau, gamma, self.lam))
        if tau <= p.tau_stop:
            self.converged = self.stopped = True
            return False
        _, ex, ey = self.field(self.field_map(vx, vy) if (p.stretch or self.nf) else M)
        gdx, gdy = self.density_grad(vx, vy, ex, ey)
        if self.k == 0:
            n1 = np.sum(np.abs(gwx)) + np.sum(np.abs(gwy))
            d1 = np.sum(np.abs(gdx)) + np.sum(np.abs(gdy))
            self.lam = p.lambda_eta * n1 / d1 if d1 > 0 else p.lambda_eta
        lam = self.lam
        prec = np.maximum(1.0, self.pins + lam * self.area)
        gx = (gwx + lam * gdx) / prec
        gy = (gwy + lam * gdy) / prec
        if self.k == 0:
            gn = math.sqrt((np.sum(gx * gx) + np.sum(gy * gy)) / (2 * (self.n + self.nf)))
            alpha = p.alpha0 * self.w_bin / gn if gn > 0 else 0.0
        else:
            alpha = lipschitz_step((vx, vy), (self.vpx, self.vpy), (gx, gy),
                                   (self.gpx, self.gpy), self.alpha)
            if backtrack(alpha, self.alpha, self.n_back, p.max_backtracks):
                # redo the step that led here, shorter, from the saved state
                self.n_back += 1
                self.n_back_total += 1
                self.alpha = alpha
                (self.ux, self.uy), (self.vx, self.vy), _ = nesterov_update(
                    (self.vpx, self.vpy), (self.upx, self.upy), (self.gpx, self.gpy),
                    self.a_prev, alpha, self.clamp)
                return True
            self.n_back = 0
        self.alpha = alpha
        (nux, nuy), (nvx, nvy), a_new = nesterov_update(
            (vx, vy), (self.ux, self.uy), (gx, gy), self.a, alpha, self.clamp)
        if self.k >= 1:
            self.lam = lam * lambda_multiplier(hp - self.hpwl_prev, self.dref,
                                               p.mu_base, p.mu_lo, p.mu_hi)
        self.hpwl_prev = hp
        self.tau_prev = tau
        self.vpx, self.vpy, self.gpx, self.gpy = vx, vy, gx, gy
        self.upx, self.upy, self.a_prev = self.ux, self.uy, self.a
        self.ux, self.uy = nux, nuy
        self.vx, self.vy = nvx, nvy
        self.a = a_new
        self.k += 1
        return True

    def run(self, n_iters=None):
        n = self.p.max_iters if n_iters is None else n_iters
        for _ in range(n):
            if not self.step():
                break
        return self

    def positions(self):
        """Current solution (the reference point v) for all cells."""
        return self.full(self.vx, self.vy)
