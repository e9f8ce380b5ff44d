"""Hybro: alternate global placement and perturbation, keep the best result
(Algorithm 1; Section 4.1).

Test infrastructure only (see ``oracle/__init__.py``).

Reading of Algorithm 1 used here: round i places s_i until convergence (the
placer of ``oracle.placer``), records (HPWL, overflow), and, unless it is the
last round, perturbs the *current* result s_i (not the best) to start round
i+1.  Rounds 0..N place N+1 times.  The returned solution is the best by the
key (overflow above tau_target, HPWL, overflow, round): the paper keeps "the
best HPWL value"; feasibility first keeps an unspread placement from winning.
"""
from __future__ import annotations

import numpy as np

from . import perturb
from . import placer as pl
from . import wiremask

SHUFFLE_MACRO = 0
SHUFFLE_ALL = 1
WIREMASK = 2


def candidates(design, op):
    """Shuffle picks from the movable macros, Shuffle (all) from every
    movable cell."""
    n = design.n_movable
    if op == SHUFFLE_ALL:
        return np.arange(n)
    if design.is_macro is None:
        return np.zeros(0, np.int64)
    return np.nonzero(design.is_macro[:n])[0]


def selection_key(hpwl, tau, index, tau_target):
    return (0 if tau <= tau_target else 1, hpwl, tau, index)


def select_best(results, tau_target):
    """results: list of (hpwl, tau); returns the index of the best."""
    keys = [selection_key(h, t, i, tau_target) for i, (h, t) in enumerate(results)]
    return min(range(len(keys)), key=lambda i: keys[i])


def run(design, params: pl.Params, n_rounds, op=SHUFFLE_ALL, p=0.5, seed=0,
        tau_target=0.1, iters_per_round=None):
    """Returns (best_index, [(hpwl, tau, x, y) per round])."""
    placer = pl.Placer(design, params)
    n = design.n_movable
    cand = candidates(design, op)
    sx = design.x[:n].astype(np.float64)
    sy = design.y[:n].astype(np.float64)
    rounds = []
    for i in range(n_rounds + 1):
        placer.reset(sx, sy)
        placer.run(iters_per_round)
        fx, fy = placer.positions()
        # both measures of the round's result at the same placement s_i: the
        # placer's last overflow belongs to v_{k-1} when it stopped at max_iters
        hp = placer.hpwl(placer.vx, placer.vy)
        tau = placer.overflow(placer.density_map(placer.vx, placer.vy))
        rounds.append((hp, tau, fx.copy(), fy.copy()))
        if i < n_rounds and op == WIREMASK:
            nx_, ny_ = wiremask.wiremask(fx, fy, design.w, design.h, design.net_ptr,
                                         design.pin_cell, design.pin_dx, design.pin_dy, n,
                                         design.is_macro, design.die, design.nx, design.ny)
            sx, sy = nx_[:n], ny_[:n]
        elif i < n_rounds:
            nx_, ny_ = perturb.shuffle(fx, fy, design.w, design.h, cand, p,
                                       seed + i, design.die)
            sx, sy = nx_[:n], ny_[:n]
    best = select_best([(r[0], r[1]) for r in rounds], tau_target)
    return best, rounds
