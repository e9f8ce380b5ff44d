"""Pins of the oracle's Hybro loop and best-solution selection (Algorithm 1)."""
import numpy as np

from oracle import hybro
from oracle import placer as pl
from paper_2402_18311_gb300 import synth


def test_selection_order():
    # feasible beats infeasible; then HPWL; then overflow; then round
    res = [(100.0, 0.2), (120.0, 0.05), (110.0, 0.08), (110.0, 0.06)]
    assert hybro.select_best(res, 0.1) == 3
    assert hybro.select_best([(5.0, 0.5), (9.0, 0.5)], 0.1) == 0
    assert hybro.select_best([(5.0, 0.05), (5.0, 0.05)], 0.1) == 0


def test_round_trip_two_rounds():
    d = synth.tiny_1k(0)
    best, rounds = hybro.run(d, pl.Params(tau_stop=-1.0, max_iters=60), n_rounds=1,
                             op=hybro.SHUFFLE_ALL, p=0.5, seed=0)
    assert len(rounds) == 2
    keys = [hybro.selection_key(r[0], r[1], i, 0.1) for i, r in enumerate(rounds)]
    assert best == int(np.argmin([0 if k == min(keys) else 1 for k in keys]))
    # round 1 starts from a shuffled copy of round 0's result, so it differs
    assert not np.array_equal(rounds[0][2], rounds[1][2])


def test_round_records_measure_the_same_placement():
    # each round's (HPWL, overflow) are both of the placement it returns
    # (Algorithm 1 keeps a solution and its measures together), also when the
    # placer stops at max_iters, one step after its last overflow evaluation
    from oracle import density as dens
    from oracle import wirelength as wl
    d = synth.tiny_1k(0)
    p = pl.Placer(d, pl.Params(tau_stop=-1.0, max_iters=40))
    best, rounds = hybro.run(d, pl.Params(tau_stop=-1.0, max_iters=40), n_rounds=1,
                             op=hybro.SHUFFLE_ALL, p=0.5, seed=3)
    n = d.n_movable
    for hp, tau, fx, fy in rounds:
        assert hp == wl.hpwl(d.net_ptr, d.pin_cell, d.pin_dx, d.pin_dy, fx, fy)
        M = dens.overlap_map(dens.quantize(fx[:n], p.F), dens.quantize(fy[:n], p.F),
                             p.W[:n], p.H[:n], p.g)
        assert tau == p.overflow(M)
