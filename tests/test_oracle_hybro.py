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
