"""Pins of the oracle's SplitMix64 and Shuffle operators (Algorithm 1)."""
import os
from collections import Counter

import numpy as np
import pytest

from oracle import hybro
from oracle import perturb as pt
from paper_2402_18311_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def test_splitmix64_reference_outputs():
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        seed, *outs = line.split()
        ref = [int(o, 16) for o in outs]
        assert pt.splitmix64(int(seed), len(ref)) == ref


def test_selection_is_k_smallest_keys():
    keys = pt.splitmix64(42, 50)
    cand = list(range(3, 47, 2))
    recv, donor = pt.select_and_permute(cand, 0.5, 42, 50)
    k = int(np.floor(0.5 * len(cand) + 0.5))
    assert len(recv) == k
    brute = sorted(cand, key=lambda i: keys[i])[:k]   # keys are distinct here
    assert recv.tolist() == brute
    assert donor.tolist() == sorted(brute)


def test_shuffle_moves_only_selected_and_preserves_centres():
    d = synth.tiny_1k(0)
    rng = np.random.default_rng(0)
    x = (rng.random(d.n_cells) * 200).astype(np.float32)
    y = (rng.random(d.n_cells) * 200).astype(np.float32)
    x[d.n_movable:], y[d.n_movable:] = d.x[d.n_movable:], d.y[d.n_movable:]
    cand = hybro.candidates(d, hybro.SHUFFLE_ALL)
    nx_, ny_ = pt.shuffle(x, y, d.w, d.h, cand, 0.5, 7, d.die)
    recv, donor = pt.select_and_permute(cand, 0.5, 7, d.n_cells)
    moved = np.zeros(d.n_cells, bool)
    moved[recv] = True
    assert np.array_equal(nx_[~moved], x[~moved]) and np.array_equal(ny_[~moved], y[~moved])
    assert moved.sum() == 500
    # no clamp is active here (all far from the edges): the centres are permuted
    c_old = sorted(zip((x[recv] + 0.5 * d.w[recv]).astype(np.float64),
                       (y[recv] + 0.5 * d.h[recv]).astype(np.float64)))
    c_new = sorted(zip(nx_[recv].astype(np.float64) + 0.5 * d.w[recv],
                       ny_[recv].astype(np.float64) + 0.5 * d.h[recv]))
    np.testing.assert_allclose(np.array(c_old), np.array(c_new), atol=1e-4)


def test_shuffle_macro_is_noop_without_movable_macros():
    d = synth.tiny_1k(0)
    cand = hybro.candidates(d, hybro.SHUFFLE_MACRO)
    assert cand.size == 0
    nx_, ny_ = pt.shuffle(d.x, d.y, d.w, d.h, cand, 0.5, 1, d.die)
    assert np.array_equal(nx_, d.x) and np.array_equal(ny_, d.y)


def test_shuffle_clamps_into_die():
    die = (0, 0, 10, 10)
    x = np.array([0.0, 8.0], np.float32); y = np.array([0.0, 0.0], np.float32)
    w = np.array([1.0, 2.0], np.float32); h = np.array([1.0, 1.0], np.float32)
    for seed in range(20):
        nx_, ny_ = pt.shuffle(x, y, w, h, [0, 1], 1.0, seed, die)
        assert np.all(nx_ >= 0) and np.all(nx_ + w <= 10)


def test_permutations_are_uniform():
    # three candidates, p = 1: all 6 permutations about equally often
    counts = Counter()
    for seed in range(3000):
        recv, donor = pt.select_and_permute([0, 1, 2], 1.0, seed, 3)
        counts[tuple(recv.tolist())] += 1
    assert len(counts) == 6
    exp = 500.0
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    assert chi2 < 20.5  # 5 dof, p = 0.001


def test_selection_is_uniform():
    hits = np.zeros(10)
    for seed in range(2000):
        recv, _ = pt.select_and_permute(range(10), 0.3, seed, 10)
        hits[recv] += 1
    np.testing.assert_allclose(hits / 2000, 0.3, atol=0.045)


def test_count_rounding():
    for n, p, k in [(10, 0.5, 5), (5, 0.5, 3), (3, 0.5, 2), (1, 0.5, 1), (7, 0.0, 0), (4, 1.0, 4)]:
        recv, _ = pt.select_and_permute(range(n), p, 0, n)
        assert len(recv) == k
