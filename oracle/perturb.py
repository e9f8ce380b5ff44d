"""Shuffle and Shuffle (all) perturbations (Algorithm 1; Section 4.2), with
SplitMix64 as the random source.

Test infrastructure only (see ``oracle/__init__.py``).

Section 4.2: Shuffle picks a fraction p of the macros at random (Shuffle
(all): of all the cells) and permutes their locations among themselves;
the experiments use p = 50%.  It does not fix the count rounding, what a
location is for cells of different sizes, or the random source.  Reading:

* Candidates: movable macros (Shuffle) or all movable cells (Shuffle (all)).
  Fixed cells never move.
* Every cell i draws a key r_i = the (i+1)-th output of SplitMix64 started
  from state ``seed`` (Steele, Lea and Flood, OOPSLA 2014).
* k = floor(p * n_candidates + 1/2) candidates with the smallest (r_i, i) are
  selected.
* Location = cell centre.  Taking the selected cells in increasing index order
  s_0 < s_1 < ... and in increasing key order t_0, t_1, ..., cell t_j receives
  the centre of cell s_j (centres before the shuffle), i.e. its new lower-left
  corner is centre(s_j) - size(t_j)/2, then clamped into the die.  Unselected
  cells are unchanged.
"""
from __future__ import annotations

import numpy as np

MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(state, n):
    """First n outputs of SplitMix64 from the given 64-bit state."""
    out = []
    s = state & MASK
    for _ in range(n):
        s = (s + GOLDEN) & MASK
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out.append(z ^ (z >> 31))
    return out


def select_and_permute(candidates, p, seed, n_cells):
    """Returns (receivers, donors): receiver t_j takes donor s_j's centre."""
    keys = splitmix64(seed, n_cells)
    cand = [int(i) for i in candidates]
    k = int(np.floor(float(np.float32(p)) * len(cand) + 0.5))
    k = max(0, min(k, len(cand)))
    by_key = sorted(cand, key=lambda i: (keys[i], i))[:k]
    by_index = sorted(by_key)
    return np.array(by_key, np.int64), np.array(by_index, np.int64)


def shuffle(x, y, w, h, candidates, p, seed, die):
    """Apply the Shuffle operator; returns new arrays of the input dtype
    (float32 or float64), computed in float64 and rounded once."""
    xl, yl, xh, yh = (float(v) for v in die)
    x = np.array(x, copy=True)
    y = np.array(y, copy=True)
    recv, donor = select_and_permute(candidates, p, seed, x.shape[0])
    if recv.size == 0:
        return x, y
    w64 = np.asarray(w, np.float64); h64 = np.asarray(h, np.float64)
    cx = x[donor].astype(np.float64) + 0.5 * w64[donor]
    cy = y[donor].astype(np.float64) + 0.5 * h64[donor]
    nx_ = cx - 0.5 * w64[recv]
    ny_ = cy - 0.5 * h64[recv]
    nx_ = np.maximum(xl, np.minimum(nx_, xh - w64[recv]))
    ny_ = np.maximum(yl, np.minimum(ny_, yh - h64[recv]))
    x[recv] = nx_.astype(x.dtype)
    y[recv] = ny_.astype(y.dtype)
    return x, y
