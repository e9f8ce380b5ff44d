"""Filler cells of the electrostatic density, float64 / int64.

Test infrastructure only (see ``oracle/__init__.py``).

The paper runs DREAMPlace as the global placer of Algorithm 1 and names the
density penalty of Eq. 2 only through ePlace.  ePlace adds filler cells:
movable cells without pins that take up the whitespace the target density
leaves, so that the density force holds the real cells together at the
target density instead of spreading them over the whole die.  Fillers are
not part of the placement: they take no part in Eq. 1 or in the overflow,
only in the density that drives the field.  The reading used here (and by
the CUDA library):

* size: the mean quantised width and height of the movable cells that are
  not macros, each rounded to the nearest multiple of 2^-F (ties to even);
* count: n_f = floor(max(0, t (A_die - A_fixed) - A_mov) / (w_f h_f)), with
  A_fixed the fixed cells' area inside the die and A_mov the movable cells'
  quantised area, all in float64 in that order;
* start: filler j's lower-left corner is
  (xl + u (xh - xl - w_f), yl + v (yh - yl - h_f)) rounded to float32, with
  u, v the (2j+1)-th and (2j+2)-th outputs of SplitMix64 from FILLER_SEED
  taken as (z >> 11) 2^-53;
* in the placer they are movable cells with zero pins: density gradient
  only, preconditioner max(1, lambda w_f h_f), and they count in the norms
  that set lambda_0 and the step lengths.
"""
from __future__ import annotations

import math

import numpy as np

from .perturb import splitmix64

FILLER_SEED = 0x46494C4C45525321  # "FILLERS!"


def size(Wq, Hq, n_movable, is_macro):
    """(W_f, H_f) in units of 2^-F: rint of the mean quantised width and
    height of the movable non-macro cells (ties to even)."""
    sel = np.arange(n_movable)
    if is_macro is not None:
        sel = sel[np.asarray(is_macro[:n_movable]) == 0]
    if sel.size == 0:
        return 0, 0
    n = int(sel.size)
    sw = int(np.sum(np.asarray(Wq, np.int64)[sel]))
    sh = int(np.sum(np.asarray(Hq, np.int64)[sel]))
    return max(1, int(round(float(sw) / n))), max(1, int(round(float(sh) / n)))


def count(die, t, fixed_area_q, mov_area_q, F, Wf, Hf):
    """Number of fillers: floor of the whitespace at target density t over one
    filler's area (float64, in the order stated in the module docstring)."""
    if Wf <= 0 or Hf <= 0:
        return 0
    xl, yl, xh, yh = (float(v) for v in die)
    s2 = 2.0 ** (-2 * F)
    a_die = (xh - xl) * (yh - yl)
    fill = float(t) * (a_die - float(fixed_area_q) * s2) - float(mov_area_q) * s2
    if not fill > 0.0:
        return 0
    wf, hf = Wf * 2.0 ** (-F), Hf * 2.0 ** (-F)
    return int(math.floor(fill / (wf * hf)))


def start(n_f, die, wf, hf, seed=FILLER_SEED):
    """Lower-left corners of the fillers (float32 arrays of length n_f)."""
    xl, yl, xh, yh = (float(v) for v in die)
    z = splitmix64(seed, 2 * n_f)
    u = np.array([(v >> 11) * 2.0 ** -53 for v in z[0::2]], np.float64)
    v = np.array([(q >> 11) * 2.0 ** -53 for q in z[1::2]], np.float64)
    x = (xl + u * ((xh - xl) - wf)).astype(np.float32)
    y = (yl + v * ((yh - yl) - hf)).astype(np.float32)
    return x, y
