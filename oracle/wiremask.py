"""WireMask perturbation (the perturbation step of Algorithm 1; Section 4.2),
float64.

Test infrastructure only (see ``oracle/__init__.py``).

Section 4.2 describes WireMask in one sentence.  It moves every macro, one
after another, to the grid position where the HPWL grows least, the wire
mask of the cited WireMask-BBO.  WireMask has no strength parameter and
draws no random numbers.  The paper leaves open:
* the macro order;
* the grid;
* which pins count;
* what a macro may not overlap;
* ties.

The reading used here:

* Macros: the movable cells flagged ``is_macro``.  They are taken in
  decreasing area w*h (exact in float64), ties by increasing index.
* Grid: the placement bins.  Candidate lower-left corners are
  X_i = fl32(xl + i*bw) for i in [0, nx), with bw = (xh - xl)/nx in float64,
  and likewise Y_j.  A candidate is inside the die when X_i + w <= xh and
  Y_j + h <= yh.
* Wire mask: the weighted HPWL (Eq. 1) of the macro's nets with the macro at
  the candidate.  Every other pin stays at its current position; macros
  moved earlier in the pass sit at their new places.  Over the design, this
  is the total HPWL up to a constant.  For one net with the other pins'
  extent [o-, o+] and the macro's own pin offsets [d-, d+], the x part at X
  is max(o+, X + d+) - min(o-, X + d-).  With no other pins,
  o+ = -inf and o- = +inf.  The mask is therefore separable,
  Fx(X_i) + Fy(Y_j).  Each axis sums w_e * (hi - lo) over the macro's nets
  in increasing net index.
* Obstacles: every fixed cell of positive area, and the macros already
  moved in this pass.  A candidate is blocked when its rectangle overlaps an
  obstacle with positive area.  Touching edges is allowed.
* Choice: the smallest (Fx + Fy, |X - x| + |Y - y|, j, i) among the
  candidates inside the die that are not blocked.  (x, y) is the macro's
  position before it moves.  With no such candidate the macro stays where it
  is.  Either way it becomes an obstacle for the macros after it.

Every comparison is on float64 values from a fixed sequence of correctly
rounded operations (each axis's mask summed over the macro's nets in
increasing net index, each extent and corner formed as written above), so
any implementation that evaluates these expressions in this order chooses
bit-identical positions; the brute-force pins in the tests check the choice
against the Eq. 1 HPWL itself.
"""
from __future__ import annotations

import numpy as np


def macro_order(w, h, is_macro, n_movable):
    """Movable macros by decreasing area, ties by increasing index."""
    w64 = np.asarray(w, np.float64)
    h64 = np.asarray(h, np.float64)
    mac = [i for i in range(int(n_movable)) if is_macro is not None and is_macro[i]]
    return sorted(mac, key=lambda i: (-(w64[i] * h64[i]), i))


def grid_corners(lo, hi, n):
    """Candidate corners fl32(lo + i * (hi - lo) / n), as float64."""
    b = (float(hi) - float(lo)) / n
    return (float(lo) + np.arange(n, dtype=np.float64) * b).astype(np.float32).astype(np.float64)


def nets_of(net_ptr, pin_cell, m):
    """Indices of the nets holding a pin of cell m, increasing."""
    net_ptr = np.asarray(net_ptr, np.int64)
    net_of_pin = np.repeat(np.arange(net_ptr.shape[0] - 1), np.diff(net_ptr))
    return np.unique(net_of_pin[np.asarray(pin_cell) == m]).tolist()


def axis_mask(corners, nets, net_ptr, pin_cell, pin_d, pos, m, net_w):
    """One axis of the wire mask of macro m: for every candidate corner c,
    sum over the macro's nets of w_e (max(o+, c + d+) - min(o-, c + d-))."""
    acc = np.zeros(corners.shape[0], np.float64)
    for e in nets:
        js = range(int(net_ptr[e]), int(net_ptr[e + 1]))
        own = [float(np.float64(pin_d[j])) for j in js if pin_cell[j] == m]
        other = [float(np.float64(pos[pin_cell[j]])) + float(np.float64(pin_d[j]))
                 for j in js if pin_cell[j] != m]
        o_hi = max(other) if other else -np.inf
        o_lo = min(other) if other else np.inf
        hi = np.maximum(o_hi, corners + max(own))
        lo = np.minimum(o_lo, corners + min(own))
        wn = 1.0 if net_w is None else float(np.float64(net_w[e]))
        acc = acc + wn * (hi - lo)
    return acc


def wiremask(x, y, w, h, net_ptr, pin_cell, pin_dx, pin_dy, n_movable, is_macro, die, nx, ny,
             net_w=None, trace=None):
    """Apply WireMask; returns new position arrays of the input dtype (float32
    or float64; the chosen corners are float32 values either way).

    ``trace``, when a list, receives for every macro a tuple
    (macro, fx, fy, chosen (i, j) or None): test hook only."""
    xl, yl, xh, yh = (float(v) for v in die)
    x = np.array(x, copy=True)
    y = np.array(y, copy=True)
    w64 = np.asarray(w, np.float64)
    h64 = np.asarray(h, np.float64)
    n_cells = x.shape[0]
    X = grid_corners(xl, xh, nx)
    Y = grid_corners(yl, yh, ny)
    obstacles = [i for i in range(int(n_movable), n_cells) if w64[i] > 0 and h64[i] > 0]
    for m in macro_order(w, h, is_macro, n_movable):
        nets = nets_of(net_ptr, pin_cell, m)
        fx = axis_mask(X, nets, net_ptr, pin_cell, pin_dx, x, m, net_w)
        fy = axis_mask(Y, nets, net_ptr, pin_cell, pin_dy, y, m, net_w)
        obj = fy[:, None] + fx[None, :]
        ok = (Y + h64[m] <= yh)[:, None] & (X + w64[m] <= xh)[None, :]
        for o in obstacles:
            ox, oy = float(x[o]), float(y[o])
            bx = (X < ox + w64[o]) & (ox < X + w64[m])
            by = (Y < oy + h64[o]) & (oy < Y + h64[m])
            ok &= ~(by[:, None] & bx[None, :])
        dist = np.abs(Y - float(y[m]))[:, None] + np.abs(X - float(x[m]))[None, :]
        # lexicographic minimum of (obj, dist, j, i) over the free candidates:
        # flat row-major index q = j nx + i orders (j, i)
        q = np.flatnonzero(ok)
        chosen = None
        if q.size:
            first = q[np.lexsort((q, dist.ravel()[q], obj.ravel()[q]))[0]]
            chosen = (int(first % nx), int(first // nx))
            x[m] = X[chosen[0]]
            y[m] = Y[chosen[1]]
        if trace is not None:
            trace.append((m, fx, fy, chosen))
        obstacles.append(m)
    return x, y
