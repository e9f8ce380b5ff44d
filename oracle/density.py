"""Electrostatic density: exact overlap-area bin map, overflow, bin density and
the density-gradient field gather, float64 / int64.

Test infrastructure only (see ``oracle/__init__.py``).

The paper names the density D of Eq. 1 / Eq. 2 only through ePlace and
DREAMPlace (Sections 1 and 3.1).  The reading used here:

* Coordinates are quantised to fixed point, X = rint(x * 2^F) with ties to
  even; x is the float32 value and scaling by 2^F is exact, so the map is a
  pure integer function of the float32 positions.
* The movable map M_b is the sum over movable cells of the exact overlap area
  of the cell rectangle with bin b, in units of 2^-2F (int64).  The fixed map
  F_b is the same over fixed cells.  No small-cell stretching here; the
  optional stretching below keeps this map for the overflow.
* Overflow tau = sum_b max(0, M_b - t (A_b - F_b)) / (total movable area).
* Bin density rho_b = (M_b + t F_b) / A_b, t the target density.

Optional density stretching (ePlace's local smoothing, off by default):
* along each axis, a movable cell narrower than sqrt(2) bins widens to
  Ws = rint(sqrt(2) BW) about its centre, Xs = X - floor((Ws - W) / 2);
* its density is scaled by W H / (Ws Hs) so that its charge stays its
  area.  In the map this is the fixed-point scale R = floor(W H 2^31 /
  (Ws Hs)), each (cell, bin) term floor(ov R / 2^31);
* the stretched map drives the field and the density gradient; the
  overflow keeps the unstretched map.
"""
from __future__ import annotations

import math

import numpy as np


class Grid:
    """Bin grid over the die in fixed point.  All members are python ints
    except the float geometry."""

    def __init__(self, die, nx, ny, F):
        xl, yl, xh, yh = (float(v) for v in die)
        self.die = (xl, yl, xh, yh)
        self.nx, self.ny, self.F = int(nx), int(ny), int(F)
        s = 2.0 ** F
        self.bin_w = (xh - xl) / nx
        self.bin_h = (yh - yl) / ny
        vals = [xl * s, yl * s, self.bin_w * s, self.bin_h * s]
        if any(v != math.floor(v) for v in vals):
            raise ValueError("die origin and bin size must be multiples of 2^-F")
        self.XL, self.YL, self.BW, self.BH = (int(v) for v in vals)
        self.scale = s


def frac_bits(die, total_area):
    """Fixed-point fraction bits F: the largest F <= 24 with
    max(|coordinate|, die width, die height) * 2^F < 2^30 and
    total_area * 2^(2F) < 2^62."""
    xl, yl, xh, yh = (float(v) for v in die)
    ext = max(abs(xl), abs(yl), abs(xh), abs(yh), xh - xl, yh - yl)
    for F in range(24, -1, -1):
        if ext * 2.0 ** F < 2.0 ** 30 and total_area * 2.0 ** (2 * F) < 2.0 ** 62:
            return F
    raise ValueError("design does not fit the fixed-point range")


def quantize(v, F):
    """X = rint(v * 2^F), ties to even, as int64.  v is float32 or float64."""
    return np.rint(np.asarray(v, np.float64) * 2.0 ** F).astype(np.int64)


def _axis_overlap(lo, size, origin, step, k):
    """Overlap length of [lo, lo+size) with bin k = [origin + k step,
    origin + (k+1) step), clipped at 0 (integers)."""
    b0 = origin + k * step
    return np.maximum(0, np.minimum(lo + size, b0 + step) - np.maximum(lo, b0))


def overlap_map(X, Y, W, H, g: Grid):
    """M_b = sum_i ov_x(i, b) * ov_y(i, b), int64 [nx, ny] (x-major).

    Every cell visits the bins its rectangle touches: columns from
    floor((X - XL)/BW) to floor((X + W - 1 - XL)/BW), clipped to the grid, and
    likewise rows.  Bins outside the die are not part of the map.
    """
    X = np.asarray(X, np.int64); Y = np.asarray(Y, np.int64)
    W = np.asarray(W, np.int64); H = np.asarray(H, np.int64)
    M = np.zeros((g.nx, g.ny), np.int64)
    if X.size == 0:
        return M
    ix0 = np.floor_divide(X - g.XL, g.BW)
    ix1 = np.floor_divide(X + W - 1 - g.XL, g.BW)
    iy0 = np.floor_divide(Y - g.YL, g.BH)
    iy1 = np.floor_divide(Y + H - 1 - g.YL, g.BH)
    span_x = int(np.max(ix1 - ix0)) + 1
    span_y = int(np.max(iy1 - iy0)) + 1
    for dx in range(span_x):
        kx = ix0 + dx
        okx = (kx <= ix1) & (kx >= 0) & (kx < g.nx)
        ox = _axis_overlap(X, W, g.XL, g.BW, kx)
        for dy in range(span_y):
            ky = iy0 + dy
            ok = okx & (ky <= iy1) & (ky >= 0) & (ky < g.ny)
            oy = _axis_overlap(Y, H, g.YL, g.BH, ky)
            area = ox * oy
            sel = ok & (area > 0)
            np.add.at(M, (kx[sel], ky[sel]), area[sel])
    return M


def overlap_map_bruteforce(X, Y, W, H, g: Grid):
    """Same map by visiting every (cell, bin) pair; for tiny cases only."""
    M = np.zeros((g.nx, g.ny), np.int64)
    for i in range(len(X)):
        for kx in range(g.nx):
            ox = max(0, min(int(X[i]) + int(W[i]), g.XL + (kx + 1) * g.BW)
                     - max(int(X[i]), g.XL + kx * g.BW))
            if ox == 0:
                continue
            for ky in range(g.ny):
                oy = max(0, min(int(Y[i]) + int(H[i]), g.YL + (ky + 1) * g.BH)
                         - max(int(Y[i]), g.YL + ky * g.BH))
                M[kx, ky] += ox * oy
    return M


def overflow(M, Fmap, t, g: Grid, movable_area_q):
    """tau = sum_b max(0, M_b - t (A_b - F_b)) / A_mov (all in units of
    2^-2F; t is the float32 target density widened to float64)."""
    abin = float(g.BW * g.BH)
    ex = M.astype(np.float64) - float(t) * (abin - Fmap.astype(np.float64))
    return float(np.sum(np.maximum(ex, 0.0)) / float(movable_area_q))


def bin_density(M, Fmap, t, g: Grid):
    """rho_b = (M_b + t F_b) / A_b, float64 [nx, ny]."""
    abin = float(g.BW * g.BH)
    return (M.astype(np.float64) + float(t) * Fmap.astype(np.float64)) / abin


def field_gather(X, Y, W, H, g: Grid, Ex, Ey):
    """Density gradient of each cell, dD/dx_i = -sum_b a_ib Ex_b and
    dD/dy_i = -sum_b a_ib Ey_b, with a_ib the overlap area of the cell with
    bin b in layout units (the integer overlap times 2^-2F)."""
    X = np.asarray(X, np.int64); Y = np.asarray(Y, np.int64)
    W = np.asarray(W, np.int64); H = np.asarray(H, np.int64)
    gx = np.zeros(X.shape[0]); gy = np.zeros(X.shape[0])
    if X.size == 0:
        return gx, gy
    inv = 2.0 ** (-2 * g.F)
    ix0 = np.floor_divide(X - g.XL, g.BW)
    ix1 = np.floor_divide(X + W - 1 - g.XL, g.BW)
    iy0 = np.floor_divide(Y - g.YL, g.BH)
    iy1 = np.floor_divide(Y + H - 1 - g.YL, g.BH)
    span_x = int(np.max(ix1 - ix0)) + 1
    span_y = int(np.max(iy1 - iy0)) + 1
    for dx in range(span_x):
        kx = ix0 + dx
        okx = (kx <= ix1) & (kx >= 0) & (kx < g.nx)
        ox = _axis_overlap(X, W, g.XL, g.BW, kx)
        for dy in range(span_y):
            ky = iy0 + dy
            ok = okx & (ky <= iy1) & (ky >= 0) & (ky < g.ny)
            oy = _axis_overlap(Y, H, g.YL, g.BH, ky)
            a = (ox * oy).astype(np.float64) * inv
            kxs = np.where(ok, kx, 0); kys = np.where(ok, ky, 0)
            gx -= np.where(ok, a * Ex[kxs, kys], 0.0)
            gy -= np.where(ok, a * Ey[kxs, kys], 0.0)
    return gx, gy


STRETCH = math.sqrt(2.0)


def stretch_axis(X, W, BW):
    """One axis of the local smoothing: widths below sqrt(2) bins become
    Ws = rint(sqrt(2) BW) (ties to even), with Xs = X - floor((Ws - W) / 2)."""
    X = np.asarray(X, np.int64); W = np.asarray(W, np.int64)
    ws = int(np.rint(STRETCH * float(BW)))
    Ws = np.maximum(W, ws)
    return X - (Ws - W) // 2, Ws


def stretch_scale(W, H, Ws, Hs):
    """R = floor(W H 2^31 / (Ws Hs)) per cell, exact (python integers)."""
    return np.array([(int(w) * int(h) << 31) // (int(a) * int(b))
                     for w, h, a, b in zip(W, H, Ws, Hs)], np.int64)


def scaled_term(ov, R):
    """floor(ov R / 2^31) for 0 <= ov < 2^62 and 0 <= R <= 2^31, exact in
    int64: ov = q 2^31 + r gives q R + floor(r R / 2^31)."""
    ov = np.asarray(ov, np.int64); R = np.asarray(R, np.int64)
    q, r = ov >> 31, ov & ((1 << 31) - 1)
    return q * R + ((r * R) >> 31)


def overlap_map_scaled(X, Y, W, H, R, g: Grid):
    """M_b = sum_i floor(ov(i, b) R_i / 2^31), int64 [nx, ny]: the map of
    overlap_map with every (cell, bin) term scaled by R_i / 2^31."""
    X = np.asarray(X, np.int64); Y = np.asarray(Y, np.int64)
    W = np.asarray(W, np.int64); H = np.asarray(H, np.int64)
    R = np.asarray(R, np.int64)
    M = np.zeros((g.nx, g.ny), np.int64)
    if X.size == 0:
        return M
    ix0 = np.floor_divide(X - g.XL, g.BW)
    ix1 = np.floor_divide(X + W - 1 - g.XL, g.BW)
    iy0 = np.floor_divide(Y - g.YL, g.BH)
    iy1 = np.floor_divide(Y + H - 1 - g.YL, g.BH)
    for dx in range(int(np.max(ix1 - ix0)) + 1):
        kx = ix0 + dx
        okx = (kx <= ix1) & (kx >= 0) & (kx < g.nx)
        ox = _axis_overlap(X, W, g.XL, g.BW, kx)
        for dy in range(int(np.max(iy1 - iy0)) + 1):
            ky = iy0 + dy
            ok = okx & (ky <= iy1) & (ky >= 0) & (ky < g.ny)
            oy = _axis_overlap(Y, H, g.YL, g.BH, ky)
            term = scaled_term(ox * oy, R)
            sel = ok & (term > 0)
            np.add.at(M, (kx[sel], ky[sel]), term[sel])
    return M


def stretched(X, Y, W, H, g: Grid):
    """Stretched rectangles (Xs, Ys, Ws, Hs), the map scale R and the
    gradient weight W H / (Ws Hs) (float64) of cells (X, Y, W, H)."""
    Xs, Ws = stretch_axis(X, W, g.BW)
    Ys, Hs = stretch_axis(Y, H, g.BH)
    R = stretch_scale(W, H, Ws, Hs)
    wgt = (np.asarray(W, np.float64) * np.asarray(H, np.float64)) / (Ws.astype(np.float64) * Hs)
    return Xs, Ys, Ws, Hs, R, wgt
