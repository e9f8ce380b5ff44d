"""Seeded synthetic placement workloads (inputs only, no placement arithmetic).

The paper evaluates on the ISPD 2005 and ICCAD 2015 suites (Section 5.1,
Table 1: 0.21M-1.93M cells, about 1.0-1.05 nets per cell, 3.3-4.5 pins per
net).  Those files are not available, so every workload here is generated from
a seed with the same shape: standard cells of height 1 and integer width 1..4,
fixed rectangular macros and IO pads, and a net-degree mix of 60% 2-pin,
20% 3-pin, 15% 4-10 pins and 5% 11-50 pins, plus an optional sliver of very
high-degree (clock/reset-like) nets.

This module is shared by the CUDA library's tests and benchmarks and by the
CPU oracle's tests.  It holds no step of the placement method: it only draws
netlists, die/bin geometry and the initial centred-Gaussian placement.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Design:
    """A placement instance.

    Cells ``[0, n_movable)`` are movable; the rest are fixed (macros, pads).
    Positions are lower-left corners.  Nets are a CSR map: the pins of net
    ``e`` are ``net_ptr[e] .. net_ptr[e+1]-1``; pin ``j`` sits on cell
    ``pin_cell[j]`` at offset ``(pin_dx[j], pin_dy[j])`` from its lower-left.
    """

    name: str
    n_movable: int
    w: np.ndarray  # float32 [n_cells]
    h: np.ndarray  # float32 [n_cells]
    x: np.ndarray  # float32 [n_cells] lower-left x (fixed cells: final)
    y: np.ndarray  # float32 [n_cells]
    net_ptr: np.ndarray  # int32 [n_nets+1]
    pin_cell: np.ndarray  # int32 [n_pins]
    pin_dx: np.ndarray  # float32 [n_pins]
    pin_dy: np.ndarray  # float32 [n_pins]
    die: tuple  # (xl, yl, xh, yh) as python floats
    nx: int
    ny: int
    target_density: float
    is_macro: np.ndarray | None = None  # uint8 [n_cells] or None

    @property
    def n_cells(self) -> int:
        return int(self.w.shape[0])

    @property
    def n_nets(self) -> int:
        return int(self.net_ptr.shape[0] - 1)

    @property
    def n_pins(self) -> int:
        return int(self.pin_cell.shape[0])

    def copy(self) -> "Design":
        return dataclasses.replace(
            self,
            w=self.w.copy(), h=self.h.copy(), x=self.x.copy(), y=self.y.copy(),
            net_ptr=self.net_ptr.copy(), pin_cell=self.pin_cell.copy(),
            pin_dx=self.pin_dx.copy(), pin_dy=self.pin_dy.copy(),
            is_macro=None if self.is_macro is None else self.is_macro.copy())


def _degrees(rng, n_nets, big_frac, big_lo, big_hi, big_log):
    """Net degrees: 60% 2, 20% 3, 15% U[4,10], 5% U[11,50]; then a fraction
    ``big_frac`` of the nets is redrawn from [big_lo, big_hi] (uniform or
    log-uniform)."""
    u = rng.random(n_nets)
    deg = np.empty(n_nets, np.int64)
    deg[u < 0.60] = 2
    m = (u >= 0.60) & (u < 0.80)
    deg[m] = 3
    m = (u >= 0.80) & (u < 0.95)
    deg[m] = rng.integers(4, 11, int(m.sum()))
    m = u >= 0.95
    deg[m] = rng.integers(11, 51, int(m.sum()))
    n_big = int(round(big_frac * n_nets))
    if n_big > 0:
        idx = rng.choice(n_nets, n_big, replace=False)
        if big_log:
            d = np.exp(rng.uniform(math.log(big_lo), math.log(big_hi + 1), n_big))
            deg[idx] = np.clip(np.floor(d), big_lo, big_hi).astype(np.int64)
        else:
            deg[idx] = rng.integers(big_lo, big_hi + 1, n_big)
    return deg


def _distinct_pins(rng, deg, n_cells):
    """Draw, for each net, ``deg`` distinct cells uniformly at random."""
    ptr = np.zeros(deg.shape[0] + 1, np.int64)
    np.cumsum(deg, out=ptr[1:])
    n_pins = int(ptr[-1])
    net_of_pin = np.repeat(np.arange(deg.shape[0], dtype=np.int64), deg)
    cells = rng.integers(0, n_cells, n_pins)
    # nets that take a large share of the cells: draw without replacement
    for e in np.nonzero(2 * deg > n_cells)[0]:
        cells[ptr[e]:ptr[e + 1]] = rng.choice(n_cells, int(deg[e]), replace=False)
    for _ in range(200):
        key = net_of_pin * n_cells + cells
        order = np.argsort(key, kind="stable")
        sk = key[order]
        dup = np.zeros(n_pins, bool)
        dup[order[1:][sk[1:] == sk[:-1]]] = True
        nd = int(dup.sum())
        if nd == 0:
            break
        cells[dup] = rng.integers(0, n_cells, nd)
    else:  # pragma: no cover - degree > n_cells would loop forever
        raise ValueError("could not draw distinct pins")
    return ptr, cells


def _place_macros(rng, n_macros, frac, die, margin, occupied):
    """Non-overlapping integer rectangles with aspect in [0.5, 2] covering
    ``frac`` of the die, placed by rejection."""
    xl, yl, xh, yh = die
    area_each = frac * (xh - xl) * (yh - yl) / max(n_macros, 1)
    rects = []
    for _ in range(n_macros):
        for _attempt in range(100000):
            r = rng.uniform(0.5, 2.0)
            w = max(1.0, round(math.sqrt(area_each * r)))
            h = max(1.0, round(area_each / w))
            if w > (xh - xl) - 2 * margin or h > (yh - yl) - 2 * margin:
                continue
            x = float(rng.integers(int(xl + margin), int(xh - margin - w) + 1))
            y = float(rng.integers(int(yl + margin), int(yh - margin - h) + 1))
            ok = True
            for (ax, ay, aw, ah) in rects + occupied:
                if x < ax + aw and ax < x + w and y < ay + ah and ay < y + h:
                    ok = False
                    break
            if ok:
                rects.append((x, y, w, h))
                break
        else:
            raise RuntimeError("macro placement by rejection failed")
    return rects


def _pads(n_pads, die):
    """``n_pads`` 1x1 IO pads, a quarter per side, evenly spaced, flush inside
    the die edge."""
    xl, yl, xh, yh = die
    per = n_pads // 4
    rects = []
    for k in range(per):
        f = (k + 0.5) / per
        px = math.floor(xl + f * (xh - xl))
        py = math.floor(yl + f * (yh - yl))
        rects.append((float(px), yl, 1.0, 1.0))          # bottom
        rects.append((float(px), yh - 1.0, 1.0, 1.0))    # top
        rects.append((xl, float(py), 1.0, 1.0))          # left
        rects.append((xh - 1.0, float(py), 1.0, 1.0))    # right
    return rects


def _centred_start(rng, w, h, die, sigma_frac):
    """Lower-left corners of cells whose centres are drawn from N(die centre,
    (sigma_frac * die extent)^2) per axis, clamped into the die."""
    xl, yl, xh, yh = die
    n = w.shape[0]
    cx = 0.5 * (xl + xh) + sigma_frac * (xh - xl) * rng.standard_normal(n)
    cy = 0.5 * (yl + yh) + sigma_frac * (yh - yl) * rng.standard_normal(n)
    mx = np.clip(cx - 0.5 * w, xl, xh - w)
    my = np.clip(cy - 0.5 * h, yl, yh - h)
    return mx.astype(np.float32), my.astype(np.float32)


def random_start(design, seed, sigma_frac=1e-3):
    """A fresh centred-Gaussian start of the same design (the random initial
    placement of an independent run): positions of all cells, the fixed ones
    unchanged, the movable ones redrawn from ``seed``."""
    rng = np.random.default_rng(seed)
    n = design.n_movable
    x, y = design.x.copy(), design.y.copy()
    x[:n], y[:n] = _centred_start(rng, design.w[:n], design.h[:n], design.die, sigma_frac)
    return x, y


def make_design(*, n_movable, die, nx, ny, n_nets, n_macros=0, macro_frac=0.0,
                n_pads=0, target_density=1.0, big_frac=0.0, big_lo=0, big_hi=0,
                big_log=False, seed=0, name="synthetic", init_sigma_frac=1e-3):
    """Draw a seeded design.

    Movable cells start at a centred Gaussian: centres ~ N(die centre,
    (init_sigma_frac * die extent)^2) per axis, clamped into the die.
    """
    rng = np.random.default_rng(seed)
    die = tuple(float(v) for v in die)
    xl, yl, xh, yh = die
    pads = _pads(n_pads, die)
    macros = _place_macros(rng, n_macros, macro_frac, die, 2.0, pads)
    fixed = macros + pads
    n_fixed = len(fixed)
    n_cells = n_movable + n_fixed
    w = np.empty(n_cells, np.float32)
    h = np.empty(n_cells, np.float32)
    x = np.empty(n_cells, np.float32)
    y = np.empty(n_cells, np.float32)
    w[:n_movable] = rng.integers(1, 5, n_movable).astype(np.float32)
    h[:n_movable] = 1.0
    for i, (fx, fy, fw, fh) in enumerate(fixed):
        x[n_movable + i], y[n_movable + i] = fx, fy
        w[n_movable + i], h[n_movable + i] = fw, fh
    is_macro = np.zeros(n_cells, np.uint8)
    is_macro[n_movable:n_movable + len(macros)] = 1

    deg = _degrees(rng, n_nets, big_frac, big_lo, big_hi, big_log)
    deg = np.minimum(deg, n_cells)
    ptr, cells = _distinct_pins(rng, deg, n_cells)
    pdx = (rng.random(cells.shape[0]) * w[cells]).astype(np.float32)
    pdy = (rng.random(cells.shape[0]) * h[cells]).astype(np.float32)

    x[:n_movable], y[:n_movable] = _centred_start(rng, w[:n_movable], h[:n_movable], die,
                                                  init_sigma_frac)

    return Design(name=name, n_movable=n_movable, w=w, h=h, x=x, y=y,
                  net_ptr=ptr.astype(np.int32), pin_cell=cells.astype(np.int32),
                  pin_dx=pdx, pin_dy=pdy, die=die, nx=nx, ny=ny,
                  target_density=float(target_density), is_macro=is_macro)


# Workload shapes.  Names describe the instance; sizes follow the paper's
# benchmark statistics (Table 1) where the workload imitates them.

def tiny_1k(seed=0):
    """1,000 movable cells on a 256x256 die with 16 IO pads, 1,100 nets,
    64x64 bins, target density 1.0."""
    return make_design(n_movable=1000, die=(0, 0, 256, 256), nx=64, ny=64,
                       n_nets=1100, n_pads=16, target_density=1.0, seed=seed,
                       name="tiny_1k")


def mixed_size_1k(seed=0, n_macros=20):
    """tiny_1k with n_macros of its movable cells enlarged into movable macros
    of 8-24 units a side (2-6 bins), flagged as macros, so Shuffle (macros)
    has candidates and cells span more than 2 x 2 bins.  Pin offsets stay
    where they were, inside the enlarged cells."""
    d = tiny_1k(seed)
    rng = np.random.default_rng(seed + 7)
    idx = rng.choice(d.n_movable, n_macros, replace=False)
    d.w[idx] = rng.integers(8, 25, n_macros).astype(np.float32)
    d.h[idx] = rng.integers(8, 25, n_macros).astype(np.float32)
    xl, yl, xh, yh = d.die
    d.x[idx] = np.clip(d.x[idx] - 0.5 * (d.w[idx] - 1.0), xl, xh - d.w[idx]).astype(np.float32)
    d.y[idx] = np.clip(d.y[idx] - 0.5 * (d.h[idx] - 1.0), yl, yh - d.h[idx]).astype(np.float32)
    d.is_macro[idx] = 1
    d.name = "mixed_size_1k"
    return d


def _enlarge_into_macros(d, rng, n_macros, lo, hi):
    """Turn n_macros random movable cells into movable macros of lo..hi units
    a side, flagged, their lower-left corners moved so that the centres stay
    and the macros stay inside the die.  Pin offsets stay where they were,
    inside the enlarged cells."""
    idx = rng.choice(d.n_movable, n_macros, replace=False)
    w0, h0 = d.w[idx].copy(), d.h[idx].copy()
    d.w[idx] = rng.integers(lo, hi + 1, n_macros).astype(np.float32)
    d.h[idx] = rng.integers(lo, hi + 1, n_macros).astype(np.float32)
    xl, yl, xh, yh = d.die
    d.x[idx] = np.clip(d.x[idx] - 0.5 * (d.w[idx] - w0), xl, xh - d.w[idx]).astype(np.float32)
    d.y[idx] = np.clip(d.y[idx] - 0.5 * (d.h[idx] - h0), yl, yh - d.h[idx]).astype(np.float32)
    d.is_macro[idx] = 1
    return d


def medium_mixed_210k(seed=0, n_macros=32):
    """medium_210k with n_macros of its movable cells enlarged into movable
    macros of 16-64 units a side (4-16 bins), flagged as macros: the
    mixed-size case where Shuffle (macros) and WireMask have work."""
    d = _enlarge_into_macros(medium_210k(seed), np.random.default_rng(seed + 11), n_macros, 16, 64)
    d.name = "medium_mixed_210k"
    return d


def medium_210k(seed=0):
    """210k movable cells on a 2000x2000 die, 10 fixed macros covering 20% of
    the area, 220k nets plus 0.1% nets of degree U[100, 2000], 512x512 bins,
    target density 0.9 (adaptec1-sized)."""
    return make_design(n_movable=210_000, die=(0, 0, 2000, 2000), nx=512, ny=512,
                       n_nets=220_000, n_macros=10, macro_frac=0.20,
                       target_density=0.9, big_frac=1e-3, big_lo=100, big_hi=2000,
                       big_log=False, seed=seed, name="medium_210k")


def large_2m(seed=0):
    """2.1M movable cells on a 4096x4096 die, 60 fixed macros covering 30% of
    the area, 2.2M nets plus 0.1% nets of log-uniform degree [51, 5000],
    1024x1024 bins, target density 0.7 (superblue7-sized)."""
    return make_design(n_movable=2_100_000, die=(0, 0, 4096, 4096), nx=1024, ny=1024,
                       n_nets=2_200_000, n_macros=60, macro_frac=0.30,
                       target_density=0.7, big_frac=1e-3, big_lo=51, big_hi=5000,
                       big_log=True, seed=seed, name="large_2m")


def scaled(n_movable, nx, seed=0, macro_frac=0.2, n_macros=10, target_density=0.9,
           name=None):
    """A smaller instance with the medium workload's shape: die area scaled
    with the cell count, grid ``nx`` x ``nx``."""
    side = 2000.0 * math.sqrt(n_movable / 210_000)
    # round the die so that nx bins have a width that is a power-of-two fraction
    side = max(nx / 8.0, round(side * 8 / nx) * nx / 8.0)
    return make_design(n_movable=n_movable, die=(0, 0, side, side), nx=nx, ny=nx,
                       n_nets=int(n_movable * 220 / 210), n_macros=n_macros,
                       macro_frac=macro_frac, target_density=target_density,
                       big_frac=1e-3, big_lo=100, big_hi=min(2000, n_movable // 4),
                       seed=seed, name=name or f"scaled_{n_movable}")
