"""HPWL (Eq. 1) and the weighted-average wirelength model (Eq. 3), float64.

Test infrastructure only (see ``oracle/__init__.py``).

Pins: the position of pin ``j`` is the lower-left corner of its cell plus the
pin offset, ``p_j = (x_c(j) + dx_j, y_c(j) + dy_j)``.  Eq. 1 writes HPWL over
cell positions; pin offsets are the standard reading for real netlists.
"""
from __future__ import annotations

import numpy as np


def pin_positions(pin_cell, pin_dx, pin_dy, x, y):
    """Pin coordinates in float64 from float32 (or float64) inputs."""
    px = np.asarray(x, np.float64)[pin_cell] + np.asarray(pin_dx, np.float64)
    py = np.asarray(y, np.float64)[pin_cell] + np.asarray(pin_dy, np.float64)
    return px, py


def _segments(net_ptr):
    net_ptr = np.asarray(net_ptr, np.int64)
    deg = np.diff(net_ptr)
    nonempty = np.nonzero(deg > 0)[0]
    return net_ptr, deg, nonempty


def hpwl_per_net(net_ptr, pin_cell, pin_dx, pin_dy, x, y, net_w=None):
    """Per-net HPWL_e = (max x - min x) + (max y - min y) over the net's pins
    (Eq. 1), times the net weight (1 when ``net_w`` is None)."""
    net_ptr, deg, ne = _segments(net_ptr)
    px, py = pin_positions(pin_cell, pin_dx, pin_dy, x, y)
    out = np.zeros(deg.shape[0], np.float64)
    if ne.size:
        st = net_ptr[ne]
        out[ne] = (np.maximum.reduceat(px, st) - np.minimum.reduceat(px, st)
                   + np.maximum.reduceat(py, st) - np.minimum.reduceat(py, st))
    if net_w is not None:
        out *= np.asarray(net_w, np.float64)
    return out


def hpwl(net_ptr, pin_cell, pin_dx, pin_dy, x, y, net_w=None):
    """Total HPWL, Eq. 1: sum over nets of HPWL_e."""
    return float(np.sum(hpwl_per_net(net_ptr, pin_cell, pin_dx, pin_dy, x, y, net_w)))


def wa_axis(net_ptr, p, gamma):
    """Weighted-average wirelength of every net along one axis (Eq. 3).

    For net e with pin coordinates p_j:
        WL_e = sum p_j e^{p_j/g} / sum e^{p_j/g} - sum p_j e^{-p_j/g} / sum e^{-p_j/g}.
    Each exponential is shifted by the net's max (resp. min) coordinate before
    it is taken; the shift cancels between numerator and denominator, so the
    value is Eq. 3 exactly, without overflow.

    Returns (WL per net, dWL/dp per pin).  The derivative of Eq. 3 is
        dWL_e/dp_j = (a_j/S+)(1 + (p_j - WL+)/g) - (b_j/S-)(1 - (p_j - WL-)/g)
    with a_j = e^{(p_j - max)/g}, S+ = sum a, WL+ = sum p a / S+ and b_j, S-,
    WL- the same with -g and the min.
    """
    net_ptr, deg, ne = _segments(net_ptr)
    n_nets = deg.shape[0]
    wl = np.zeros(n_nets, np.float64)
    grad = np.zeros(p.shape[0], np.float64)
    if ne.size == 0:
        return wl, grad
    st = net_ptr[ne]
    net_of_pin = np.repeat(np.arange(n_nets), deg)
    pmax = np.zeros(n_nets)
    pmin = np.zeros(n_nets)
    pmax[ne] = np.maximum.reduceat(p, st)
    pmin[ne] = np.minimum.reduceat(p, st)
    a = np.exp((p - pmax[net_of_pin]) / gamma)
    b = np.exp((pmin[net_of_pin] - p) / gamma)
    sp = np.zeros(n_nets); tp = np.zeros(n_nets)
    sm = np.zeros(n_nets); tm = np.zeros(n_nets)
    sp[ne] = np.add.reduceat(a, st)
    tp[ne] = np.add.reduceat(p * a, st)
    sm[ne] = np.add.reduceat(b, st)
    tm[ne] = np.add.reduceat(p * b, st)
    wlp = np.zeros(n_nets); wlm = np.zeros(n_nets)
    wlp[ne] = tp[ne] / sp[ne]
    wlm[ne] = tm[ne] / sm[ne]
    wl = wlp - wlm
    e = net_of_pin
    grad = (a / sp[e]) * (1.0 + (p - wlp[e]) / gamma) - (b / sm[e]) * (1.0 - (p - wlm[e]) / gamma)
    return wl, grad


def wa_wirelength(net_ptr, pin_cell, pin_dx, pin_dy, x, y, gamma, n_movable,
                  net_w=None):
    """Sum over nets of WL_e(x) + WL_e(y) (Eq. 2's wirelength term, Eq. 3) and
    its gradient with respect to the lower-left corners of the movable cells.

    A cell's gradient is the sum of its pins' gradients (pin offsets are
    constant); fixed cells get none.  Returns (WL, grad_x[n_movable],
    grad_y[n_movable]).
    """
    px, py = pin_positions(pin_cell, pin_dx, pin_dy, x, y)
    wlx, gpx = wa_axis(net_ptr, px, gamma)
    wly, gpy = wa_axis(net_ptr, py, gamma)
    if net_w is not None:
        nw = np.asarray(net_w, np.float64)
        wlx = wlx * nw
        wly = wly * nw
        deg = np.diff(np.asarray(net_ptr, np.int64))
        pw = np.repeat(nw, deg)
        gpx = gpx * pw
        gpy = gpy * pw
    pc = np.asarray(pin_cell, np.int64)
    mov = pc < n_movable
    gx = np.zeros(n_movable)
    gy = np.zeros(n_movable)
    np.add.at(gx, pc[mov], gpx[mov])
    np.add.at(gy, pc[mov], gpy[mov])
    return float(np.sum(wlx) + np.sum(wly)), gx, gy
