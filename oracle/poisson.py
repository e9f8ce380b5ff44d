"""Spectral Poisson solve for the electrostatic potential and field, float64.

Test infrastructure only (see ``oracle/__init__.py``).

The paper cites ePlace ("electrostatics-based placement using fast Fourier
transform", reference list) for the density penalty but does not restate it.
The reading used here (Neumann boundary, cell-centred bins, continuous
wavenumbers):

    grid M x N bins of size hx x hy, bin centres X_x = (x + 1/2) hx,
    Y_y = (y + 1/2) hy, wavenumbers w_u = pi u / (M hx), w_v = pi v / (N hy),
    c_0 = 1, c_k = 2 (k > 0).

    a_uv = c_u c_v / (M N) sum_x sum_y rho_xy cos(w_u X_x) cos(w_v Y_y)
    psi_xy = sum_{(u,v) != (0,0)} a_uv / (w_u^2 + w_v^2) cos(w_u X_x) cos(w_v Y_y)
    Ex_xy  = sum a_uv w_u / (w_u^2 + w_v^2) sin(w_u X_x) cos(w_v Y_y)
    Ey_xy  = sum a_uv w_v / (w_u^2 + w_v^2) cos(w_u X_x) sin(w_v Y_y)

so that the Laplacian of psi is -(rho - mean(rho)) and E = -grad psi.
Arrays are x-major: ``rho[x, y]``.
"""
from __future__ import annotations

import math

import numpy as np


def wavenumbers(M, N, hx, hy):
    wu = math.pi * np.arange(M) / (M * hx)
    wv = math.pi * np.arange(N) / (N * hy)
    return wu, wv


def _weights(M, N, hx, hy):
    wu, wv = wavenumbers(M, N, hx, hy)
    den = wu[:, None] ** 2 + wv[None, :] ** 2
    den[0, 0] = 1.0
    wpsi = 1.0 / den
    wx = wu[:, None] / den
    wy = wv[None, :] / den
    for w in (wpsi, wx, wy):
        w[0, 0] = 0.0
    return wpsi, wx, wy


def _c(n):
    c = np.full(n, 2.0)
    c[0] = 1.0
    return c


def cos_sin_tables(n):
    """T[k, i] = cos(pi k (i + 1/2) / n) and the same with sin."""
    k = np.arange(n)[:, None]
    i = np.arange(n)[None, :]
    arg = math.pi * k * (i + 0.5) / n
    return np.cos(arg), np.sin(arg)


def coefficients_naive(rho):
    """a_uv by the direct double sum for every (u, v): O(M^2 N^2)."""
    M, N = rho.shape
    cx, _ = cos_sin_tables(M)
    cy, _ = cos_sin_tables(N)
    cu, cv = _c(M), _c(N)
    a = np.zeros((M, N))
    for u in range(M):
        for v in range(N):
            basis = np.outer(cx[u], cy[v])
            a[u, v] = cu[u] * cv[v] / (M * N) * np.sum(rho * basis)
    return a


def poisson_naive(rho, hx, hy):
    """(psi, Ex, Ey) by direct summation of the series for every output
    point: O(M^2 N^2).  For grids up to about 64 x 64."""
    M, N = rho.shape
    a = coefficients_naive(rho)
    wpsi, wx, wy = _weights(M, N, hx, hy)
    cx, sx = cos_sin_tables(M)
    cy, sy = cos_sin_tables(N)
    psi = np.zeros((M, N)); ex = np.zeros((M, N)); ey = np.zeros((M, N))
    for u in range(M):
        for v in range(N):
            if u == 0 and v == 0:
                continue
            psi += a[u, v] * wpsi[u, v] * np.outer(cx[u], cy[v])
            ex += a[u, v] * wx[u, v] * np.outer(sx[u], cy[v])
            ey += a[u, v] * wy[u, v] * np.outer(cx[u], sy[v])
    return psi, ex, ey


def coefficients(rho):
    """a_uv by separable products: diag(c/M) Cx rho Cy^T diag(c/N)."""
    M, N = rho.shape
    cx, _ = cos_sin_tables(M)
    cy, _ = cos_sin_tables(N)
    a = cx @ rho @ cy.T
    return a * (_c(M)[:, None] / M) * (_c(N)[None, :] / N)


def poisson(rho, hx, hy):
    """(psi, Ex, Ey) by separable products: O(M N (M + N))."""
    M, N = rho.shape
    a = coefficients(rho)
    wpsi, wx, wy = _weights(M, N, hx, hy)
    cx, sx = cos_sin_tables(M)
    cy, sy = cos_sin_tables(N)
    psi = cx.T @ (a * wpsi) @ cy
    ex = sx.T @ (a * wx) @ cy
    ey = cx.T @ (a * wy) @ sy
    return psi, ex, ey


def density_energy(rho, psi, hx, hy):
    """D = 1/2 sum_b A_b rho_b psi_b (electrostatic energy)."""
    return 0.5 * hx * hy * float(np.sum(rho * psi))
