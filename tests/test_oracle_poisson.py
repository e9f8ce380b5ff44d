"""Pins of the oracle's spectral Poisson solve: the DCT-II of scipy, naive
against separable evaluation, single-mode closed forms, the discrete
Neumann Laplacian, reconstruction and E = -grad psi."""
import math

import numpy as np
import pytest
import scipy.fft

from oracle import poisson as pois


def test_coefficients_are_scaled_dct2():
    # scipy's unnormalised DCT-II: X_k = 2 sum_n x_n cos(pi k (2n+1) / 2N) per axis
    rng = np.random.default_rng(0)
    for M, N in [(8, 8), (8, 5), (16, 12)]:
        rho = rng.random((M, N))
        ref = scipy.fft.dctn(rho, type=2) / 4.0
        cu = np.where(np.arange(M) == 0, 1.0, 2.0)
        cv = np.where(np.arange(N) == 0, 1.0, 2.0)
        ref *= cu[:, None] * cv[None, :] / (M * N)
        np.testing.assert_allclose(pois.coefficients(rho), ref, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(pois.coefficients_naive(rho), ref, rtol=1e-12, atol=1e-14)


def test_reconstruction_from_coefficients():
    rng = np.random.default_rng(1)
    rho = rng.random((12, 9))
    a = pois.coefficients(rho)
    cx, _ = pois.cos_sin_tables(12)
    cy, _ = pois.cos_sin_tables(9)
    np.testing.assert_allclose(cx.T @ a @ cy, rho, rtol=1e-12, atol=1e-12)


def test_naive_equals_separable():
    rng = np.random.default_rng(2)
    rho = rng.random((16, 12)) * 3
    a = pois.poisson_naive(rho, 1.5, 0.75)
    b = pois.poisson(rho, 1.5, 0.75)
    for p, q in zip(a, b):
        np.testing.assert_allclose(p, q, rtol=1e-11, atol=1e-11 * np.abs(q).max())


@pytest.mark.parametrize("u,v", [(1, 0), (0, 3), (2, 5), (7, 1)])
def test_single_mode_closed_form(u, v):
    M, N, hx, hy = 16, 8, 2.0, 1.25
    X = (np.arange(M) + 0.5) * hx
    Y = (np.arange(N) + 0.5) * hy
    wu, wv = math.pi * u / (M * hx), math.pi * v / (N * hy)
    rho = np.outer(np.cos(wu * X), np.cos(wv * Y))
    psi, ex, ey = pois.poisson(rho, hx, hy)
    k2 = wu * wu + wv * wv
    np.testing.assert_allclose(psi, rho / k2, atol=1e-12)
    np.testing.assert_allclose(ex, wu / k2 * np.outer(np.sin(wu * X), np.cos(wv * Y)), atol=1e-12)
    np.testing.assert_allclose(ey, wv / k2 * np.outer(np.cos(wu * X), np.sin(wv * Y)), atol=1e-12)
    # 5-point Laplacian with mirror (Neumann) ghost cells: the cosine mode is an
    # eigenvector with eigenvalue -(lu + lv), lu = (2 sin(pi u / 2M) / hx)^2
    pp = np.pad(psi, 1, mode="symmetric")
    lap = ((pp[2:, 1:-1] - 2 * psi + pp[:-2, 1:-1]) / hx ** 2
           + (pp[1:-1, 2:] - 2 * psi + pp[1:-1, :-2]) / hy ** 2)
    lu = (2 * math.sin(math.pi * u / (2 * M)) / hx) ** 2
    lv = (2 * math.sin(math.pi * v / (2 * N)) / hy) ** 2
    np.testing.assert_allclose(lap, -(lu + lv) / k2 * rho, atol=1e-12)


def test_constant_density_has_no_field():
    psi, ex, ey = pois.poisson(np.full((8, 8), 0.7), 1.0, 1.0)
    for a in (psi, ex, ey):
        assert np.abs(a).max() < 1e-13


def test_field_is_minus_gradient_of_potential():
    # smooth density (modes u, v <= 3 on a 64 grid): central differences of psi
    # approximate -E to O(h^2)
    M = N = 64
    h = 1.0
    rng = np.random.default_rng(3)
    X = (np.arange(M) + 0.5) * h
    rho = np.zeros((M, N))
    for u in range(4):
        for v in range(4):
            rho += rng.standard_normal() * np.outer(np.cos(math.pi * u * X / (M * h)),
                                                   np.cos(math.pi * v * X / (N * h)))
    psi, ex, ey = pois.poisson(rho, h, h)
    dx = -(psi[2:, 1:-1] - psi[:-2, 1:-1]) / (2 * h)
    dy = -(psi[1:-1, 2:] - psi[1:-1, :-2]) / (2 * h)
    scale = max(np.abs(ex).max(), np.abs(ey).max())
    assert np.abs(dx - ex[1:-1, 1:-1]).max() < 2e-3 * scale
    assert np.abs(dy - ey[1:-1, 1:-1]).max() < 2e-3 * scale
    # a sign or axis mistake would be off by O(scale)
    assert np.abs(dx + ex[1:-1, 1:-1]).max() > 0.5 * np.abs(ex).max()


def test_spectral_laplacian_of_potential():
    # the Laplacian of the series (coefficient-wise -(wu^2 + wv^2)) gives back
    # -(rho - mean rho)
    rng = np.random.default_rng(4)
    M, N, hx, hy = 16, 16, 1.0, 2.0
    rho = rng.random((M, N))
    psi, _, _ = pois.poisson(rho, hx, hy)
    ap = pois.coefficients(psi)
    wu, wv = pois.wavenumbers(M, N, hx, hy)
    lap_coef = -(wu[:, None] ** 2 + wv[None, :] ** 2) * ap
    cx, _ = pois.cos_sin_tables(M)
    cy, _ = pois.cos_sin_tables(N)
    lap = cx.T @ lap_coef @ cy
    np.testing.assert_allclose(lap, -(rho - rho.mean()), atol=1e-12)


@pytest.mark.parametrize("u,v", [(1, 0), (0, 3), (2, 5)])
def test_density_energy_of_single_modes(u, v):
    # rho = cos(wu X) cos(wv Y) has psi = rho / (wu^2 + wv^2), so
    # D = 1/2 hx hy sum rho psi = 1/2 hx hy (Sx Sy) / (wu^2 + wv^2) with
    # Sx = sum_x cos^2(pi u (x + 1/2) / M) = M/2 for 0 < u < M and M for u = 0
    M, N, hx, hy = 16, 8, 2.0, 1.25
    X = (np.arange(M) + 0.5) * hx
    Y = (np.arange(N) + 0.5) * hy
    wu, wv = math.pi * u / (M * hx), math.pi * v / (N * hy)
    rho = np.outer(np.cos(wu * X), np.cos(wv * Y))
    psi, _, _ = pois.poisson(rho, hx, hy)
    Sx = M / 2 if u else M
    Sy = N / 2 if v else N
    D = 0.5 * hx * hy * Sx * Sy / (wu * wu + wv * wv)
    assert pois.density_energy(rho, psi, hx, hy) == pytest.approx(D, rel=1e-12)
    # a constant offset carries no energy (the (0, 0) mode is dropped), and
    # two orthogonal modes add their energies
    psi_c, _, _ = pois.poisson(rho + 3.0, hx, hy)
    assert pois.density_energy(rho, psi_c, hx, hy) == pytest.approx(D, rel=1e-12)
    rho2 = np.outer(np.cos(math.pi * 3 * X / (M * hx)), np.cos(math.pi * 1 * Y / (N * hy)))
    psi2, _, _ = pois.poisson(rho2, hx, hy)
    psi12, _, _ = pois.poisson(rho + rho2, hx, hy)
    assert pois.density_energy(rho + rho2, psi12, hx, hy) == pytest.approx(
        D + pois.density_energy(rho2, psi2, hx, hy), rel=1e-12)
