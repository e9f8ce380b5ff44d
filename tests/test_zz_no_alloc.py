"""place_overflow_noalloc: the density map and overflow computed into
caller-owned buffers with the library's static scratch only.

Callers that cannot allocate device memory at the point where they need the
overflow (a framework whose memory pool owns the device during a step, a
real-time service that forbids allocation after start-up) use this entry
point instead of a handle.  It must give the same map and overflow as
place_eval_density on the same positions, on consecutive calls (the shared
scratch keeps the previous call's contents and must be cleared each time),
and the FP64 oracle's map and overflow where the sizes are not multiples of
the fixed-point unit.  This file is collected last on purpose.
"""
import os

import numpy as np
import pytest

from oracle import density as odens
from paper_2402_18311_gb300 import place, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(place.LIB_PATH):
        from paper_2402_18311_gb300 import build
        build.build()
    place.lib()
    torch.cuda.set_device(0)
    return torch


def _reference(h, d):
    G = d.nx * d.ny
    gm = np.empty(G, np.int64)
    tau = place.place_eval_density(h, 0, gm)
    return gm, tau


def _noalloc(torch, x, y, w, h, d, F, fixed=None):
    """One call on the current stream; returns (map, overflow) on the host."""
    G = d.nx * d.ny
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    mp = torch.full((G,), -7, dtype=torch.int64, device="cuda")
    n = len(x)
    place.place_overflow_noalloc(dev(x), dev(y), dev(w), dev(h), n, d.die,
                                 (d.nx, d.ny, d.target_density), F, fixed, out, mp,
                                 torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return mp.cpu().numpy(), float(out.item())


def _oracle(d, x, y, F, with_fixed=True):
    g = odens.Grid(d.die, d.nx, d.ny, F)
    n = d.n_movable
    W, H = odens.quantize(d.w, F), odens.quantize(d.h, F)
    M = odens.overlap_map(odens.quantize(x[:n], F), odens.quantize(y[:n], F), W[:n], H[:n], g)
    if with_fixed:
        Fm = odens.overlap_map(odens.quantize(d.x[n:], F), odens.quantize(d.y[n:], F), W[n:], H[n:], g)
    else:
        Fm = np.zeros_like(M)
    tau = odens.overflow(M, Fm, np.float32(d.target_density), g, int(np.sum(W[:n] * H[:n])))
    return M, tau


def test_noalloc_matches_handle_on_consecutive_calls(torch_cuda):
    torch = torch_cuda
    d = synth.scaled(20000, 128, seed=4)
    h = place.place_create(d, place.place_default_params(tau_stop=-1.0, max_iters=1000))
    try:
        info = place.place_get_info(h)
        n, G = d.n_movable, d.nx * d.ny
        fixed = torch.empty(G, dtype=torch.int64, device="cuda")
        place.place_get_fixed_map(h, fixed)
        for iters in (0, 120):  # two calls in a row, on different placements
            place.place_step(h, iters)
            x = np.empty(d.n_cells, np.float32); y = np.empty(d.n_cells, np.float32)
            place.place_get_positions(h, 0, x, y)
            ref_map, ref_tau = _reference(h, d)
            mp, tau = _noalloc(torch, x[:n], y[:n], d.w[:n], d.h[:n], d, info.frac_bits, fixed)
            np.testing.assert_array_equal(mp, ref_map)
            assert tau == pytest.approx(ref_tau, rel=1e-12, abs=1e-15)
    finally:
        place.place_destroy(h)


def test_noalloc_non_square_grid_non_dyadic_sizes_without_fixed_cells(torch_cuda):
    # a 256 x 128 grid (the x-major layout is not symmetric), no fixed cells
    # (fixed_map NULL), and widths that are not multiples of 2^-F: the map and
    # the overflow (over the quantised movable area) equal the oracle's, on
    # two calls in a row
    torch = torch_cuda
    rng = np.random.default_rng(21)
    n = 5000
    d = synth.make_design(n_movable=n, die=(0, 0, 1024, 512), nx=256, ny=128, n_nets=10,
                          n_pads=0, target_density=0.9, seed=21)
    d.w[:n] = (rng.integers(1, 5, n) * 1.3).astype(np.float32)
    d.h[:n] = np.float32(0.7)
    F = odens.frac_bits(d.die, float(np.sum(d.w.astype(np.float64) * d.h)))
    assert (d.w[:n].astype(np.float64) * 2.0 ** F % 1 != 0).any()
    for spread in (0.05, 0.4):
        x = (512 + rng.normal(0, spread * 1024, n)).clip(0, 1000).astype(np.float32)
        y = (256 + rng.normal(0, spread * 512, n)).clip(0, 500).astype(np.float32)
        d.x[:n], d.y[:n] = x, y
        mp, tau = _noalloc(torch, x, y, d.w[:n], d.h[:n], d, F, None)
        M, otau = _oracle(d, d.x, d.y, F, with_fixed=False)
        np.testing.assert_array_equal(mp.reshape(d.nx, d.ny), M)
        assert tau == pytest.approx(otau, rel=1e-12, abs=1e-15)
        assert otau > 0


def test_noalloc_at_the_largest_grid(torch_cuda):
    # PLACE_NOALLOC_MAX_BINS = 1024 x 1024 bins, with fixed cells
    torch = torch_cuda
    d = synth.make_design(n_movable=60000, die=(0, 0, 2048, 2048), nx=1024, ny=1024, n_nets=10,
                          n_pads=64, target_density=0.8, seed=9)
    n = d.n_movable
    F = odens.frac_bits(d.die, float(np.sum(d.w.astype(np.float64) * d.h)))
    M, otau = _oracle(d, d.x, d.y, F)
    g = odens.Grid(d.die, d.nx, d.ny, F)
    W, H = odens.quantize(d.w, F), odens.quantize(d.h, F)
    Fm = odens.overlap_map(odens.quantize(d.x[n:], F), odens.quantize(d.y[n:], F), W[n:], H[n:], g)
    fixed = torch.from_numpy(np.ascontiguousarray(Fm.ravel())).cuda()
    mp, tau = _noalloc(torch, d.x[:n], d.y[:n], d.w[:n], d.h[:n], d, F, fixed)
    np.testing.assert_array_equal(mp.reshape(d.nx, d.ny), M)
    assert tau == pytest.approx(otau, rel=1e-12, abs=1e-15)


def test_noalloc_flags_cells_outside_the_fixed_point_range(torch_cuda):
    # a zero-width cell quantises to W = 0: the kernel skips it and the
    # overflow comes back NaN instead of a number
    torch = torch_cuda
    d = synth.scaled(2000, 128, seed=5)
    n = d.n_movable
    w = d.w[:n].copy()
    w[17] = 0.0
    _, tau = _noalloc(torch, d.x[:n], d.y[:n], w, d.h[:n], d, 10, None)
    assert np.isnan(tau)
    _, tau = _noalloc(torch, d.x[:n], d.y[:n], d.w[:n], d.h[:n], d, 10, None)
    assert np.isfinite(tau)


def test_noalloc_rejects_bad_arguments_on_the_host(torch_cuda):
    torch = torch_cuda
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    with pytest.raises(place.PlaceError) as ei:
        place.place_overflow_noalloc(x, x, x + 1, x + 1, 4, (0, 0, 2048, 2048),
                                     (2048, 1024, 1.0), 10, None, out)
    assert ei.value.code == place.PLACE_EINVAL
    assert "exceed the static scratch" in str(ei.value)
    # 2048 * 2^19 = 2^30: too fine a resolution for this die
    with pytest.raises(place.PlaceError) as ei:
        place.place_overflow_noalloc(x, x, x + 1, x + 1, 4, (0, 0, 2048, 2048),
                                     (128, 128, 1.0), 19, None, out)
    assert ei.value.code == place.PLACE_ERANGE
    with pytest.raises(place.PlaceError) as ei:
        place.place_overflow_noalloc(x, x, x + 1, x + 1, 4, (0.3, 0, 2048, 2048),
                                     (128, 128, 1.0), 4, None, out)
    assert ei.value.code == place.PLACE_EINVAL
