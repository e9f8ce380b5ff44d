"""place_overflow_noalloc: the density map and overflow computed into
caller-owned buffers with the library's static scratch only.

Callers that cannot allocate device memory at the point where they need the
overflow (a framework whose memory pool owns the device during a step, a
real-time service that forbids allocation after start-up) use this entry
point instead of a handle.  It must give the same map and overflow as
place_eval_density on the same positions, on consecutive calls (the shared
scratch keeps the previous call's contents and must be cleared each time).
This file is collected last on purpose.
"""
import os

import numpy as np
import pytest

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


def test_noalloc_matches_handle_on_consecutive_calls(torch_cuda):
    torch = torch_cuda
    d = synth.scaled(20000, 128, seed=4)
    h = place.place_create(d, place.place_default_params(tau_stop=-1.0, max_iters=1000))
    try:
        info = place.place_get_info(h)
        n, G = d.n_movable, d.nx * d.ny
        fixed = torch.empty(G, dtype=torch.int64, device="cuda")
        place.place_get_fixed_map(h, fixed)
        w = torch.from_numpy(d.w[:n].copy()).cuda()
        hh = torch.from_numpy(d.h[:n].copy()).cuda()
        mov_area = float(np.sum(d.w[:n].astype(np.float64) * d.h[:n]))
        die = d.die
        bins = (d.nx, d.ny, d.target_density)
        for iters in (0, 120):  # two calls in a row, on different placements
            place.place_step(h, iters)
            xs = torch.empty(d.n_cells, dtype=torch.float32, device="cuda")
            ys = torch.empty(d.n_cells, dtype=torch.float32, device="cuda")
            place.place_get_positions(h, 0, xs, ys)
            ref_map, ref_tau = _reference(h, d)
            out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
            mp = torch.full((G,), -7, dtype=torch.int64, device="cuda")
            place.place_overflow_noalloc(xs[:n].contiguous(), ys[:n].contiguous(), w, hh, n,
                                         mov_area, die, bins, info.frac_bits, fixed, out, mp,
                                         torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(mp.cpu().numpy(), ref_map)
            assert float(out.item()) == pytest.approx(ref_tau, rel=1e-12, abs=1e-15)
    finally:
        place.place_destroy(h)


def test_noalloc_rejects_grids_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    with pytest.raises(place.PlaceError) as ei:
        place.place_overflow_noalloc(x, x, x + 1, x + 1, 4, 4.0, (0, 0, 2048, 2048),
                                     (2048, 1024, 1.0), 10, None, out)
    assert ei.value.code == place.PLACE_EINVAL
    assert "exceed the static scratch" in str(ei.value)
