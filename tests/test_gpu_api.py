"""Host-visible API calls beyond the parity path: borrowed device views of the
positions, stepping several handles at once, checkpoint and resume, and the
bounded waits' failure path."""
import numpy as np
import pytest

from paper_2402_18311_gb300 import place, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    if not os.path.exists(place.LIB_PATH):
        from paper_2402_18311_gb300 import build
        build.build()
    place.lib()


class _View:
    """A device array described by __cuda_array_interface__ (zero copy; the
    test only reads it, torch accepts no read-only flag)."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n, 2), "typestr": "<f4", "data": (ptr, False),
                                         "version": 3, "strides": None}


def _positions(h, n):
    x = np.empty(n, np.float32); y = np.empty(n, np.float32)
    place.place_get_positions(h, 0, x, y)
    return x, y


def test_device_views_alias_the_interleaved_positions():
    import torch
    d = synth.tiny_1k(0)
    h = place.place_create(d, place.place_default_params(tau_stop=-1.0, max_iters=100))
    try:
        place.place_step(h, 7)
        x, y = _positions(h, d.n_cells)
        px, py = place.place_device_views(h, 0)
        assert py == px + 4
        torch.cuda.synchronize()
        t = torch.as_tensor(_View(px, d.n_cells), device="cuda").cpu().numpy()
        np.testing.assert_array_equal(t[:, 0], x)
        np.testing.assert_array_equal(t[:, 1], y)
        with pytest.raises(place.PlaceError):
            place.place_device_views(h, 1)  # one copy only
    finally:
        place.place_destroy(h)


def test_step_multi_equals_separate_steps():
    import torch
    designs = [synth.tiny_1k(0), synth.scaled(5000, 64, seed=4)]
    prm = place.place_default_params(tau_stop=-1.0, max_iters=1000)
    streams = [torch.cuda.Stream() for _ in designs]
    multi = [place.place_create(d, prm, stream=s.cuda_stream) for d, s in zip(designs, streams)]
    solo = [place.place_create(d, prm) for d in designs]
    try:
        conv = np.full(2, -1, np.int32)
        place.place_step_multi(multi, 60, conv)
        assert conv.tolist() == [0, 0]
        for h in solo:
            place.place_step(h, 60)
        for d, hm, hs in zip(designs, multi, solo):
            xm, ym = _positions(hm, d.n_cells)
            xs, ys = _positions(hs, d.n_cells)
            np.testing.assert_array_equal(xm, xs)
            np.testing.assert_array_equal(ym, ys)
    finally:
        for h in multi + solo:
            place.place_destroy(h)
        torch.cuda.synchronize()


def test_bounded_waits_give_up_and_the_handle_stays_usable():
    # The tensor-core GEMM's waits on its shared-memory barriers are bounded.
    # With its copy producer idle no tile ever lands: the waits give up after
    # about a second, the kernel frees its tensor memory and raises the error
    # flag, the call reports PLACE_ETIMEOUT, and the handle then places exactly
    # like a handle that never saw the failure.
    d = synth.scaled(2000, 128, seed=1)
    prm = place.place_default_params(tau_stop=-1.0, max_iters=1000)
    h = place.place_create(d, prm)
    ref = place.place_create(d, prm)
    try:
        assert place.place_get_info(h).dct_mode == place.PLACE_DCT_BF16X3
        assert place.place_test_wait_timeout(h) == place.PLACE_ETIMEOUT
        assert "gave up" in place.place_last_error()
        place.place_step(h, 30)
        place.place_step(ref, 30)
        conv = np.zeros(1, np.int32)
        place.place_step(h, 0, conv)  # reads the error flag: clear
        x, y = _positions(h, d.n_cells)
        rx, ry = _positions(ref, d.n_cells)
        np.testing.assert_array_equal(x, rx)
        np.testing.assert_array_equal(y, ry)
    finally:
        place.place_destroy(h)
        place.place_destroy(ref)
    # a handle on the FP32 path has no such wait to test
    d = synth.tiny_1k(0)
    h = place.place_create(d, place.place_default_params())
    try:
        assert place.place_test_wait_timeout(h) == place.PLACE_EINVAL
    finally:
        place.place_destroy(h)


def _resume_case(d, prm, first, rest, copy=0):
    """Run first + rest iterations straight, and first, checkpoint, rest on a
    new handle from the checkpoint: positions, state and history agree bit
    for bit."""
    a = place.place_create(d, prm)
    b = place.place_create(d, prm)
    try:
        place.place_step(a, first)
        buf = place.place_checkpoint_save(a, copy)
        assert buf.size == place.place_checkpoint_bytes(a)
        place.place_step(a, rest)
        place.place_checkpoint_load(b, copy, buf)
        place.place_step(b, rest)
        n = d.n_cells
        xa = np.empty(n, np.float32); ya = np.empty(n, np.float32)
        xb = np.empty(n, np.float32); yb = np.empty(n, np.float32)
        place.place_get_positions(a, copy, xa, ya)
        place.place_get_positions(b, copy, xb, yb)
        np.testing.assert_array_equal(xa, xb)
        np.testing.assert_array_equal(ya, yb)
        sa, sb = place.place_get_state(a, copy), place.place_get_state(b, copy)
        for f in ("iter", "converged", "stopped", "backtracks", "lambda_", "gamma", "alpha", "a",
                  "overflow", "hpwl_wa", "bins_effective"):
            assert getattr(sa, f) == getattr(sb, f), f
        ha = [(r.iter, r.hpwl_wa, r.overflow, r.lambda_) for r in place.place_get_history(a, copy)]
        hb = [(r.iter, r.hpwl_wa, r.overflow, r.lambda_) for r in place.place_get_history(b, copy)]
        assert ha == hb and len(ha) > 0
        if place.place_get_info(a).n_fillers:
            fa, fb = place.place_get_fillers(a, copy), place.place_get_fillers(b, copy)
            np.testing.assert_array_equal(fa[0], fb[0])
            np.testing.assert_array_equal(fa[1], fb[1])
        return sa
    finally:
        place.place_destroy(a)
        place.place_destroy(b)


def test_checkpoint_resume_is_bit_exact_fp32_path():
    d = synth.tiny_1k(0)
    st = _resume_case(d, place.place_default_params(tau_stop=-1.0, max_iters=10 ** 6), 90, 110)
    assert st.iter == 200


def test_checkpoint_resume_is_bit_exact_tensor_core_path_with_knobs():
    # BF16x3 spectral path, fillers, backtracking: every array the knobs add
    d = synth.scaled(20000, 128, seed=2)
    prm = place.place_default_params(tau_stop=-1.0, max_iters=10 ** 6, fillers=1,
                                     max_backtracks=2, n_copies=2)
    _resume_case(d, prm, 75, 80, copy=1)


def test_checkpoint_rejects_another_design_and_short_buffers():
    d1, d2 = synth.tiny_1k(0), synth.tiny_1k(1)
    prm = place.place_default_params(tau_stop=-1.0, max_iters=100)
    a = place.place_create(d1, prm)
    try:
        buf = place.place_checkpoint_save(a, 0)
        with pytest.raises(place.PlaceError):
            place.place_checkpoint_load(a, 0, buf[:-8])
        with pytest.raises(place.PlaceError):
            place.place_checkpoint_load(a, 1, buf)  # one copy only
        other = place.place_create(d2, place.place_default_params(tau_stop=-1.0, max_iters=100,
                                                                   hpwl_ref=0.5))
        try:
            with pytest.raises(place.PlaceError):
                place.place_checkpoint_load(other, 0, buf)  # another lambda reference step
        finally:
            place.place_destroy(other)
        place.place_checkpoint_load(a, 0, buf)  # its own checkpoint loads
    finally:
        place.place_destroy(a)


def test_wa_floor_measurement_leaves_the_placement_unchanged():
    # The gather-and-reduce floor of the WA stage adds into the gradient sums
    # and clears them again: a placement measured between two steps goes on
    # bit for bit as one that was not.
    d = synth.scaled(20000, 128, seed=2)
    out = []
    for measure in (False, True):
        h = place.place_create(d, place.place_default_params(tau_stop=-1.0, max_iters=10 ** 6))
        try:
            place.place_step(h, 20)
            if measure:
                assert place.place_measure_wa_floor(h, 5) > 0
            place.place_step(h, 20)
            out.append(_positions(h, d.n_cells))
        finally:
            place.place_destroy(h)
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_scatter_floor_measurement_leaves_the_map_to_the_next_pass():
    d = synth.scaled(20000, 128, seed=2)
    h = place.place_create(d, place.place_default_params(tau_stop=-1.0, max_iters=10 ** 6))
    try:
        place.place_step(h, 300)
        m0 = np.empty(d.nx * d.ny, np.int64)
        place.place_eval_density(h, 0, m0)
        t_scatter, t_floor = place.place_measure_scatter_floor(h, 5)
        assert t_scatter > 0 and t_floor > 0
        m1 = np.empty(d.nx * d.ny, np.int64)
        place.place_eval_density(h, 0, m1)
        np.testing.assert_array_equal(m0, m1)
        place.place_step(h, 5)  # and the placement goes on
    finally:
        place.place_destroy(h)
