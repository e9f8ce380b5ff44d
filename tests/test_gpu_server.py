"""Job server (continuous batching): every job's result is the same alone and
in the mix, restarts start from their parent's converged result, and the
device-memory budget bounds admission."""
import os

import numpy as np
import pytest

from paper_2402_18311_gb300 import place, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    if not os.path.exists(place.LIB_PATH):
        from paper_2402_18311_gb300 import build
        build.build()
    place.lib()


def designs():
    return [synth.scaled(4000, 128, seed=11, name="a"), synth.scaled(9000, 128, seed=12, name="b"),
            synth.scaled(6000, 128, seed=13, name="c")]


def params():
    return place.place_default_params(tau_stop=0.15, max_iters=1500,
                                      dct_mode=place.PLACE_DCT_BF16X3)


def run_trace(max_active, budget=8 << 30, arrivals=(0.0, 0.0, 0.05, 0.0, 0.0, 0.1, 0.0)):
    ds = designs()
    s = place.Server(budget, max_active, iters_per_tick=16)
    try:
        ids = [s.submit(ds[0], params(), arrival_s=arrivals[0]),
               s.submit(ds[1], params(), arrival_s=arrivals[1]),
               s.submit(ds[2], params(), arrival_s=arrivals[2])]
        ids.append(s.submit(ds[0], params(), kind=place.PLACE_JOB_RESTART, parent=ids[0], seed=3,
                            arrival_s=arrivals[3]))
        ids.append(s.submit(ds[0], params(), kind=place.PLACE_JOB_RESTART, parent=ids[0], seed=4,
                            arrival_s=arrivals[4]))
        ids.append(s.submit(ds[1], params(), kind=place.PLACE_JOB_RESTART, parent=ids[1], seed=5,
                            arrival_s=arrivals[5]))
        ids.append(s.submit(ds[2], params(), kind=place.PLACE_JOB_RESTART, parent=ids[2], seed=6,
                            arrival_s=arrivals[6]))
        s.run(timeout_s=300)
        res = {r.id: r for r in s.results()}
        return res, s.stats()
    finally:
        s.close()


def test_results_identical_alone_and_in_the_mix():
    fifo, (peak_b1, peak_a1) = run_trace(1)
    mix, (peak_b, peak_a) = run_trace(8)
    assert peak_a1 == 1 and peak_a >= 2
    assert sorted(fifo) == sorted(mix) == list(range(7))
    for i in range(7):
        a, b = fifo[i], mix[i]
        assert a.hpwl == b.hpwl and a.overflow == b.overflow, i
        assert a.position_hash == b.position_hash, i
        assert a.iterations == b.iterations
        assert b.admit_s >= b.arrival_s - 1e-9 and b.done_s > b.admit_s
    # restarts begin after their parent finished
    for child, parent in ((3, 0), (4, 0), (5, 1), (6, 2)):
        assert mix[child].admit_s >= mix[parent].done_s - 1e-9
        assert fifo[child].converged == 1 or fifo[child].iterations == 1500


def test_placement_job_equals_plain_handle_run():
    res, _ = run_trace(4)
    d = designs()[1]
    h = place.place_create(d, params())
    try:
        conv = np.zeros(1, np.int32)
        while True:
            place.place_step(h, 16, conv)
            if conv[0]:
                break
        hp = np.empty(1); tv = np.empty(1)
        place.place_eval_hpwl_overflow(h, hp, tv)
        assert res[1].hpwl == hp[0] and res[1].overflow == tv[0]
    finally:
        place.place_destroy(h)


def test_budget_bounds_admission():
    ds = designs()
    need = max(place.place_estimate_device_bytes(d, params()) for d in ds)
    free, _ = run_trace(8)
    # room for one handle at a time: jobs run one after another, restarts adopt
    # their parent's resident handle, and nothing deadlocks
    budget = need + need // 5
    res, (peak_bytes, peak_active) = run_trace(8, budget=budget)
    assert len(res) == 7
    assert peak_bytes <= budget
    assert peak_active == 1
    for i in range(7):
        assert res[i].position_hash == free[i].position_hash
    # two handles at a time
    budget2 = 2 * need + need // 5
    res2, (peak_bytes2, peak_active2) = run_trace(8, budget=budget2)
    assert len(res2) == 7 and peak_bytes2 <= budget2 and 1 <= peak_active2 <= 2


def test_wiremask_restart_job_equals_plain_handle_run():
    # a restart job with the WireMask perturbation (Section 4.2) perturbs its
    # parent's converged result exactly as place_perturb on a plain handle
    d = synth.scaled(6000, 128, seed=14, name="m")
    rng = np.random.default_rng(14)
    mac = rng.choice(d.n_movable, 10, replace=False)
    d.w[mac] = rng.integers(6, 24, 10).astype(np.float32)
    d.h[mac] = rng.integers(6, 24, 10).astype(np.float32)
    d.x[mac] = np.minimum(d.x[mac], d.die[2] - d.w[mac]).astype(np.float32)
    d.y[mac] = np.minimum(d.y[mac], d.die[3] - d.h[mac]).astype(np.float32)
    d.is_macro[mac] = 1
    s = place.Server(8 << 30, 4, iters_per_tick=16)
    try:
        a = s.submit(d, params())
        b = s.submit(d, params(), kind=place.PLACE_JOB_RESTART, parent=a, op=place.PLACE_WIREMASK)
        s.run(timeout_s=300)
        res = {r.id: r for r in s.results()}
    finally:
        s.close()
    h = place.place_create(d, params())
    try:
        conv = np.zeros(1, np.int32)
        hp = np.empty(1); tv = np.empty(1)
        for phase in range(2):
            if phase == 1:
                place.place_perturb(h, place.PLACE_WIREMASK, 0.0, 0, 0)
                conv[:] = 0
            while not conv[0]:
                place.place_step(h, 16, conv)
            place.place_eval_hpwl_overflow(h, hp, tv)
            r = res[a if phase == 0 else b]
            assert r.hpwl == hp[0] and r.overflow == tv[0], phase
    finally:
        place.place_destroy(h)


def _alone(d, prm):
    s = place.Server(8 << 30, 1, iters_per_tick=16)
    try:
        s.submit(d, prm)
        s.run(timeout_s=300)
        return s.results()[0]
    finally:
        s.close()


def test_a_job_past_its_wall_clock_budget_expires_at_a_chunk_boundary():
    ds = designs()
    endless = place.place_default_params(tau_stop=-1.0, max_iters=10 ** 6,
                                         dct_mode=place.PLACE_DCT_BF16X3)
    s = place.Server(8 << 30, 4, iters_per_tick=16)
    try:
        a = s.submit(ds[0], params())
        b = s.submit(ds[1], endless, max_seconds=1e-6)  # over budget after its first chunk
        rb = s.submit(ds[1], params(), kind=place.PLACE_JOB_RESTART, parent=b, seed=5)
        s.run(timeout_s=300)
        res = {r.id: r for r in s.results()}
    finally:
        s.close()
    assert res[b].status == place.PLACE_JOB_EXPIRED and res[b].iterations == 16
    assert np.isfinite(res[b].hpwl) and res[b].position_hash != 0
    # the others run to their stop test, and the restart starts from b's positions
    assert res[a].status == res[rb].status == place.PLACE_JOB_FINISHED
    assert res[rb].converged == 1
    ra = _alone(ds[0], params())
    assert (res[a].position_hash, res[a].iterations) == (ra.position_hash, ra.iterations)


def test_cancelling_a_running_job_stops_it_and_leaves_the_others_alone():
    import threading
    import time
    ds = designs()
    endless = place.place_default_params(tau_stop=-1.0, max_iters=10 ** 6,
                                         dct_mode=place.PLACE_DCT_BF16X3)
    s = place.Server(8 << 30, 4, iters_per_tick=16)
    try:
        a = s.submit(ds[0], params())
        b = s.submit(ds[1], endless)
        rb = s.submit(ds[1], params(), kind=place.PLACE_JOB_RESTART, parent=b, seed=5)
        err = []
        t = threading.Thread(target=lambda: err.append(s.run(timeout_s=300)))
        t.start()
        time.sleep(1.0)
        s.cancel(b)  # from this thread while the server runs in the other
        t.join(timeout=300)
        assert not t.is_alive()
        res = {r.id: r for r in s.results()}
    finally:
        s.close()
    assert res[b].status == place.PLACE_JOB_CANCELLED
    assert 0 < res[b].iterations < 10 ** 6 and res[b].iterations % 16 == 0
    assert res[rb].status == place.PLACE_JOB_CANCELLED and res[rb].iterations == 0
    assert res[a].status == place.PLACE_JOB_FINISHED
    ra = _alone(ds[0], params())
    assert (res[a].position_hash, res[a].iterations) == (ra.position_hash, ra.iterations)


def test_cancelling_one_restart_of_a_resident_parent_leaves_the_other_alone():
    # the parent's handle stays resident for a restart with its parameters;
    # one of its two restarts is cancelled while queued, the other adopts the
    # handle and gives the result it gives without the cancelled one
    ds = designs()

    def trace(cancel):
        s = place.Server(8 << 30, 1, iters_per_tick=16)
        try:
            a = s.submit(ds[0], params())
            r1 = s.submit(ds[0], params(), kind=place.PLACE_JOB_RESTART, parent=a, seed=3)
            r2 = s.submit(ds[0], params(), kind=place.PLACE_JOB_RESTART, parent=a, seed=4)
            if cancel:
                s.cancel(r1)
            s.run(timeout_s=300)
            return {r.id: r for r in s.results()}, (a, r1, r2)
        finally:
            s.close()

    full, (a, r1, r2) = trace(False)
    part, _ = trace(True)
    assert part[r1].status == place.PLACE_JOB_CANCELLED and part[r1].iterations == 0
    for j in (a, r2):
        assert part[j].status == place.PLACE_JOB_FINISHED
        assert (part[j].position_hash, part[j].iterations) == (full[j].position_hash, full[j].iterations)
