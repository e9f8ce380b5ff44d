"""Benchmark of the electrostatic global-placement inner loop on GB300.

One step = one Nesterov iteration of Eq. 2 over the whole hot path: density
scatter and overflow, the spectral Poisson solve, WA wirelength and
gradients (Eq. 3), per-cell gradient assembly, preconditioned
Nesterov/Lipschitz update, all copies of the design (the global-placement
step of Algorithm 1).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload large_2m|medium_210k|tiny_1k]

Prints one JSON line (rank 0).  For N > 1 (torchrun) every rank places its own
replica of the design: the design does not shard (the density map and the
Poisson solve are global per iteration), so the ranks are independent and
``value`` is the sum of their iterations/s (weak scaling, no collective on
the data path).

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the
same workload (host cores of this machine).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2402_18311_gb300 import synth  # noqa: E402

METRIC = "Nesterov iters/s @2M cells"
WORKLOADS = {
    "large_2m": (synth.large_2m, "2.1M movable cells, 60 fixed macros (30% area), 2.2M nets "
                 "(12.0M pins, max degree 5000), 4096x4096 die, 1024x1024 bins, t=0.7"),
    "medium_210k": (synth.medium_210k, "210k movable cells, 10 fixed macros (20% area), 220k "
                    "nets (1.18M pins), 2000x2000 die, 512x512 bins, t=0.9"),
    "tiny_1k": (synth.tiny_1k, "1k movable cells, 16 pads, 1.1k nets, 256x256 die, 64x64 bins, t=1.0"),
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def stage_traffic(stage, workload):
    """DRAM bytes of one pass of `stage` from the committed ncu capture
    (profiles/traffic_<workload>.txt), or None when there is none or the
    stage's kernel source changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.txt")
    if not os.path.exists(path):
        return None
    total, found, sha_ok = 0, False, True
    for line in open(path):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "sha" and f[1] == stage:
            src = os.path.join(ROOT, "paper_2402_18311_gb300", "csrc", f[2])
            cur = hashlib.sha1(open(src, "rb").read()).hexdigest() if os.path.exists(src) else ""
            sha_ok = sha_ok and cur == f[3]
        elif f[0] == stage and len(f) == 3:
            total += int(f[2])
            found = True
    return total if (found and sha_ok) else None


def aggregate_ranks(ms, steps, world, device="cpu"):
    """Whole-job throughput of replicas: every rank ran `steps` iterations of
    its own copy of the design; the job took the slowest rank's time."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * steps / (ms_max / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def algorithmic(d, info):
    """Algorithmic bytes / flops of one iteration per stage (one copy)."""
    C, P, E, G = d.n_movable, d.n_pins, d.n_nets, d.nx * d.ny
    n_all = d.n_cells
    return {
        # scatter: x, y, W, H per cell (16 B), map clear + atomics 8 B/bin written,
        # finish: map + fixed map read 16 B/bin, rho written 4 B/bin
        "density": {"bytes": 16 * C + 8 * G + 16 * G + 4 * G},
        # six M^3-type GEMMs (two per 2D transform: forward, Ex, Ey); on the
        # tensor pipe: three bf16 products each (BF16x3), and half the
        # contraction with the even/odd split of every transform
        "spectral": {"flops": 2.0 * (2 * d.ny * d.ny * d.nx + 2 * d.nx * d.nx * d.ny) * 1.5,
                     "flops_pipe": (2.0 * (2 * d.ny * d.ny * d.nx + 2 * d.nx * d.nx * d.ny) * 1.5
                                    * (3 if info.dct_mode == 1 else 1)
                                    * (0.5 if getattr(info, "dct_fold", 0) else 1.0))},
        # pin_cell 4 + offsets 8 per pin, net_ptr 4 per net, positions 8 per
        # cell (gathered once), the packed gradient sum 8 per movable cell
        # (accumulated in L2 by 64-bit reductions, written once)
        "wirelength": {"bytes": 12 * P + 4 * E + 8 * n_all + 8 * C},
        # per cell: gradient sum read 8 + cleared 8, position 8, sizes 8,
        # field 8, pins/area 8, previous gradient 8, gradient written 8 (the
        # raw gradients are written only at k = 0)
        "cellgrad": {"bytes": 64 * C},
        # read w, h 8, v 8, u 8, g 8; write u 8, v 8 per cell (the step norm
        # |v_{k+1} - v_k| is reduced here, so v_k is not stored)
        "update": {"bytes": 48 * C},
    }


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2402_18311_gb300 import build, place
    if not os.path.exists(place.LIB_PATH):
        if rank == 0:
            build.build()
        if world > 1:
            torch.distributed.barrier()
    maker, desc = WORKLOADS[args.workload]
    d = maker(0)
    prm = place.place_default_params(tau_stop=-1.0, max_iters=1 << 30, dct_mode=args.dct,
                                     autotune=args.autotune)
    stream = torch.cuda.current_stream()
    h = place.place_create(d, prm, stream=stream.cuda_stream)
    info = place.place_get_info(h)

    # untimed iterations to a later phase of the placement (profiling), then
    # the warm-up (which also captures the iteration graph)
    if args.advance > 0:
        place.place_step(h, args.advance)
    place.place_step(h, args.warmup)
    torch.cuda.synchronize()

    # device-timed steps: inputs resident in HBM
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    place.place_step(h, args.steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    clocks = clk.stop()

    # per-stage device time (same kernels, launched stage by stage with events)
    stage_ms = np.zeros(5, np.float32)
    nprof = max(3, min(args.steps, 20))
    place.place_step_timed(h, nprof, stage_ms)
    stage_ms /= nprof
    # the WA stage's gather-and-reduce floor on this netlist: only the pin
    # streams, one position gather and one 64-bit reduction per pin
    wa_floor_ms = place.place_measure_wa_floor(h, 10)

    # end to end through the C ABI with pinned host buffers: every step uploads
    # the movable positions (place_set_positions, which restarts the optimiser
    # from them), runs one iteration and reads back all positions
    xs = torch.empty(d.n_cells, dtype=torch.float32).pin_memory()
    ys = torch.empty(d.n_cells, dtype=torch.float32).pin_memory()
    place.place_get_positions(h, 0, xs, ys)
    n_e2e = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        place.place_set_positions(h, 0, xs, ys)
        place.place_step(h, 1)
        place.place_get_positions(h, 0, xs, ys)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0

    hp = np.empty(prm.n_copies)
    tv = np.empty(prm.n_copies)
    place.place_eval_hpwl_overflow(h, hp, tv)
    place.place_destroy(h)

    full = None
    if not args.no_full_run and world == 1:
        full = run_full(args, place, torch, d, stream)
    configs = None
    if not args.no_configs and world == 1:
        configs = run_configs(args, place, torch)

    restarts = None
    if not args.no_restarts:
        restarts = run_restarts(args, place, torch)
        restarts["hybro_wiremask"] = run_wiremask(args, place, torch)
    serving = None
    if args.serving_jobs > 0:
        serving = run_serving(args, place, args.serving_jobs, 10_000, args.serving_max_cells)

    ms_max, value = aggregate_ranks(ms, args.steps, world, device="cuda")
    e2e_v = world * n_e2e / e2e_s

    alg = algorithmic(d, info)
    pk, pk_kind = peaks()
    names = ["density", "spectral", "wirelength", "cellgrad", "update"]
    dom = int(np.argmax(stage_ms))
    per = {}
    for i, n in enumerate(names):
        a = alg[n]
        sec = float(stage_ms[i]) / 1e3
        if "flops" in a:
            per[n] = {"ms": float(stage_ms[i]), "TFLOP/s": a["flops"] / sec / 1e12 if sec > 0 else None}
            if info.dct_mode == 1 and sec > 0:
                # what the tensor pipe executed, against the measured bf16 peak
                per[n]["pipe_TFLOP/s"] = a["flops_pipe"] / sec / 1e12
                per[n]["pipe_frac_of_bf16"] = a["flops_pipe"] / sec / 1e12 / pk["bf16_tflops"]
                per[n]["dct_fold"] = int(info.dct_fold)
        else:
            per[n] = {"ms": float(stage_ms[i]), "GB/s": a["bytes"] / sec / 1e9 if sec > 0 else None}
    dn = names[dom]
    sec = float(stage_ms[dom]) / 1e3
    if dn == "spectral":
        if args.dct == 1:
            peak = pk["bf16_tflops"]
            unit, bound = "TFLOP/s", "tensor"
            achieved = alg[dn]["flops_pipe"] / sec / 1e12
            peak_note = f"bf16 dense ({pk_kind}, burst); 3 bf16 products per GEMM (BF16x3)"
        else:
            # FP32 FMA on CUDA cores: 152 SMs x 128 lanes x 2 flop x max clock
            peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            unit, bound = "TFLOP/s", "alu"
            achieved = alg[dn]["flops"] / sec / 1e12
            peak_note = "FP32 CUDA-core peak from 152 SMs x 128 FMA lanes x max SM clock"
    else:
        peak = pk["hbm_gbs"]
        unit, bound = "GB/s", "hbm"
        achieved = alg[dn]["bytes"] / sec / 1e9
        peak_note = f"HBM copy bandwidth ({pk_kind})"
    roofline = {"kernel": dn, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": stage_traffic(dn, args.workload),
                "algorithmic": alg[dn], "peak_source": peak_note, "stages": per,
                "traffic_note": "DRAM bytes of one pass of the stage from the committed ncu "
                                "capture (cold L2), null if the kernel source changed since"}
    if dn == "wirelength" and wa_floor_ms > 0:
        # random 32-byte sector accesses in L2, not HBM bytes, bound this
        # index stream: the floor's rate is what the stage can approach
        roofline["floor"] = {"ms": wa_floor_ms,
                             "GB/s": alg[dn]["bytes"] / (wa_floor_ms / 1e3) / 1e9,
                             "stage_frac_of_floor_rate": wa_floor_ms / float(stage_ms[dom]),
                             "what": "place_measure_wa_floor: pin streams, one random position "
                                     "gather and one random 64-bit reduction per pin"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(d, args)
    out = {
        "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.dct == 0 else "f32+bf16x3", "data": "synthetic",
        "config": {"workload": args.workload, "desc": desc, "copies_per_gpu": prm.n_copies,
                   "parallelism": f"replicas{world}", "l2": "inputs larger than L2 "
                   "(per-iteration working set > 129 MB)" if args.workload == "large_2m"
                   else "working set fits L2 (no flush)",
                   "dct_mode": ["fp32", "bf16x3"][args.dct], "tuning": tuning(info),
                   "timed_iterations": [args.advance + args.warmup + 1,
                                        args.advance + args.warmup + args.steps]},
        "e2e": {"value": e2e_v, "unit": "iters/s",
                "h2d_bytes_per_step": 8 * d.n_movable, "d2h_bytes_per_step": 8 * d.n_cells,
                "note": "per step: set_positions (h2d, restarts the optimiser) + 1 iteration "
                        "+ get_positions (d2h), pinned host buffers"},
        "gpu_launches": int(info.kernels_per_iter) * args.steps,
        "roofline": roofline,
        "clocks": clocks,
        "final_hpwl": float(hp[0]), "final_overflow": float(tv[0]),
    }
    if cpu is not None:
        out["cpu_baseline"] = cpu
    if full is not None:
        out["full_run"] = full
    if configs is not None:
        out["configs"] = configs
    if restarts is not None:
        out["restarts"] = restarts
    if serving is not None:
        out["serving"] = serving
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def tuning(info):
    """The kernel variants a handle runs with (chosen by the autotuner or the
    fixed rules)."""
    return {"autotuned": bool(info.autotuned), "autotune_ms": info.autotune_ms,
            "gemm_bn": list(info.gemm_bn), "gemm_split": list(info.gemm_split),
            "wa_big_cap": info.wa_big_cap, "wa_streams": info.wa_streams,
            "scatter_thresholds": [info.scatter_t1, info.scatter_t2]}


def _stage_sample(place, h, n=5):
    """Mean per-stage device time (ms) of n iterations run stage by stage
    (place_step_timed advances the placement like place_step)."""
    st = np.zeros(5, np.float32)
    place.place_step_timed(h, n, st)
    return {k: float(v / n) for k, v in zip(place.PLACE_STAGES, st)}


def run_full(args, place, torch, d, stream, tau_stop=0.07, max_iters=4000, chunk=100,
             samples=(5, 155, 305, 505, 805, 1205)):
    """A whole placement of the headline workload from its centred start: to
    overflow <= tau_stop or max_iters iterations, with the library's default
    parameters.  Reports the average rate over the run, the rate of each chunk
    of iterations, and per-stage times sampled at several phases (5
    iterations each, included in the run)."""
    prm = place.place_default_params(tau_stop=tau_stop, max_iters=max_iters, dct_mode=args.dct)
    hpwl_ref = prm.hpwl_ref
    h = place.place_create(d, prm, stream=stream.cuda_stream)
    conv = np.zeros(1, np.int32)
    chunks, stages = [], {}
    scatter_floor = None
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    done, total_ms = 0, 0.0
    torch.cuda.synchronize()
    while done < max_iters:
        nxt = min([k for k in samples if k >= done] + [max_iters])
        if nxt == done:  # a stage sample here
            stages[str(done)] = _stage_sample(place, h)
            if done == samples[-1]:
                # the scatter against its floor (same loads, one 64-bit
                # reduction per covered bin) once the cells have spread
                sc, fl = place.place_measure_scatter_floor(h, 10)
                scatter_floor = {"iteration": done, "scatter_ms": sc, "floor_ms": fl}
            done += 5
            place.place_step(h, 0, conv)
            if conv[0]:
                break
            continue
        n = min(chunk, nxt - done)
        ev[0].record(stream)
        place.place_step(h, n)
        ev[1].record(stream)
        ev[1].synchronize()
        ms = ev[0].elapsed_time(ev[1])
        place.place_step(h, 0, conv)
        st = place.place_get_state(h, 0)
        ran = st.iter - done
        total_ms += ms
        chunks.append({"from": done, "iters": ran, "ms_per_iter": ms / max(ran, 1),
                       "overflow": st.overflow, "bins_effective": st.bins_effective})
        done = st.iter
        if conv[0]:
            break
    st = place.place_get_state(h, 0)
    hp = np.empty(1); tv = np.empty(1)
    place.place_eval_hpwl_overflow(h, hp, tv)
    place.place_destroy(h)
    graph_iters = sum(c["iters"] for c in chunks)
    return {"workload": args.workload, "tau_stop": tau_stop, "max_iters": max_iters,
            "hpwl_ref": round(float(hpwl_ref), 6),
            "iterations": int(st.iter), "converged": bool(st.converged),
            "final_overflow": float(tv[0]), "final_hpwl": float(hp[0]),
            "avg_iters_per_s": 1e3 * graph_iters / total_ms if total_ms > 0 else None,
            "timed_iterations": graph_iters,
            "note": "graph-launched iterations timed with CUDA events chunk by chunk; the "
                    "stage samples (place_step_timed, 5 iterations each) are part of the run "
                    "but not of the average",
            "chunks": chunks, "stage_ms_at_iteration": stages, "scatter_floor": scatter_floor}


def run_configs(args, place, torch):
    """The small and medium workloads as their configurations state them: the
    1k-cell design for 300 iterations then one Shuffle (all) round of 300 more
    (Algorithm 1 with one perturbation), and the 210k-cell design until
    overflow <= 0.07 or 1,000 iterations."""
    out = {}
    d = synth.tiny_1k(0)
    h = place.place_create(d, place.place_default_params(tau_stop=-1.0, max_iters=300,
                                                         dct_mode=place.PLACE_DCT_AUTO))
    info = place.place_get_info(h)
    bh = np.empty(1); bt = np.empty(1); br = np.empty(1, np.int32)
    place.place_step(h, 1)  # graph capture outside the timed region
    place.place_set_positions(h, 0, d.x, d.y)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    place.place_hybro(h, 1, place.PLACE_SHUFFLE_ALL, 0.5, 0, 0.1, bh, bt, br)
    el = time.perf_counter() - t0
    rh, rt = place.place_get_hybro_rounds(h, 0)
    place.place_destroy(h)
    out["tiny_1k"] = {"desc": WORKLOADS["tiny_1k"][1], "iterations": 600, "seconds": el,
                      "iters_per_s": 600 / el, "spectral": ["fp32", "bf16x3"][info.dct_mode],
                      "round_hpwl": rh.tolist(), "round_overflow": rt.tolist(),
                      "best_round": int(br[0]), "best_hpwl": float(bh[0]),
                      "note": "300 iterations, Shuffle (all) p = 0.5 seed 0, 300 more; host "
                              "wall time with the evaluations and the perturbation"}
    d = synth.medium_210k(0)
    h = place.place_create(d, place.place_default_params(tau_stop=0.07, max_iters=1000,
                                                         dct_mode=args.dct))
    info = place.place_get_info(h)
    place.place_step(h, 1)
    place.place_set_positions(h, 0, d.x, d.y)
    conv = np.zeros(1, np.int32)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    while not conv[0]:
        place.place_step(h, 50, conv)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    st = place.place_get_state(h, 0)
    hp = np.empty(1); tv = np.empty(1)
    place.place_eval_hpwl_overflow(h, hp, tv)
    place.place_destroy(h)
    out["medium_210k"] = {"desc": WORKLOADS["medium_210k"][1], "iterations": int(st.iter),
                          "converged": bool(st.converged), "seconds": ms / 1e3,
                          "iters_per_s": 1e3 * st.iter / ms, "final_overflow": float(tv[0]),
                          "final_hpwl": float(hp[0]),
                          "spectral": ["fp32", "bf16x3"][info.dct_mode],
                          "note": "to overflow <= 0.07 or 1,000 iterations, CUDA events around "
                                  "the whole run (50-iteration launches, stop flags read back)"}
    return out


def run_restarts(args, place, torch, K=32, p=0.5):
    """Batched Hybro restarts (Algorithm 1, a population of perturbations of
    one converged solution): K Shuffle (all) perturbations of the 210k-cell
    design with seeds 0..K-1, re-optimised until every copy meets the overflow
    target, as one K-copy handle against K sequential single-copy runs.  Also
    the paper's baseline of independent runs from K random starts (batched)."""
    d = synth.medium_210k(0)
    mk = lambda k: place.place_default_params(tau_stop=0.07, max_iters=3000, dct_mode=args.dct,
                                              n_copies=k)

    def until_done(h, k):
        conv = np.zeros(k, np.int32)
        while True:
            place.place_step(h, 50, conv)
            if conv.all():
                return

    h1 = place.place_create(d, mk(1))
    until_done(h1, 1)
    x0 = torch.empty(d.n_cells, dtype=torch.float32, device="cuda")
    y0 = torch.empty(d.n_cells, dtype=torch.float32, device="cuda")
    place.place_get_positions(h1, 0, x0, y0)
    base_hp = np.empty(1); base_tau = np.empty(1)
    place.place_eval_hpwl_overflow(h1, base_hp, base_tau)
    # batched: one handle, K copies in one captured graph per iteration
    hb = place.place_create(d, mk(K))
    tune_b = tuning(place.place_get_info(hb))
    place.place_step(hb, 1)  # capture the graph outside the timed region
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    place.place_set_positions(hb, -1, x0, y0)
    place.place_perturb(hb, place.PLACE_SHUFFLE_ALL, p, 0, -1)
    until_done(hb, K)
    hp_b = np.empty(K); tau_b = np.empty(K)
    place.place_eval_hpwl_overflow(hb, hp_b, tau_b)
    t_b = time.perf_counter() - t0
    iters_b = [place.place_get_state(hb, c).iter for c in range(K)]
    place.place_destroy(hb)
    # serial: the same K restarts one at a time on a single-copy handle
    hp_s = np.empty(K); tau_s = np.empty(K)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in range(K):
        place.place_set_positions(h1, 0, x0, y0)
        place.place_perturb(h1, place.PLACE_SHUFFLE_ALL, p, c, 0)
        until_done(h1, 1)
        a = np.empty(1); b = np.empty(1)
        place.place_eval_hpwl_overflow(h1, a, b)
        hp_s[c], tau_s[c] = a[0], b[0]
    t_s = time.perf_counter() - t0
    place.place_destroy(h1)
    # the paper's baseline, independent runs ("multiple DMP"): K copies from
    # independent random centred starts of the same netlist, batched the
    # same way, to the same overflow target
    hr = place.place_create(d, mk(K))
    place.place_step(hr, 1)
    starts = [synth.random_start(d, 1000 + c) for c in range(K)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c, (xr, yr) in enumerate(starts):
        place.place_set_positions(hr, c, xr, yr)
    until_done(hr, K)
    hp_r = np.empty(K); tau_r = np.empty(K)
    place.place_eval_hpwl_overflow(hr, hp_r, tau_r)
    t_r = time.perf_counter() - t0
    iters_r = [place.place_get_state(hr, c).iter for c in range(K)]
    place.place_destroy(hr)
    br = int(np.argmin(np.where(tau_r <= 0.1, hp_r, np.inf)))
    bb, bs = int(np.argmin(np.where(tau_b <= 0.1, hp_b, np.inf))), int(np.argmin(np.where(tau_s <= 0.1, hp_s, np.inf)))
    return {"workload": "medium_210k: 210k cells, 220k nets, 512x512 bins, t=0.9",
            "copies": K, "operator": "Shuffle (all)", "p": p, "tau_stop": 0.07,
            "tuning_batched": tune_b,
            "batched_restarts_per_s": K / t_b, "serial_restarts_per_s": K / t_s,
            "speedup": t_s / t_b, "batched_s": t_b, "serial_s": t_s,
            "iters_per_restart_mean": float(np.mean(iters_b)),
            "best_hpwl_batched": float(hp_b[bb]), "best_hpwl_serial": float(hp_s[bs]),
            "best_overflow_batched": float(tau_b[bb]),
            "max_rel_hpwl_diff_batched_vs_serial": float(np.max(np.abs(hp_b - hp_s) / hp_s)),
            "start_hpwl": float(base_hp[0]), "start_overflow": float(base_tau[0]),
            "random_starts": {"copies": K, "seeds": "1000..%d" % (999 + K),
                              "runs_per_s": K / t_r, "seconds": t_r,
                              "iters_per_run_mean": float(np.mean(iters_r)),
                              "best_hpwl": float(hp_r[br]), "best_overflow": float(tau_r[br]),
                              "median_hpwl": float(np.median(hp_r)),
                              "hybro_best_over_random_best": float(hp_b[bb] / hp_r[br])}}


def run_wiremask(args, place, torch, rounds=3, reps=5):
    """Hybro-WireMask (Algorithm 1 with the WireMask perturbation of Section
    4.2) on the mixed-size 210k-cell design with 32 movable macros.  Measures
    one WireMask pass on a converged placement, then `rounds` Hybro rounds
    with WireMask and with Shuffle (all) (p = 0.5) from that placement, on
    one copy, with the best HPWL of each."""
    d = synth.medium_mixed_210k(0)
    prm = place.place_default_params(tau_stop=0.07, max_iters=3000, dct_mode=args.dct, n_copies=1)
    h = place.place_create(d, prm)
    conv = np.zeros(1, np.int32)
    while not conv.all():
        place.place_step(h, 50, conv)
    x0 = torch.empty(d.n_cells, dtype=torch.float32, device="cuda")
    y0 = torch.empty(d.n_cells, dtype=torch.float32, device="cuda")
    place.place_get_positions(h, 0, x0, y0)
    hp0 = np.empty(1); tau0 = np.empty(1)
    place.place_eval_hpwl_overflow(h, hp0, tau0)
    # the first pass allocates the scratch; the timed passes each restore the
    # converged placement (a device copy plus an optimiser reset) and run
    # WireMask (four launches per macro)
    place.place_set_positions(h, 0, x0, y0)
    place.place_perturb(h, place.PLACE_WIREMASK, 0.0, 0, 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        place.place_set_positions(h, 0, x0, y0)
        place.place_perturb(h, place.PLACE_WIREMASK, 0.0, 0, 0)
    torch.cuda.synchronize()
    t_wm = (time.perf_counter() - t0) / reps
    hp1 = np.empty(1); tau1 = np.empty(1)
    place.place_eval_hpwl_overflow(h, hp1, tau1)
    out = {"workload": "medium_mixed_210k: medium_210k with 32 movable macros of 16-64 units",
           "macros": int(d.is_macro[:d.n_movable].sum()), "grid": f"{d.nx}x{d.ny}",
           "wiremask_pass_ms": 1e3 * t_wm, "launches_per_pass": 4 * 32,
           "converged_hpwl": float(hp0[0]), "converged_overflow": float(tau0[0]),
           "hpwl_after_wiremask": float(hp1[0]), "rounds": rounds}
    for name, op, p in (("wiremask", place.PLACE_WIREMASK, 0.0),
                        ("shuffle_all", place.PLACE_SHUFFLE_ALL, 0.5)):
        place.place_set_positions(h, 0, x0, y0)
        bh = np.empty(1); bt = np.empty(1); br = np.empty(1, np.int32)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        place.place_hybro(h, rounds, op, p, 0, 0.1, bh, bt, br)
        out[name] = {"best_hpwl": float(bh[0]), "best_overflow": float(bt[0]),
                     "best_round": int(br[0]), "seconds": time.perf_counter() - t0}
    place.place_destroy(h)
    return out


def serving_trace(n_jobs, min_cells, max_cells, seed=0):
    """Jobs of the serving workload: designs of log-uniform size, grid
    clamp(2^round(log2 sqrt(C)), 128, 1024), target density U[0.7, 1.0];
    half placement jobs and half restarts of an earlier placement job."""
    import math
    rng = np.random.default_rng(seed)
    jobs, designs = [], []
    for i in range(n_jobs):
        if i > 0 and rng.random() < 0.5 and any(j[0] == "place" for j in jobs):
            parents = [k for k, j in enumerate(jobs) if j[0] == "place"]
            par = int(rng.choice(parents))
            jobs.append(("restart", jobs[par][1], par, int(rng.integers(0, 2 ** 31))))
        else:
            c = int(round(math.exp(rng.uniform(math.log(min_cells), math.log(max_cells)))))
            g = int(min(1024, max(128, 2 ** round(math.log2(math.sqrt(c))))))
            t = float(rng.uniform(0.7, 1.0))
            designs.append(synth.scaled(c, g, seed=int(rng.integers(0, 2 ** 31)),
                                        target_density=t, name=f"job{i}"))
            jobs.append(("place", len(designs) - 1, -1, 0))
    return jobs, designs


def run_serving(args, place, n_jobs, min_cells, max_cells, max_active=16):
    """Continuous batching against one job at a time on the same Poisson
    arrival trace (rate 0.8 x the measured one-at-a-time service rate)."""
    jobs, designs = serving_trace(n_jobs, min_cells, max_cells)
    prm = place.place_default_params(tau_stop=0.1, max_iters=2000, dct_mode=args.dct)
    budget = 64 << 30

    def run(slots, arrivals):
        srv = place.Server(budget, slots, iters_per_tick=32)
        try:
            for (kind, di, par, seed), a in zip(jobs, arrivals):
                if kind == "place":
                    srv.submit(designs[di], prm, arrival_s=a)
                else:
                    srv.submit(designs[di], prm, kind=place.PLACE_JOB_RESTART, parent=par,
                               seed=seed, arrival_s=a)
            span = srv.run(timeout_s=600)
            res = srv.results()
            return span, res, srv.stats()
        finally:
            srv.close()

    span0, res0, st0 = run(1, [0.0] * n_jobs)
    rate = 0.8 * n_jobs / span0
    gaps = np.random.default_rng(1).exponential(1.0 / rate, n_jobs)
    arrivals = np.cumsum(gaps) - gaps[0]
    out = {"jobs": n_jobs, "cells": [min_cells, max_cells], "arrival_rate_per_s": rate,
           "fifo_service_rate_per_s": n_jobs / span0, "tau_stop": 0.1}
    for name, slots in (("fifo", 1), ("batched", max_active)):
        span, res, (peak_b, peak_a) = run(slots, arrivals)
        lat = np.array([r.done_s - r.arrival_s for r in res]) * 1e3
        iters = sum(r.iterations for r in res)
        out[name] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "mean_ms": float(lat.mean()), "makespan_s": span,
                     "agg_iters_per_s": iters / span, "peak_active": peak_a,
                     "peak_device_bytes": peak_b, "max_active": slots}
        out.setdefault("_hash", {})[name] = [int(r.position_hash) for r in res]
    # saturated: every job arrives at t = 0, so throughput, not arrivals,
    # decides the makespan (the one-at-a-time run is the calibration run above)
    spanb, resb, (peak_b, peak_a) = run(max_active, [0.0] * n_jobs)
    sat = {}
    for name, span, res in (("fifo", span0, res0), ("batched", spanb, resb)):
        iters = sum(r.iterations for r in res)
        lat = np.array([r.done_s - r.arrival_s for r in res]) * 1e3
        sat[name] = {"makespan_s": span, "agg_iters_per_s": iters / span,
                     "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}
    sat["throughput_gain"] = sat["batched"]["agg_iters_per_s"] / sat["fifo"]["agg_iters_per_s"]
    sat["peak_active"] = peak_a
    out["saturated"] = sat
    h = out.pop("_hash")
    out["results_identical"] = (h["fifo"] == h["batched"]
                                and [int(r.position_hash) for r in res0] == h["fifo"]
                                and [int(r.position_hash) for r in resb] == h["fifo"])
    return out


def cpu_model():
    """The host CPU's model name (lscpu, then /proc/cpuinfo), else its
    architecture."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


ONE_THREAD_ENV = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def _oracle_child(code, timeout=600):
    """Run `code` in a child process whose BLAS and OpenMP pools have one
    thread (set before numpy loads); returns the float it prints last."""
    env = dict(os.environ, **ONE_THREAD_ENV)
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                           timeout=timeout)
        return float(r.stdout.strip().splitlines()[-1]) if r.returncode == 0 else None
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        return None


def oracle_one_core(workload, n_iters=1):
    """Oracle iterations/s of `workload` on one thread."""
    code = ("import sys, time; sys.path.insert(0, %r); "
            "from paper_2402_18311_gb300 import synth; from oracle import placer as opl; "
            "d = getattr(synth, %r)(0); o = opl.Placer(d, opl.Params(tau_stop=-1.0, max_iters=1 << 30)); "
            "t = time.perf_counter(); o.run(%d); print(%d / (time.perf_counter() - t))"
            % (ROOT, workload, n_iters, n_iters))
    return _oracle_child(code)


def oracle_config1_seconds():
    """Seconds the oracle takes, on one thread, for the 1k-cell configuration:
    300 iterations, one Shuffle (all) round, 300 more (Algorithm 1)."""
    code = ("import sys, time; sys.path.insert(0, %r); "
            "from paper_2402_18311_gb300 import synth; from oracle import placer as opl, hybro; "
            "d = synth.tiny_1k(0); t = time.perf_counter(); "
            "hybro.run(d, opl.Params(tau_stop=-1.0, max_iters=300), n_rounds=1, "
            "op=hybro.SHUFFLE_ALL, p=0.5, seed=0, tau_target=0.1); "
            "print(time.perf_counter() - t)" % (ROOT,))
    return _oracle_child(code)


def cpu_baseline(d, args, n_iters=1):
    """The FP64 oracle as it stands, on the same workload: n_iters full
    iterations after its set-up, on one thread (``value``, ``cores`` = 1), and
    in this process (``value_all_cores``: numpy's elementwise work stays on
    one thread there too; only its BLAS matrix products use the other cores).
    Also the oracle's time for the 1k-cell configuration on one thread."""
    from oracle import placer as opl
    t0 = time.perf_counter()
    o = opl.Placer(d, opl.Params(tau_stop=-1.0, max_iters=1 << 30))
    setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    o.run(n_iters)
    el = time.perf_counter() - t0
    v1 = oracle_one_core(args.workload, n_iters)
    c1 = oracle_config1_seconds()
    return {"value": v1, "unit": "iters/s", "cores": 1, "kind": "oracle",
            "cpu_model": cpu_model(),
            "value_all_cores": n_iters / el, "cores_all": os.cpu_count(),
            "config_tiny_1k_seconds_1_core": c1,
            "sample": f"{n_iters} full iteration(s) of the {args.workload} workload after "
                      f"{setup:.1f} s of oracle set-up; numpy float64 on one thread (BLAS and "
                      f"OpenMP pools set to 1); value_all_cores: the same in-process, where only "
                      f"BLAS matrix products use more than one core"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    maker, desc = WORKLOADS[args.workload]
    d = maker(0)
    from oracle import placer as opl
    o = opl.Placer(d, opl.Params(tau_stop=-1.0, max_iters=1 << 30))
    o.run(args.warmup)
    t0 = time.perf_counter()
    o.run(args.steps)
    el = time.perf_counter() - t0
    v = args.steps / el
    out = {"metric": METRIC, "value": v, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference",
           "config": {"workload": args.workload, "desc": desc, "parallelism": "cpu"},
           "cpu_baseline": {"value": v, "unit": "iters/s", "cores": 1,
                            "kind": "oracle",
                            "sample": f"{args.steps} timed oracle iterations after {args.warmup} "
                                      f"warm-up iterations of the {args.workload} workload, "
                                      f"numpy float64 on one thread"},
           "e2e": {"value": v, "unit": "iters/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large_2m", choices=sorted(WORKLOADS))
    ap.add_argument("--dct", type=int, default=1, choices=[0, 1],
                    help="spectral solve: 1 = BF16x3 on tcgen05 tensor cores, 0 = FP32 CUDA cores")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-restarts", action="store_true",
                    help="skip the batched-vs-serial restarts measurement")
    ap.add_argument("--serving-jobs", type=int, default=200,
                    help="jobs in the serving trace (0: skip)")
    ap.add_argument("--serving-max-cells", type=int, default=1_000_000,
                    help="largest design of the serving trace")
    ap.add_argument("--no-full-run", action="store_true",
                    help="skip the whole placement of the headline workload")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the 1k-cell and 210k-cell configuration runs")
    ap.add_argument("--autotune", type=int, default=1, choices=[0, 1],
                    help="1: tile shapes and kernel variants timed at create; 0: fixed rules")
    ap.add_argument("--advance", type=int, default=0,
                    help="untimed iterations before the warm-up (to time or profile a later "
                         "phase of the placement)"),
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        # the oracle runs on one thread: re-run this process with the BLAS and
        # OpenMP pools set to one thread before numpy loads
        if any(os.environ.get(k) != v for k, v in ONE_THREAD_ENV.items()):
            os.environ.update(ONE_THREAD_ENV)
            os.execv(sys.executable, [sys.executable] + sys.argv)
        # bounded sample: one oracle iteration takes about three seconds at 2M
        # cells, so at most 3 warm-up and 3 timed iterations are run
        args.steps = min(args.steps, 3)
        args.warmup = min(args.warmup, 3)
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
