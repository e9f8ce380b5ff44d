"""The bounds-checking build (``-DPLACE_DEBUG_BOUNDS``, in its place for
compute-sanitizer): every index check in the kernels passes on the library's
workloads, and the results are bit-identical to those of the normal build
(the kernels write their floating-point arithmetic with explicit rounding
where a multiply-add could be contracted either way, so both builds compute
the same bits).

Each build runs in a child process (the binding loads one library per
process), through the same script; the script raises on any non-zero return
code, so a failed index check (PLACE_EINTERNAL) fails the test."""
import json
import os
import subprocess
import sys

import pytest

from paper_2402_18311_gb300 import place

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import hashlib, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2402_18311_gb300 import place, synth

out = {}
def hsh(*arrs):
    m = hashlib.sha1()
    for a in arrs:
        m.update(np.ascontiguousarray(a).tobytes())
    return m.hexdigest()

def positions(h, d, copy=0):
    x = np.empty(d.n_cells, np.float32); y = np.empty(d.n_cells, np.float32)
    place.place_get_positions(h, copy, x, y)
    return x, y

def evals(tag, h, d):
    hp = np.empty(place.place_get_info(h).n_copies); tv = np.empty_like(hp)
    place.place_eval_hpwl_overflow(h, hp, tv)
    G = d.nx * d.ny
    m = np.empty(G, np.int64)
    tau = place.place_eval_density(h, 0, m)
    gx = np.empty(d.n_movable, np.float32); gy = np.empty(d.n_movable, np.float32)
    wl = place.place_eval_wirelength(h, 0, 4.0, gx, gy)
    psi = np.empty(G, np.float32); ex = np.empty(G, np.float32); ey = np.empty(G, np.float32)
    place.place_eval_field(h, 0, psi, ex, ey)
    dx = np.empty(d.n_movable, np.float32); dy = np.empty(d.n_movable, np.float32)
    place.place_eval_density_grad(h, 0, dx, dy)
    out[tag] = {"pos": hsh(*positions(h, d)), "hpwl": hp.tolist(), "tau": tv.tolist(),
                "map": hsh(m), "tau0": tau, "wl": wl, "gw": hsh(gx, gy),
                "field": hsh(psi, ex, ey), "gd": hsh(dx, dy)}

checked = []
# FP32 spectral path, 64 x 64 bins, every scatter way forced in turn
d = synth.tiny_1k(0)
for mode in (-1, 0, 1, 2):
    h = place.place_create(d, place.place_default_params(tau_stop=-1.0, max_iters=10**6,
                                                         scatter_mode=mode))
    checked.append(place.place_get_info(h).bounds_checked)
    place.place_step(h, 120)
    evals(f"tiny_scatter{mode}", h, d)
    place.place_destroy(h)

# the failure path: a check that fails (no access is made with the index)
h = place.place_create(d, place.place_default_params(tau_stop=-1.0, max_iters=10**6))
rc = place.place_test_bounds_check(h)
msg = place.place_last_error()
place.place_step(h, 5)  # the handle stays usable; the flag was cleared
failpath = {"rc": rc, "msg": msg}
place.place_destroy(h)

# mixed-size: Shuffle (macros), WireMask, Hybro rounds, knobs
d = synth.mixed_size_1k(0)
h = place.place_create(d, place.place_default_params(tau_stop=0.1, max_iters=400, n_copies=2,
                                                     max_backtracks=2, stretch=1,
                                                     macro_precond=4.0))
place.place_step(h, 400)
place.place_perturb(h, place.PLACE_SHUFFLE_MACRO, 0.5, 7, -1)
place.place_perturb(h, place.PLACE_WIREMASK, 0.0, 0, -1)
evals("mixed_perturbed", h, d)
bh = np.empty(2); bt = np.empty(2); br = np.empty(2, np.int32)
place.place_hybro(h, 2, place.PLACE_SHUFFLE_ALL, 0.5, 11, 0.1, bh, bt, br)
out["mixed_hybro"] = {"bh": bh.tolist(), "bt": bt.tolist(), "br": br.tolist(),
                      "hist": [(r.iter, r.hpwl_wa, r.overflow) for r in place.place_get_history(h, 1, 64)]}
place.place_destroy(h)

# tensor-core path with big nets, fillers, the autotuner's every GEMM variant
d = synth.scaled(20000, 128, seed=2)
h = place.place_create(d, place.place_default_params(tau_stop=-1.0, max_iters=10**6, fillers=1,
                                                     autotune=1))
checked.append(place.place_get_info(h).bounds_checked)
place.place_step(h, 150)
evals("scaled20k_fill", h, d)
fx, fy = place.place_get_fillers(h, 0)
out["scaled20k_fillers"] = hsh(fx, fy)
place.place_destroy(h)
for bn, split in ((64, 1), (128, 2)):
    h = place.place_create(d, place.place_default_params(tau_stop=-1.0, max_iters=10**6,
                                                         autotune=0, gemm_bn=bn, gemm_split=split))
    place.place_step(h, 60)
    evals(f"scaled20k_bn{bn}_split{split}", h, d)
    place.place_destroy(h)

# the allocation-free overflow on device buffers
import torch
d = synth.tiny_1k(0)
n = d.n_movable
dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
x, y, w, hh = dev(d.x[:n]), dev(d.y[:n]), dev(d.w[:n]), dev(d.h[:n])
ov = torch.zeros(1, dtype=torch.float64, device="cuda")
mp = torch.zeros(d.nx * d.ny, dtype=torch.int64, device="cuda")
place.place_overflow_noalloc(x, y, w, hh, n, d.die, (d.nx, d.ny, d.target_density), 8, None, ov, mp)
torch.cuda.synchronize()
out["noalloc"] = {"tau": float(ov.item()), "map": hsh(mp.cpu().numpy())}
print(json.dumps({"checked": checked, "out": out, "failpath": failpath}))
"""


def _run(bounds):
    env = dict(os.environ, HYBRO_PLACE_BOUNDS="1" if bounds else "0")
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.mark.gpu
def test_bounds_checked_build_passes_and_matches_the_normal_build():
    if not os.path.exists(place.BOUNDS_LIB_PATH):
        from paper_2402_18311_gb300 import build
        build.build(variant="bounds")
    chk = _run(True)
    ref = _run(False)
    assert all(v == 1 for v in chk["checked"]), chk["checked"]
    assert all(v == 0 for v in ref["checked"]), ref["checked"]
    # a failing check is reported with its site and index, and only there
    assert chk["failpath"]["rc"] == place.PLACE_EINTERNAL, chk["failpath"]
    assert "WA: a pin's cell" in chk["failpath"]["msg"]
    assert ref["failpath"]["rc"] == place.PLACE_EINVAL
    for k, v in ref["out"].items():
        assert chk["out"][k] == v, k
