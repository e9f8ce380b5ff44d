"""The C-ABI library loads, exports every entry point its header declares, and
rejects malformed input on the host before touching the GPU."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from oracle import placer as opl
from paper_2402_18311_gb300 import place, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hybro_place.h")


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(place.LIB_PATH):
        from paper_2402_18311_gb300 import build
        build.build()
    return place.lib()


def declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(place_[a-z_0-9]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert sorted(place.exported_symbols()) == names


def test_bounds_checked_build_exports_every_declared_symbol(L):
    # the -DPLACE_DEBUG_BOUNDS twin of the library (loaded by the binding when
    # HYBRO_PLACE_BOUNDS=1) exports the same entry points
    if not os.path.exists(place.BOUNDS_LIB_PATH):
        from paper_2402_18311_gb300 import build
        build.build(variant="bounds")
    Lb = ct.CDLL(place.BOUNDS_LIB_PATH)
    for n in declared():
        assert hasattr(Lb, n), n


def test_default_params_match_the_oracle_reading(L):
    p = place.place_default_params()
    o = opl.Params()
    assert p.n_copies == 1
    for f in ("gamma_base", "lambda_eta", "alpha0", "hpwl_ref", "mu_base", "mu_lo", "mu_hi",
              "tau_stop"):
        assert getattr(p, f) == pytest.approx(getattr(o, f), rel=1e-7), f
    assert p.max_iters == o.max_iters
    assert p.max_backtracks == o.max_backtracks == 0
    assert p.dct_mode == place.PLACE_DCT_AUTO and p.autotune == 1 and p.scatter_mode == -1
    assert p.gemm_bn == 0 and p.wa_big_cap == 0 and p.gemm_split == 0 and p.fillers == 0
    assert p.wa_streams == 0 and p.dct_fold == 1
    assert p.macro_precond == o.macro_precond == 1.0


def test_struct_sizes_match_header_layout():
    assert ct.sizeof(place.place_netlist) == 4 * 4 + 10 * 8
    assert ct.sizeof(place.place_params) == 23 * 4
    assert ct.sizeof(place.place_state) == 4 * 4 + 7 * 8
    assert ct.sizeof(place.place_info) == 8 * 4 + 2 * 8 + 2 * 8 + 8 + 4 * 4 + 10 * 4 + 3 * 8 + 2 * 4
    assert ct.sizeof(place.place_job) == 4 * 4 + 8 + 8 + 8 + 8
    assert ct.sizeof(place.place_job_result) == 8 + 4 * 4 + 5 * 8 + 8 + 8


def test_struct_layouts_match_the_compiled_header(tmp_path):
    # every ctypes struct of the binding against a C compile of the header:
    # same field names, offsets and total size
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [getattr(place, n) for n in dir(place)
               if n.startswith("place_") and isinstance(getattr(place, n), type)
               and issubclass(getattr(place, n), ct.Structure)]
    assert len(structs) >= 8
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hybro_place.h"',
             "int main(void) {"]
    expect = []
    for S in structs:
        t = S.__name__
        lines.append(f'  printf("%zu\\n", sizeof({t}));')
        expect.append(ct.sizeof(S))
        for f, _ in S._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({t}, {f.rstrip("_")}));')
            expect.append(getattr(S, f).offset)
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert got == expect


def _design():
    return synth.make_design(n_movable=20, die=(0, 0, 64, 64), nx=16, ny=16, n_nets=15,
                             n_pads=4, seed=3)


@pytest.mark.parametrize("mut,msg", [
    (lambda d: setattr(d, "nx", 12), "multiples of 16"),
    (lambda d: d.pin_cell.__setitem__(0, 10 ** 6), "out of range"),
    (lambda d: d.w.__setitem__(3, 0.0), "non-positive size"),
    (lambda d: d.net_ptr.__setitem__(1, d.net_ptr[2] + 1), "monotone"),
    (lambda d: setattr(d, "die", (0.1, 0, 64, 64)), "multiples of 2^-"),
])
def test_create_rejects_malformed_input_on_host(L, mut, msg):
    d = _design()
    mut(d)
    with pytest.raises(place.PlaceError) as ei:
        place.place_create(d)
    assert ei.value.code == place.PLACE_EINVAL
    assert msg in str(ei.value)


def test_create_rejects_a_cell_beyond_the_gradient_fixed_point(L):
    # one net weighted so heavily that its pins' wirelength-gradient bound
    # leaves fewer than 10 fraction bits in the 32-bit per-cell sums
    d = _design()
    d.net_w = np.ones(d.n_nets, np.float32)
    d.net_w[d.n_nets // 2] = 1e7
    with pytest.raises(place.PlaceError) as ei:
        place.place_create(d)
    assert ei.value.code == place.PLACE_ERANGE
    assert "too many pins" in str(ei.value)


def test_create_rejects_bad_params(L):
    d = _design()
    with pytest.raises(place.PlaceError) as ei:
        place.place_create(d, place.place_default_params(n_copies=0))
    assert ei.value.code == place.PLACE_EINVAL
    with pytest.raises(place.PlaceError):
        place.place_create(d, place.place_default_params(dct_mode=7))
    with pytest.raises(place.PlaceError) as ei:
        place.place_create(d, place.place_default_params(stretch=2))
    assert ei.value.code == place.PLACE_EINVAL and "stretch" in str(ei.value)
    for field, bad in (("autotune", 2), ("scatter_mode", 3), ("gemm_bn", 96), ("wa_big_cap", 16),
                       ("gemm_split", 3), ("fillers", 2), ("macro_precond", 0.0),
                       ("wa_streams", 4), ("dct_fold", 2)):
        with pytest.raises(place.PlaceError) as ei:
            place.place_create(d, place.place_default_params(**{field: bad}))
        assert ei.value.code == place.PLACE_EINVAL and field in str(ei.value)
    for mb in (-1, 65):
        with pytest.raises(place.PlaceError) as ei:
            place.place_create(d, place.place_default_params(max_backtracks=mb))
        assert ei.value.code == place.PLACE_EINVAL and "max_backtracks" in str(ei.value)


def test_null_handle_calls_fail_cleanly(L):
    assert L.place_step(None, 1, None) == place.PLACE_EINVAL
    assert L.place_step_multi(None, 0, 1, None) == place.PLACE_EINVAL
    arr = (ct.c_void_p * 2)(None, None)
    assert L.place_step_multi(arr, 2, 1, None) == place.PLACE_EINVAL
    x, y = ct.c_void_p(), ct.c_void_p()
    assert L.place_device_views(None, 0, ct.byref(x), ct.byref(y)) == place.PLACE_EINVAL
    n = ct.c_int64()
    assert L.place_checkpoint_bytes(None, ct.byref(n)) == place.PLACE_EINVAL
    buf = (ct.c_uint8 * 64)()
    assert L.place_checkpoint_save(None, 0, buf, 64) == place.PLACE_EINVAL
    assert L.place_checkpoint_load(None, 0, buf, 64) == place.PLACE_EINVAL
    assert L.place_destroy(None) == place.PLACE_OK
    assert b"null" in L.place_last_error()


def test_server_rejects_bad_arguments_on_host(L):
    with pytest.raises(place.PlaceError):
        place.Server(0, 1)
    s = place.Server(1 << 30, 2)
    try:
        d = _design()
        with pytest.raises(place.PlaceError) as ei:
            s.submit(d, kind=place.PLACE_JOB_RESTART, parent=5)
        assert ei.value.code == place.PLACE_EINVAL
    finally:
        s.close()


def test_server_cancels_queued_jobs_and_their_restarts_on_host(L):
    # failure handling on the host, no GPU: a job cancelled before it runs is
    # never admitted, nor are its restarts; a negative budget is rejected
    s = place.Server(1 << 30, 2)
    try:
        d = _design()
        with pytest.raises(place.PlaceError):
            s.submit(d, max_seconds=-1.0)
        a = s.submit(d)
        r1 = s.submit(d, kind=place.PLACE_JOB_RESTART, parent=a, seed=1)
        r2 = s.submit(d, kind=place.PLACE_JOB_RESTART, parent=a, seed=2)
        s.cancel(a)
        with pytest.raises(place.PlaceError):
            s.cancel(99)
        s.run()
        res = s.results()
        assert [r.id for r in res] == [a, r1, r2]
        for r in res:
            assert r.status == place.PLACE_JOB_CANCELLED
            assert r.iterations == 0 and r.position_hash == 0 and np.isnan(r.hpwl)
    finally:
        s.close()


def test_footprint_estimate_grows_with_the_design(L):
    small = synth.scaled(2000, 128, seed=1)
    big = synth.scaled(20000, 256, seed=1)
    a = place.place_estimate_device_bytes(small)
    b = place.place_estimate_device_bytes(big)
    assert 0 < a < b
    b4 = place.place_estimate_device_bytes(big, place.place_default_params(n_copies=4))
    assert b < b4 < 4 * b  # the netlist and transform tables are shared by the copies
    # backtracking keeps u_k and v_k (the redone step starts there): 16 bytes
    # per movable cell and copy (plus alignment)
    bb = place.place_estimate_device_bytes(big, place.place_default_params(max_backtracks=3))
    assert 16 * big.n_movable <= bb - b <= 16 * big.n_movable + 512
    # stretching: a second map (8 bytes per bin) and 20 bytes per movable cell
    bs = place.place_estimate_device_bytes(big, place.place_default_params(stretch=1))
    extra = 8 * big.nx * big.ny + 20 * big.n_movable
    assert extra <= bs - b <= extra + 768
    # fillers: the oracle's count of cells more, and a second map per copy
    from oracle import placer as opl
    nf = opl.Placer(big, opl.Params(fillers=True)).nf
    assert nf > 0
    bf = place.place_estimate_device_bytes(big, place.place_default_params(fillers=1))
    assert 8 * big.nx * big.ny + 100 * nf <= bf - b <= 8 * big.nx * big.ny + 200 * nf + 8192
