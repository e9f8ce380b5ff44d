"""ctypes binding of the C ABI in ``include/hybro_place.h``.

Argument marshalling only: every computation runs in ``libhybro_place.so``.
Functions keep the C names.  Array arguments accept numpy arrays (host
memory) or torch tensors (host or CUDA); results are written into the
caller's buffers, as in C.  The library must have been built
(``paper_2402_18311_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhybro_place.so")
# the same library built with index checks in its kernels (-DPLACE_DEBUG_BOUNDS);
# loaded instead of LIB_PATH when HYBRO_PLACE_BOUNDS=1 is set before the first call
BOUNDS_LIB_PATH = os.path.join(HERE, "libhybro_place_bounds.so")

PLACE_OK = 0
PLACE_EINVAL = -1
PLACE_ENOMEM = -2
PLACE_ECUDA = -3
PLACE_ERANGE = -4
PLACE_ETIMEOUT = -5
PLACE_EINTERNAL = -6
PLACE_SHUFFLE_MACRO = 0
PLACE_SHUFFLE_ALL = 1
PLACE_WIREMASK = 2
PLACE_DCT_AUTO = -1
PLACE_DCT_FP32 = 0
PLACE_DCT_BF16X3 = 1
PLACE_STAGES = ("density", "spectral", "wirelength", "cellgrad", "update")


class PlaceError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"place error {code}: {msg}")
        self.code = code


class place_netlist(ct.Structure):
    _fields_ = [("n_cells", ct.c_int32), ("n_movable", ct.c_int32), ("n_nets", ct.c_int32),
                ("n_pins", ct.c_int32),
                ("w", ct.c_void_p), ("h", ct.c_void_p), ("x0", ct.c_void_p), ("y0", ct.c_void_p),
                ("net_ptr", ct.c_void_p), ("pin_cell", ct.c_void_p),
                ("pin_dx", ct.c_void_p), ("pin_dy", ct.c_void_p),
                ("net_w", ct.c_void_p), ("is_macro", ct.c_void_p)]


class place_die(ct.Structure):
    _fields_ = [("xl", ct.c_double), ("yl", ct.c_double), ("xh", ct.c_double), ("yh", ct.c_double)]


class place_bins(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("ny", ct.c_int32), ("target_density", ct.c_float)]


class place_params(ct.Structure):
    _fields_ = [("n_copies", ct.c_int32), ("gamma_base", ct.c_float), ("lambda_eta", ct.c_float),
                ("alpha0", ct.c_float), ("hpwl_ref", ct.c_float), ("mu_base", ct.c_float),
                ("mu_lo", ct.c_float), ("mu_hi", ct.c_float), ("tau_stop", ct.c_float),
                ("max_iters", ct.c_int32), ("constant_gamma", ct.c_float), ("dct_mode", ct.c_int32),
                ("max_backtracks", ct.c_int32), ("stretch", ct.c_int32),
                ("autotune", ct.c_int32), ("scatter_mode", ct.c_int32), ("gemm_bn", ct.c_int32),
                ("wa_big_cap", ct.c_int32), ("gemm_split", ct.c_int32), ("fillers", ct.c_int32),
                ("macro_precond", ct.c_float), ("wa_streams", ct.c_int32),
                ("dct_fold", ct.c_int32)]


class place_info(ct.Structure):
    _fields_ = [("n_cells", ct.c_int32), ("n_movable", ct.c_int32), ("n_nets", ct.c_int32),
                ("n_pins", ct.c_int32), ("nx", ct.c_int32), ("ny", ct.c_int32),
                ("n_copies", ct.c_int32), ("frac_bits", ct.c_int32),
                ("bin_w_q", ct.c_int64), ("bin_h_q", ct.c_int64),
                ("bin_w", ct.c_double), ("bin_h", ct.c_double), ("device_bytes", ct.c_int64),
                ("kernels_per_iter", ct.c_int32), ("dct_mode", ct.c_int32),
                ("n_fillers", ct.c_int32), ("bounds_checked", ct.c_int32),
                ("gemm_bn", ct.c_int32 * 4), ("gemm_split", ct.c_int32 * 4),
                ("wa_big_cap", ct.c_int32), ("autotuned", ct.c_int32),
                ("scatter_t1", ct.c_double), ("scatter_t2", ct.c_double),
                ("autotune_ms", ct.c_double), ("wa_streams", ct.c_int32), ("dct_fold", ct.c_int32)]


class place_state(ct.Structure):
    _fields_ = [("iter", ct.c_int32), ("converged", ct.c_int32), ("stopped", ct.c_int32),
                ("backtracks", ct.c_int32), ("lambda_", ct.c_double), ("gamma", ct.c_double),
                ("alpha", ct.c_double), ("a", ct.c_double), ("overflow", ct.c_double),
                ("hpwl_wa", ct.c_double), ("bins_effective", ct.c_double)]


class place_iter_record(ct.Structure):
    _fields_ = [("iter", ct.c_int32), ("backtracks", ct.c_int32), ("hpwl_wa", ct.c_double),
                ("overflow", ct.c_double), ("lambda_", ct.c_double), ("gamma", ct.c_double),
                ("alpha", ct.c_double)]


PLACE_HISTORY_CAP = 4096


class place_job(ct.Structure):
    _fields_ = [("kind", ct.c_int32), ("op", ct.c_int32), ("p", ct.c_float), ("pad", ct.c_int32),
                ("seed", ct.c_uint64), ("parent", ct.c_int64), ("arrival_s", ct.c_double),
                ("max_seconds", ct.c_double)]


class place_job_result(ct.Structure):
    _fields_ = [("id", ct.c_int64), ("kind", ct.c_int32), ("iterations", ct.c_int32),
                ("converged", ct.c_int32), ("status", ct.c_int32), ("arrival_s", ct.c_double),
                ("admit_s", ct.c_double), ("done_s", ct.c_double), ("hpwl", ct.c_double),
                ("overflow", ct.c_double), ("device_bytes", ct.c_int64),
                ("position_hash", ct.c_uint64)]


PLACE_JOB_PLACE = 0
PLACE_JOB_RESTART = 1
PLACE_JOB_FINISHED = 0
PLACE_JOB_CANCELLED = 1
PLACE_JOB_EXPIRED = 2

_VP = ct.c_void_p
_SIGS = {
    "place_default_params": (None, [ct.POINTER(place_params)]),
    "place_create": (ct.c_int, [ct.POINTER(place_netlist), ct.POINTER(place_die),
                                ct.POINTER(place_bins), ct.POINTER(place_params), _VP,
                                ct.POINTER(_VP)]),
    "place_destroy": (ct.c_int, [_VP]),
    "place_get_info": (ct.c_int, [_VP, ct.POINTER(place_info)]),
    "place_step": (ct.c_int, [_VP, ct.c_int32, _VP]),
    "place_perturb": (ct.c_int, [_VP, ct.c_int32, ct.c_float, ct.c_uint64, ct.c_int32]),
    "place_eval_hpwl_overflow": (ct.c_int, [_VP, _VP, _VP]),
    "place_get_positions": (ct.c_int, [_VP, ct.c_int32, _VP, _VP]),
    "place_set_positions": (ct.c_int, [_VP, ct.c_int32, _VP, _VP]),
    "place_get_state": (ct.c_int, [_VP, ct.c_int32, ct.POINTER(place_state)]),
    "place_step_multi": (ct.c_int, [ct.POINTER(_VP), ct.c_int32, ct.c_int32, _VP]),
    "place_device_views": (ct.c_int, [_VP, ct.c_int32, ct.POINTER(_VP), ct.POINTER(_VP)]),
    "place_eval_wirelength": (ct.c_int, [_VP, ct.c_int32, ct.c_float, _VP, _VP, _VP]),
    "place_eval_density": (ct.c_int, [_VP, ct.c_int32, _VP, _VP]),
    "place_get_fixed_map": (ct.c_int, [_VP, _VP]),
    "place_get_stretched_map": (ct.c_int, [_VP, ct.c_int32, _VP]),
    "place_eval_field": (ct.c_int, [_VP, ct.c_int32, _VP, _VP, _VP]),
    "place_eval_density_grad": (ct.c_int, [_VP, ct.c_int32, _VP, _VP]),
    "place_hybro": (ct.c_int, [_VP, ct.c_int32, ct.c_int32, ct.c_float, ct.c_uint64, ct.c_float,
                               _VP, _VP, _VP]),
    "place_get_best_positions": (ct.c_int, [_VP, ct.c_int32, _VP, _VP]),
    "place_step_timed": (ct.c_int, [_VP, ct.c_int32, _VP]),
    "place_measure_wa_floor": (ct.c_int, [_VP, ct.c_int32, ct.POINTER(ct.c_float)]),
    "place_test_wait_timeout": (ct.c_int, [_VP]),
    "place_test_bounds_check": (ct.c_int, [_VP]),
    "place_measure_scatter_floor": (ct.c_int, [_VP, ct.c_int32, ct.POINTER(ct.c_float),
                                               ct.POINTER(ct.c_float)]),
    "place_get_hybro_rounds": (ct.c_int, [_VP, ct.c_int32, _VP, _VP, ct.c_int32,
                                          ct.POINTER(ct.c_int32)]),
    "place_overflow_noalloc": (ct.c_int, [_VP, _VP, _VP, _VP, ct.c_int32,
                                          ct.POINTER(place_die), ct.POINTER(place_bins),
                                          ct.c_int32, _VP, _VP, _VP, _VP]),
    "place_estimate_device_bytes": (ct.c_int, [ct.POINTER(place_netlist), ct.POINTER(place_die),
                                                ct.POINTER(place_bins), ct.POINTER(place_params),
                                                ct.POINTER(ct.c_int64)]),
    "place_get_fillers": (ct.c_int, [_VP, ct.c_int32, _VP, _VP, ct.c_int32, ct.POINTER(ct.c_int32)]),
    "place_get_history": (ct.c_int, [_VP, ct.c_int32, _VP, ct.c_int32, ct.POINTER(ct.c_int32)]),
    "place_set_fillers": (ct.c_int, [_VP, ct.c_int32, _VP, _VP]),
    "place_checkpoint_bytes": (ct.c_int, [_VP, ct.POINTER(ct.c_int64)]),
    "place_checkpoint_save": (ct.c_int, [_VP, ct.c_int32, _VP, ct.c_int64]),
    "place_checkpoint_load": (ct.c_int, [_VP, ct.c_int32, _VP, ct.c_int64]),
    "place_server_create": (ct.c_int, [ct.c_int64, ct.c_int32, ct.c_int32, ct.POINTER(_VP)]),
    "place_server_submit": (ct.c_int, [_VP, ct.POINTER(place_netlist), ct.POINTER(place_die),
                                       ct.POINTER(place_bins), ct.POINTER(place_params),
                                       ct.POINTER(place_job), ct.POINTER(ct.c_int64)]),
    "place_server_run": (ct.c_int, [_VP, ct.c_double, ct.POINTER(ct.c_double)]),
    "place_server_cancel": (ct.c_int, [_VP, ct.c_int64]),
    "place_server_results": (ct.c_int, [_VP, _VP, ct.c_int32, ct.POINTER(ct.c_int32)]),
    "place_server_stats": (ct.c_int, [_VP, ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int32)]),
    "place_server_destroy": (ct.c_int, [_VP]),
    "place_last_error": (ct.c_char_p, []),
}

_lib = None


def lib_path():
    """The library this process loads: the bounds-checking build when the
    environment variable HYBRO_PLACE_BOUNDS is 1, else the normal one."""
    return BOUNDS_LIB_PATH if os.environ.get("HYBRO_PLACE_BOUNDS") == "1" else LIB_PATH


def lib():
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "paper_2402_18311_gb300.build.build()")
        L = ct.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(rc):
    if rc != PLACE_OK:
        raise PlaceError(rc, lib().place_last_error().decode(errors="replace"))
    return rc


def _ptr(a):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


# ---- C entry points with their C names ------------------------------------

def place_default_params(**overrides):
    p = place_params()
    lib().place_default_params(ct.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _netlist(design):
    """place_netlist of a ``synth.Design`` plus the arrays it points into
    (which must stay alive while the netlist is in use)."""
    keep = dict(w=np.ascontiguousarray(design.w, np.float32),
                h=np.ascontiguousarray(design.h, np.float32),
                x0=np.ascontiguousarray(design.x, np.float32),
                y0=np.ascontiguousarray(design.y, np.float32),
                net_ptr=np.ascontiguousarray(design.net_ptr, np.int32),
                pin_cell=np.ascontiguousarray(design.pin_cell, np.int32),
                pin_dx=np.ascontiguousarray(design.pin_dx, np.float32),
                pin_dy=np.ascontiguousarray(design.pin_dy, np.float32))
    net_w = getattr(design, "net_w", None)
    if net_w is not None:
        keep["net_w"] = np.ascontiguousarray(net_w, np.float32)
    if design.is_macro is not None:
        keep["is_macro"] = np.ascontiguousarray(design.is_macro, np.uint8)
    nl = place_netlist(design.n_cells, design.n_movable, design.n_nets, design.n_pins,
                       *(_ptr(keep[k]) for k in ("w", "h", "x0", "y0", "net_ptr", "pin_cell",
                                                 "pin_dx", "pin_dy")),
                       _ptr(keep.get("net_w")), _ptr(keep.get("is_macro")))
    return nl, keep


def place_create(design, params=None, stream=None):
    """Create a handle for a ``synth.Design`` (host arrays are copied)."""
    nl, keep = _netlist(design)
    die = place_die(*design.die)
    bins = place_bins(design.nx, design.ny, design.target_density)
    prm = params if params is not None else place_default_params()
    h = _VP()
    _check(lib().place_create(ct.byref(nl), ct.byref(die), ct.byref(bins), ct.byref(prm),
                              _VP(stream or 0), ct.byref(h)))
    return h


def place_destroy(h):
    return _check(lib().place_destroy(h))


def place_get_info(h):
    o = place_info()
    _check(lib().place_get_info(h, ct.byref(o)))
    return o


def place_step(h, n_iters, converged=None):
    return _check(lib().place_step(h, int(n_iters), _ptr(converged)))


def place_perturb(h, op, p, seed, copy=-1):
    return _check(lib().place_perturb(h, int(op), float(p), int(seed), int(copy)))


def place_eval_hpwl_overflow(h, hpwl=None, overflow=None):
    return _check(lib().place_eval_hpwl_overflow(h, _ptr(hpwl), _ptr(overflow)))


def place_get_positions(h, copy, x, y):
    return _check(lib().place_get_positions(h, int(copy), _ptr(x), _ptr(y)))


def place_step_multi(handles, n_iters, converged=None):
    """Step several handles together; ``converged`` (optional int32 array of
    the handles' total copy count) receives the stopped flags."""
    arr = (_VP * len(handles))(*[hh.value if isinstance(hh, _VP) else hh for hh in handles])
    return _check(lib().place_step_multi(arr, len(handles), int(n_iters), _ptr(converged)))


def place_device_views(h, copy):
    """(x, y) borrowed device addresses of copy ``copy``'s interleaved
    positions: cell i is at element 2 i of each."""
    x, y = _VP(), _VP()
    _check(lib().place_device_views(h, int(copy), ct.byref(x), ct.byref(y)))
    return x.value, y.value


def place_set_positions(h, copy, x, y):
    return _check(lib().place_set_positions(h, int(copy), _ptr(x), _ptr(y)))


def place_get_state(h, copy):
    o = place_state()
    _check(lib().place_get_state(h, int(copy), ct.byref(o)))
    return o


def place_eval_wirelength(h, copy, gamma, grad_x=None, grad_y=None):
    wl = ct.c_double()
    _check(lib().place_eval_wirelength(h, int(copy), float(gamma), ct.byref(wl),
                                       _ptr(grad_x), _ptr(grad_y)))
    return wl.value


def place_eval_density(h, copy, out_map=None):
    tau = ct.c_double()
    _check(lib().place_eval_density(h, int(copy), _ptr(out_map), ct.byref(tau)))
    return tau.value


def place_get_fixed_map(h, out_map):
    return _check(lib().place_get_fixed_map(h, _ptr(out_map)))


def place_get_stretched_map(h, copy, out_map):
    return _check(lib().place_get_stretched_map(h, int(copy), _ptr(out_map)))


def place_eval_field(h, copy, psi=None, ex=None, ey=None):
    return _check(lib().place_eval_field(h, int(copy), _ptr(psi), _ptr(ex), _ptr(ey)))


def place_eval_density_grad(h, copy, grad_x=None, grad_y=None):
    return _check(lib().place_eval_density_grad(h, int(copy), _ptr(grad_x), _ptr(grad_y)))


def place_hybro(h, n_rounds, op, p, seed, tau_target, best_hpwl=None, best_overflow=None,
                best_round=None):
    return _check(lib().place_hybro(h, int(n_rounds), int(op), float(p), int(seed),
                                    float(tau_target), _ptr(best_hpwl), _ptr(best_overflow),
                                    _ptr(best_round)))


def place_get_best_positions(h, copy, x, y):
    return _check(lib().place_get_best_positions(h, int(copy), _ptr(x), _ptr(y)))


def place_measure_wa_floor(h, reps=10):
    """Mean milliseconds of one gather-and-reduce floor pass (see the header)."""
    ms = ct.c_float()
    _check(lib().place_measure_wa_floor(h, int(reps), ct.byref(ms)))
    return ms.value


def place_measure_scatter_floor(h, reps=10):
    """(scatter ms, floor ms) at the current positions (see the header)."""
    a, b = ct.c_float(), ct.c_float()
    _check(lib().place_measure_scatter_floor(h, int(reps), ct.byref(a), ct.byref(b)))
    return a.value, b.value


def place_get_hybro_rounds(h, copy):
    """(hpwl, overflow) float64 arrays, one entry per round of the last
    place_hybro call, for copy ``copy``."""
    n = ct.c_int32()
    _check(lib().place_get_hybro_rounds(h, int(copy), None, None, 0, ct.byref(n)))
    hp = np.empty(n.value, np.float64)
    tv = np.empty(n.value, np.float64)
    _check(lib().place_get_hybro_rounds(h, int(copy), _ptr(hp), _ptr(tv), n.value, ct.byref(n)))
    return hp, tv


def place_step_timed(h, n_iters, stage_ms):
    """stage_ms: float32 numpy array [5]; per-stage milliseconds are added."""
    return _check(lib().place_step_timed(h, int(n_iters), _ptr(stage_ms)))


def place_overflow_noalloc(x, y, w, h, n_movable, die, bins, frac_bits, fixed_map,
                           overflow, map_out=None, stream=None):
    """Overflow (and optionally the density map) into caller-owned device
    buffers, using only the library's static scratch (no allocation).
    ``die``: (xl, yl, xh, yh); ``bins``: (nx, ny, target_density)."""
    d = place_die(*die)
    b = place_bins(*bins)
    return _check(lib().place_overflow_noalloc(_ptr(x), _ptr(y), _ptr(w), _ptr(h),
                                               int(n_movable), ct.byref(d),
                                               ct.byref(b), int(frac_bits), _ptr(fixed_map),
                                               _ptr(overflow), _ptr(map_out), _VP(stream or 0)))


def place_estimate_device_bytes(design, params=None):
    nl, keep = _netlist(design)
    b = ct.c_int64()
    die = place_die(*design.die)
    bins = place_bins(design.nx, design.ny, design.target_density)
    prm = params if params is not None else place_default_params()
    _check(lib().place_estimate_device_bytes(ct.byref(nl), ct.byref(die), ct.byref(bins),
                                             ct.byref(prm), ct.byref(b)))
    return b.value


def place_test_bounds_check(h):
    """The C return code (PLACE_EINTERNAL expected in the bounds-checking
    build, PLACE_EINVAL in the normal one); does not raise."""
    return lib().place_test_bounds_check(h)


def place_test_wait_timeout(h):
    """The C return code (PLACE_ETIMEOUT expected); does not raise."""
    return lib().place_test_wait_timeout(h)


def place_get_history(h, copy, cap=PLACE_HISTORY_CAP):
    """Per-iteration records (place_iter_record list) of copy ``copy``."""
    n = ct.c_int32()
    arr = (place_iter_record * max(int(cap), 1))()
    _check(lib().place_get_history(h, int(copy), ct.cast(arr, _VP), int(cap), ct.byref(n)))
    return [arr[i] for i in range(min(n.value, int(cap)))]


def place_set_fillers(h, copy, x, y):
    return _check(lib().place_set_fillers(h, int(copy), _ptr(x), _ptr(y)))


def place_checkpoint_bytes(h):
    n = ct.c_int64()
    _check(lib().place_checkpoint_bytes(h, ct.byref(n)))
    return n.value


def place_checkpoint_save(h, copy):
    """Copy ``copy``'s optimiser state as a uint8 numpy array."""
    buf = np.empty(place_checkpoint_bytes(h), np.uint8)
    _check(lib().place_checkpoint_save(h, int(copy), _ptr(buf), buf.size))
    return buf


def place_checkpoint_load(h, copy, buf):
    buf = np.ascontiguousarray(buf, np.uint8)
    return _check(lib().place_checkpoint_load(h, int(copy), _ptr(buf), buf.size))


def place_get_fillers(h, copy):
    """(x, y) float32 arrays of copy ``copy``'s filler corners."""
    n = ct.c_int32()
    _check(lib().place_get_fillers(h, int(copy), None, None, 0, ct.byref(n)))
    x = np.empty(n.value, np.float32)
    y = np.empty(n.value, np.float32)
    _check(lib().place_get_fillers(h, int(copy), _ptr(x), _ptr(y), n.value, ct.byref(n)))
    return x, y


class Server:
    """Job server (continuous batching).  Keeps every submitted design's host
    arrays alive until the server is destroyed, as the C ABI requires."""

    def __init__(self, hbm_budget, max_active, iters_per_tick=32):
        self.h = _VP()
        _check(lib().place_server_create(int(hbm_budget), int(max_active), int(iters_per_tick),
                                         ct.byref(self.h)))
        self._keep = []

    def submit(self, design, params=None, kind=PLACE_JOB_PLACE, arrival_s=0.0, parent=-1,
               op=PLACE_SHUFFLE_ALL, p=0.5, seed=0, max_seconds=0.0):
        nl, keep = _netlist(design)
        die = place_die(*design.die)
        bins = place_bins(design.nx, design.ny, design.target_density)
        prm = params if params is not None else place_default_params()
        job = place_job(kind, op, p, 0, seed, parent, arrival_s, max_seconds)
        jid = ct.c_int64()
        _check(lib().place_server_submit(self.h, ct.byref(nl), ct.byref(die), ct.byref(bins),
                                         ct.byref(prm), ct.byref(job), ct.byref(jid)))
        self._keep.append((nl, keep, die, bins, prm))
        return jid.value

    def run(self, timeout_s=0.0):
        m = ct.c_double()
        _check(lib().place_server_run(self.h, float(timeout_s), ct.byref(m)))
        return m.value

    def cancel(self, job_id):
        return _check(lib().place_server_cancel(self.h, int(job_id)))

    def results(self):
        n = ct.c_int32()
        _check(lib().place_server_results(self.h, None, 0, ct.byref(n)))
        arr = (place_job_result * max(n.value, 1))()
        _check(lib().place_server_results(self.h, ct.cast(arr, _VP), n.value, ct.byref(n)))
        return [arr[i] for i in range(n.value)]

    def stats(self):
        b = ct.c_int64(); a = ct.c_int32()
        _check(lib().place_server_stats(self.h, ct.byref(b), ct.byref(a)))
        return b.value, a.value

    def close(self):
        if self.h:
            lib().place_server_destroy(self.h)
            self.h = None


def place_last_error():
    return lib().place_last_error().decode(errors="replace")
