"""ctypes binding of the C ABI in ``include/sgmf.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does
nothing but convert arguments: all stages of the pipeline run in the CUDA
kernels of ``libsgmf.so``.  There is no CPU fallback; if the library is
missing or cannot be loaded, ``lib()`` raises.

``Context`` is a small convenience wrapper that passes torch tensors (device
memory, streams) to the same entry points.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, asdict, fields

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libsgmf.so")

SGMF_OK, SGMF_ERR_ARG, SGMF_ERR_PARAM, SGMF_ERR_SHAPE, SGMF_ERR_OOM, SGMF_ERR_CUDA, SGMF_ERR_TIMEOUT = range(7)
SGMF_CENSUS_CS9X7, SGMF_CENSUS_9X7 = 0, 1
SGMF_CHECK_STEREO_LIDAR, SGMF_CHECK_STEREO, SGMF_CHECK_LIDAR, SGMF_CHECK_NONE = 0, 1, 2, 3
SGMF_WAIT_CENSUS = 0
BAND_TILE = 8   # banded mode: pixels per side of a band tile (include/sgmf.h)
(SGMF_STAGE_DBAR, SGMF_STAGE_CENSUS_L, SGMF_STAGE_CENSUS_R, SGMF_STAGE_DHAT, SGMF_STAGE_COST,
 SGMF_STAGE_SUM, SGMF_STAGE_DSTAR, SGMF_STAGE_DPRIME, SGMF_STAGE_DSUB, SGMF_STAGE_BOX_S,
 SGMF_STAGE_BOX_C) = range(11)

# symbols declared in include/sgmf.h
EXPORTS = (
    "sgmf_default_params", "sgmf_create", "sgmf_create_batched", "sgmf_batch_capacity", "sgmf_set_params",
    "sgmf_get_params", "sgmf_set_stream", "sgmf_compute", "sgmf_compute_batch", "sgmf_compute_host",
    "sgmf_compute_host_batch", "sgmf_sync", "sgmf_destroy", "sgmf_last_error",
    "sgmf_status_string", "sgmf_set_debug", "sgmf_debug_stage", "sgmf_launches_per_compute",
    "sgmf_set_profiling", "sgmf_kernel_times", "sgmf_device_bytes", "sgmf_check_static",
    "sgmf_set_wait_limit", "sgmf_debug_fail_alloc", "sgmf_measure_rates",
    "sgmf_set_tuning", "sgmf_get_tuning", "sgmf_autotune",
    "sgmf_multi_create", "sgmf_multi_frame", "sgmf_multi_classes", "sgmf_multi_class_info",
    "sgmf_multi_autotune", "sgmf_multi_launch", "sgmf_multi_sync", "sgmf_multi_launches",
    "sgmf_multi_device_bytes", "sgmf_multi_destroy",
    "sgmf_server_create", "sgmf_server_add_camera", "sgmf_server_submit", "sgmf_server_poll",
    "sgmf_server_stats", "sgmf_server_destroy",
    "sgmf_create_banded", "sgmf_compute_banded", "sgmf_band_width", "sgmf_compute_host_batch_async",
    "sgmf_compute_front", "sgmf_prior_device", "sgmf_compute_banded_back",
    "sgmf_bn_pack", "sgmf_bn_conv", "sgmf_bn_wgrad", "sgmf_bn_input", "sgmf_bn_labels", "sgmf_bn_loss",
    "sgmf_bn_adam", "sgmf_bn_tiles", "sgmf_bn_gather", "sgmf_bn_to_bf16", "sgmf_bn_decide", "sgmf_set_gate",
)


class SgmfError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_status_name(status)}: {msg}")
        self.status = status


class sgmf_params(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in (
        "p1", "p2", "q1", "q2", "alpha_num", "alpha_den", "ts", "rs", "tc", "rc",
        "lr_max_diff", "census", "semidense", "consistency", "num_paths", "subpixel")]


class sgmf_rates(ctypes.Structure):
    _fields_ = [("sms", ctypes.c_int)] + [(k, ctypes.c_double) for k in (
        "min3_u16x2", "addmin_u16x2", "iadd", "popc", "prmt")]


class sgmf_tuning(ctypes.Structure):
    _fields_ = [("line_warps", ctypes.c_int32), ("cost_px", ctypes.c_int32), ("sweep", ctypes.c_int32),
                ("parts", ctypes.c_int32)]


class sgmf_server_counters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("batched_frames", ctypes.c_uint64), ("largest_batch", ctypes.c_int32),
                ("max_concurrent_batches", ctypes.c_int32), ("slots", ctypes.c_int32),
                ("device_bytes", ctypes.c_size_t), ("peak_device_bytes", ctypes.c_size_t),
                ("budget_bytes", ctypes.c_size_t)]


class sgmf_shape(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("max_disp", ctypes.c_int32)]


def mask_words(D: int) -> int:
    """Word planes of the box-OR masks: Dp / 32 with Dp = 64, 128, 192 or 256."""
    return 2 if D <= 64 else 4 if D <= 128 else 6 if D <= 192 else 8


@dataclass
class Params:
    """Mirror of sgmf_params; defaults are Table II of the paper."""

    p1: int = 10
    p2: int = 120
    q1: int = 5
    q2: int = 160
    alpha_num: int = 7
    alpha_den: int = 10
    ts: int = 2
    rs: int = 6
    tc: int = 2
    rc: int = 20
    lr_max_diff: int = 1
    census: int = SGMF_CENSUS_CS9X7
    semidense: int = 1
    consistency: int = SGMF_CHECK_STEREO_LIDAR
    num_paths: int = 8
    subpixel: int = 0

    def to_c(self) -> sgmf_params:
        return sgmf_params(**asdict(self))

    @classmethod
    def from_c(cls, c: sgmf_params) -> "Params":
        return cls(**{f.name: getattr(c, f.name) for f in fields(cls)})


_lib = None


def lib(path: str | None = None):
    """Load libsgmf.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} not built: run __graft_entry__.build() or "
                                "python paper_2504_05148_gb300/build.py")
    L = ctypes.CDLL(path)
    P, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    ctx_pp = ctypes.POINTER(ctypes.c_void_p)
    prm_p = ctypes.POINTER(sgmf_params)
    sig = {
        "sgmf_default_params": (None, [prm_p]),
        "sgmf_create": (i, [i, i, i, ctx_pp]),
        "sgmf_create_batched": (i, [i, i, i, i, ctx_pp]),
        "sgmf_batch_capacity": (i, [P]),
        "sgmf_compute_batch": (i, [P, i, P, P, P, P]),
        "sgmf_compute_host_batch": (i, [P, i, P, P, P, P]),
        "sgmf_compute_host_batch_async": (i, [P, i, P, P, P, P]),
        "sgmf_set_params": (i, [P, prm_p]),
        "sgmf_get_params": (i, [P, prm_p]),
        "sgmf_set_stream": (i, [P, P]),
        "sgmf_compute": (i, [P, P, P, P, P]),
        "sgmf_compute_host": (i, [P, P, P, P, P]),
        "sgmf_sync": (i, [P]),
        "sgmf_destroy": (None, [P]),
        "sgmf_last_error": (ctypes.c_char_p, [P]),
        "sgmf_status_string": (ctypes.c_char_p, [i]),
        "sgmf_set_debug": (i, [P, i]),
        "sgmf_debug_stage": (i, [P, i, P, sz]),
        "sgmf_launches_per_compute": (i, [P]),
        "sgmf_set_profiling": (i, [P, i]),
        "sgmf_kernel_times": (i, [P, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_float),
                                  ctypes.POINTER(ctypes.c_int)]),
        "sgmf_device_bytes": (sz, [P]),
        "sgmf_set_wait_limit": (i, [P, i, ctypes.c_longlong]),
        "sgmf_debug_fail_alloc": (None, [i]),
        "sgmf_measure_rates": (i, [i, ctypes.POINTER(sgmf_rates)]),
        "sgmf_check_static": (i, [i, i, i, prm_p, P, P, P, P, P]),
        "sgmf_set_tuning": (i, [P, ctypes.POINTER(sgmf_tuning)]),
        "sgmf_get_tuning": (i, [P, ctypes.POINTER(sgmf_tuning)]),
        "sgmf_autotune": (i, [P, i, P, P, P, P, i, ctypes.POINTER(sgmf_tuning), ctypes.POINTER(ctypes.c_float)]),
        "sgmf_multi_create": (i, [ctypes.POINTER(sgmf_shape), i, prm_p, ctx_pp]),
        "sgmf_multi_frame": (i, [P, i, ctx_pp, ctx_pp, ctx_pp, ctx_pp]),
        "sgmf_multi_classes": (i, [P]),
        "sgmf_multi_class_info": (i, [P, i, ctypes.POINTER(sgmf_shape), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(sgmf_tuning)]),
        "sgmf_multi_autotune": (i, [P, i]),
        "sgmf_multi_launch": (i, [P, P]),
        "sgmf_multi_sync": (i, [P]),
        "sgmf_multi_launches": (i, [P]),
        "sgmf_multi_device_bytes": (sz, [P]),
        "sgmf_multi_destroy": (None, [P]),
        "sgmf_server_create": (i, [prm_p, sz, i, i, ctx_pp]),
        "sgmf_server_add_camera": (i, [P, i, i, i]),
        "sgmf_server_submit": (i, [P, i, P, P, P, P, ctypes.c_uint64]),
        "sgmf_server_poll": (i, [P, i, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
        "sgmf_server_stats": (i, [P, ctypes.POINTER(sgmf_server_counters)]),
        "sgmf_server_destroy": (None, [P]),
        "sgmf_create_banded": (i, [i, i, i, i, i, ctx_pp]),
        "sgmf_compute_banded": (i, [P, i, P, P, P, P, P]),
        "sgmf_band_width": (i, [P]),
        "sgmf_compute_front": (i, [P, i, P, P, P]),
        "sgmf_prior_device": (P, [P]),
        "sgmf_compute_banded_back": (i, [P, i, P, P]),
        "sgmf_bn_pack": (i, [P, P, P, P]),
        "sgmf_bn_conv": (i, [i, i, i, P, P, P, i, P, P, P, P, P]),
        "sgmf_bn_wgrad": (i, [i, i, i, P, P, P, P, P, P]),
        "sgmf_bn_input": (i, [i, i, i, i, P, P, P, P]),
        "sgmf_bn_labels": (i, [i, i, i, P, P, P, P]),
        "sgmf_bn_loss": (i, [ctypes.c_longlong, i, P, P, P, P, P, ctypes.c_float, ctypes.c_float, P]),
        "sgmf_bn_adam": (i, [i, P, P, P, P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, i, P,
                             P]),
        "sgmf_bn_tiles": (i, [i, i, i, i, i, ctypes.c_float, P, P, P, P]),
        "sgmf_bn_gather": (i, [i, P, ctypes.c_longlong, ctypes.c_longlong, P, P, P]),
        "sgmf_bn_to_bf16": (i, [i, P, P, P]),
        "sgmf_bn_decide": (i, [i, i, ctypes.c_float, P, i, i, P, P]),
        "sgmf_set_gate": (i, [P, P, i]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _status_name(s: int) -> str:
    try:
        return lib().sgmf_status_string(s).decode()
    except Exception:
        return f"status {s}"


def _check(status: int, ctx=None) -> None:
    if status != SGMF_OK:
        raise SgmfError(status, lib().sgmf_last_error(ctx).decode())


# ---- one function per entry point ---------------------------------------------

def sgmf_default_params() -> Params:
    c = sgmf_params()
    lib().sgmf_default_params(ctypes.byref(c))
    return Params.from_c(c)


def sgmf_create(width: int, height: int, max_disp: int) -> int:
    out = ctypes.c_void_p()
    _check(lib().sgmf_create(width, height, max_disp, ctypes.byref(out)), None)
    return out.value


def sgmf_create_batched(width: int, height: int, max_disp: int, max_batch: int) -> int:
    out = ctypes.c_void_p()
    _check(lib().sgmf_create_batched(width, height, max_disp, max_batch, ctypes.byref(out)), None)
    return out.value


def sgmf_batch_capacity(ctx: int) -> int:
    return lib().sgmf_batch_capacity(ctx)


def sgmf_set_params(ctx: int, params: Params) -> None:
    c = params.to_c()
    _check(lib().sgmf_set_params(ctx, ctypes.byref(c)), ctx)


def sgmf_get_params(ctx: int) -> Params:
    c = sgmf_params()
    _check(lib().sgmf_get_params(ctx, ctypes.byref(c)), ctx)
    return Params.from_c(c)


def sgmf_set_stream(ctx: int, stream: int | None) -> None:
    _check(lib().sgmf_set_stream(ctx, stream or None), ctx)


def sgmf_compute(ctx: int, left: int, right: int, lidar: int | None, out: int) -> None:
    """Device pointers (ints); lidar may be None."""
    _check(lib().sgmf_compute(ctx, left, right, lidar or None, out), ctx)


def sgmf_compute_batch(ctx: int, n: int, left: int, right: int, lidar: int | None, out: int) -> None:
    """n frames, contiguous [n][H][W] device buffers; lidar may be None."""
    _check(lib().sgmf_compute_batch(ctx, n, left, right, lidar or None, out), ctx)


def sgmf_compute_host_batch(ctx: int, n: int, left: int, right: int, lidar: int | None, out: int) -> None:
    """n frames, contiguous [n][H][W] host buffers.  Waits for the result."""
    _check(lib().sgmf_compute_host_batch(ctx, n, left, right, lidar or None, out), ctx)


def sgmf_compute_host_batch_async(ctx: int, n: int, left: int, right: int, lidar: int | None, out: int) -> None:
    """As sgmf_compute_host_batch, without waiting (sgmf_sync waits); pinned host buffers."""
    _check(lib().sgmf_compute_host_batch_async(ctx, n, left, right, lidar or None, out), ctx)


def sgmf_compute_host(ctx: int, left: int, right: int, lidar: int | None, out: int) -> None:
    """Host pointers (ints); lidar may be None.  Waits for the result."""
    _check(lib().sgmf_compute_host(ctx, left, right, lidar or None, out), ctx)


def sgmf_sync(ctx: int) -> None:
    _check(lib().sgmf_sync(ctx), ctx)


def sgmf_destroy(ctx: int | None) -> None:
    lib().sgmf_destroy(ctx)


def sgmf_last_error(ctx: int | None) -> str:
    return lib().sgmf_last_error(ctx).decode()


def sgmf_set_debug(ctx: int, enable: bool) -> None:
    _check(lib().sgmf_set_debug(ctx, int(bool(enable))), ctx)


def sgmf_debug_stage(ctx: int, stage: int, host_ptr: int, nbytes: int) -> None:
    _check(lib().sgmf_debug_stage(ctx, stage, host_ptr, nbytes), ctx)


def sgmf_launches_per_compute(ctx: int) -> int:
    return lib().sgmf_launches_per_compute(ctx)


def sgmf_set_profiling(ctx: int, enable: bool) -> None:
    _check(lib().sgmf_set_profiling(ctx, int(bool(enable))), ctx)


def sgmf_kernel_times(ctx: int, cap: int = 32) -> list[tuple[str, float]]:
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_float * cap)()
    n = ctypes.c_int(cap)
    _check(lib().sgmf_kernel_times(ctx, names, ms, ctypes.byref(n)), ctx)
    return [(names[i].decode(), float(ms[i])) for i in range(min(n.value, cap))]


def sgmf_device_bytes(ctx: int) -> int:
    return lib().sgmf_device_bytes(ctx)


def sgmf_set_wait_limit(ctx: int, which: int, polls: int) -> None:
    """Poll limit of one kind of device wait (polls < 0: the default)."""
    _check(lib().sgmf_set_wait_limit(ctx, which, polls), ctx)


def sgmf_debug_fail_alloc(n: int) -> None:
    """Test hook: the n-th device allocation from now on, on this thread, fails (n <= 0: off)."""
    lib().sgmf_debug_fail_alloc(n)


def sgmf_measure_rates(iters: int = 256) -> dict:
    """Lanes per clock per SM of the path's instruction kinds on the current device."""
    r = sgmf_rates()
    _check(lib().sgmf_measure_rates(iters, ctypes.byref(r)), None)
    return {k: getattr(r, k) for k, _ in sgmf_rates._fields_}


def sgmf_check_static(width: int, height: int, max_disp: int, params: Params, dstar: int, dprime: int,
                      lidar: int | None, out: int, stream: int | None = None) -> None:
    """Consistency stage without a context or allocation (device pointers)."""
    c = params.to_c()
    _check(lib().sgmf_check_static(width, height, max_disp, ctypes.byref(c), dstar, dprime, lidar or None, out,
                                   stream or None), None)


def sgmf_create_banded(width: int, height: int, max_disp: int, band: int, max_batch: int) -> int:
    out = ctypes.c_void_p()
    _check(lib().sgmf_create_banded(width, height, max_disp, band, max_batch, ctypes.byref(out)), None)
    return out.value


def sgmf_compute_banded(ctx: int, n: int, left: int, right: int, lidar: int | None, band_lo: int, out: int) -> None:
    """Device pointers; band_lo int16 [n][ceil(H/8)][ceil(W/8)]."""
    _check(lib().sgmf_compute_banded(ctx, n, left, right, lidar or None, band_lo, out), ctx)


def sgmf_band_width(ctx: int) -> int:
    return lib().sgmf_band_width(ctx)


def sgmf_compute_front(ctx: int, n: int, left: int, right: int, lidar: int | None) -> None:
    _check(lib().sgmf_compute_front(ctx, n, left, right, lidar or None), ctx)


def sgmf_prior_device(ctx: int) -> int:
    return lib().sgmf_prior_device(ctx)


def sgmf_compute_banded_back(ctx: int, n: int, band_lo: int, out: int) -> None:
    _check(lib().sgmf_compute_banded_back(ctx, n, band_lo, out), ctx)


# band-proposal network kernels (device pointers; asynchronous on `stream`)
def sgmf_bn_pack(w: int, packed_fwd: int | None, packed_dgrad: int | None, stream: int | None = None) -> None:
    _check(lib().sgmf_bn_pack(w, packed_fwd or None, packed_dgrad or None, stream or None), None)


def sgmf_bn_conv(n: int, h: int, w: int, x: int, packed: int, bias: int | None, relu: bool, mask: int | None,
                 y: int | None, yf: int | None, err: int, stream: int | None = None) -> None:
    _check(lib().sgmf_bn_conv(n, h, w, x, packed, bias or None, int(bool(relu)), mask or None, y or None,
                              yf or None, err, stream or None), None)


def sgmf_bn_wgrad(n: int, h: int, w: int, x: int, dy: int, dw: int, db: int, err: int,
                  stream: int | None = None) -> None:
    _check(lib().sgmf_bn_wgrad(n, h, w, x, dy, dw, db, err, stream or None), None)


def sgmf_bn_input(n: int, width: int, height: int, max_disp: int, left: int, dhat: int, x: int,
                  stream: int | None = None) -> None:
    _check(lib().sgmf_bn_input(n, width, height, max_disp, left, dhat, x, stream or None), None)


def sgmf_bn_labels(n: int, width: int, height: int, disp: int, lohi: int, count: int,
                   stream: int | None = None) -> None:
    _check(lib().sgmf_bn_labels(n, width, height, disp, lohi, count, stream or None), None)


def sgmf_bn_loss(npix: int, max_disp: int, out: int, lohi: int, count: int, grad: int, loss: int,
                 lam_c: float = 1.0, lam_w: float = 0.25, stream: int | None = None) -> None:
    _check(lib().sgmf_bn_loss(npix, max_disp, out, lohi, count, grad, loss, lam_c, lam_w, stream or None), None)


def sgmf_bn_adam(count: int, w: int, m: int, v: int, g: int, lr: float, b1: float, b2: float, eps: float,
                 step: int, w_bf16: int | None, stream: int | None = None) -> None:
    _check(lib().sgmf_bn_adam(count, w, m, v, g, lr, b1, b2, eps, step, w_bf16 or None, stream or None), None)


def sgmf_bn_tiles(n: int, width: int, height: int, max_disp: int, band: int, conf_min: float, out: int,
                  lo_tiles: int, uncertain: int, stream: int | None = None) -> None:
    _check(lib().sgmf_bn_tiles(n, width, height, max_disp, band, conf_min, out, lo_tiles, uncertain,
                               stream or None), None)


def sgmf_bn_gather(n: int, idx: int, rows: int, row_bytes: int, src: int, dst: int, stream: int | None = None) -> None:
    """dst row i = src row idx[i] (device pointers; idx int32 on the device)."""
    _check(lib().sgmf_bn_gather(n, idx, rows, row_bytes, src, dst, stream or None), None)


def sgmf_bn_to_bf16(count: int, w: int, w_bf16: int, stream: int | None = None) -> None:
    _check(lib().sgmf_bn_to_bf16(count, w, w_bf16, stream or None), None)


def sgmf_bn_decide(n: int, tiles: int, max_frac: float, uncertain: int, value: int, otherwise: int, gate: int,
                   stream: int | None = None) -> None:
    _check(lib().sgmf_bn_decide(n, tiles, max_frac, uncertain, value, otherwise, gate, stream or None), None)


def sgmf_set_gate(ctx: int, gate: int | None, run: int = 0) -> None:
    """Per-frame gating of the context's kernels (gate: device int pointer or None)."""
    _check(lib().sgmf_set_gate(ctx, gate or None, run), ctx)


def sgmf_set_tuning(ctx: int, line_warps: int, cost_px: int, sweep: int = 0, parts: int = 1) -> None:
    t = sgmf_tuning(line_warps, cost_px, sweep, parts)
    _check(lib().sgmf_set_tuning(ctx, ctypes.byref(t)), ctx)


def sgmf_tuning_of(ctx: int) -> sgmf_tuning:
    """The context's whole tuning struct (sgmf_get_tuning returns its first three fields)."""
    t = sgmf_tuning()
    _check(lib().sgmf_get_tuning(ctx, ctypes.byref(t)), ctx)
    return t


def sgmf_get_tuning(ctx: int) -> tuple[int, int, int]:
    """(line_warps, cost_px, sweep)"""
    t = sgmf_tuning()
    _check(lib().sgmf_get_tuning(ctx, ctypes.byref(t)), ctx)
    return t.line_warps, t.cost_px, t.sweep


def sgmf_autotune(ctx: int, n: int, left: int, right: int, lidar: int | None, out: int,
                  reps: int = 3) -> tuple[tuple[int, int, int], float]:
    """Device pointers; returns ((line_warps, cost_px, sweep), median ms) of the winner."""
    t = sgmf_tuning()
    ms = ctypes.c_float()
    _check(lib().sgmf_autotune(ctx, n, left, right, lidar or None, out, reps, ctypes.byref(t),
                               ctypes.byref(ms)), ctx)
    return (t.line_warps, t.cost_px, t.sweep), ms.value


def sgmf_multi_create(shapes: list[tuple[int, int, int]], params: Params | None = None) -> int:
    """shapes: (width, height, max_disp) per frame."""
    arr = (sgmf_shape * len(shapes))(*[sgmf_shape(*s) for s in shapes])
    out = ctypes.c_void_p()
    c = params.to_c() if params is not None else None
    _check(lib().sgmf_multi_create(arr, len(shapes), ctypes.byref(c) if c is not None else None,
                                   ctypes.byref(out)), None)
    return out.value


def sgmf_multi_frame(m: int, i: int) -> tuple[int, int, int, int]:
    """Device pointers (left, right, lidar, out) of frame i's resident buffers."""
    ptrs = [ctypes.c_void_p() for _ in range(4)]
    _check(lib().sgmf_multi_frame(m, i, *[ctypes.byref(p) for p in ptrs]), None)
    return tuple(p.value for p in ptrs)


def sgmf_multi_classes(m: int) -> int:
    return lib().sgmf_multi_classes(m)


def sgmf_multi_class_info(m: int, cls: int) -> tuple[tuple[int, int, int], int, tuple[int, int, int]]:
    s, n, t = sgmf_shape(), ctypes.c_int(), sgmf_tuning()
    _check(lib().sgmf_multi_class_info(m, cls, ctypes.byref(s), ctypes.byref(n), ctypes.byref(t)), None)
    return (s.width, s.height, s.max_disp), n.value, (t.line_warps, t.cost_px, t.sweep)


def sgmf_multi_autotune(m: int, reps: int = 3) -> None:
    _check(lib().sgmf_multi_autotune(m, reps), None)


def sgmf_multi_launch(m: int, stream: int | None = None) -> None:
    _check(lib().sgmf_multi_launch(m, stream or None), None)


def sgmf_multi_sync(m: int) -> None:
    _check(lib().sgmf_multi_sync(m), None)


def sgmf_multi_launches(m: int) -> int:
    return lib().sgmf_multi_launches(m)


def sgmf_multi_device_bytes(m: int) -> int:
    return lib().sgmf_multi_device_bytes(m)


def sgmf_multi_destroy(m: int | None) -> None:
    lib().sgmf_multi_destroy(m)


def sgmf_server_create(params: Params | None, budget_bytes: int, max_batch: int, max_slots_per_shape: int) -> int:
    out = ctypes.c_void_p()
    c = params.to_c() if params is not None else None
    _check(lib().sgmf_server_create(ctypes.byref(c) if c is not None else None, budget_bytes, max_batch,
                                    max_slots_per_shape, ctypes.byref(out)), None)
    return out.value


def sgmf_server_add_camera(srv: int, width: int, height: int, max_disp: int) -> int:
    r = lib().sgmf_server_add_camera(srv, width, height, max_disp)
    if r < 0:
        raise SgmfError(-r, sgmf_last_error(None))
    return r


def sgmf_server_submit(srv: int, camera: int, left: int, right: int, lidar: int | None, out: int,
                       tag: int) -> None:
    """Host pointers that must stay valid until the request is polled."""
    _check(lib().sgmf_server_submit(srv, camera, left, right, lidar or None, out, tag), None)


def sgmf_server_poll(srv: int, wait_ms: int):
    """None, or (tag, camera, status, latency_ms) of one finished request."""
    tag, cam, st, lat = ctypes.c_uint64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    r = lib().sgmf_server_poll(srv, wait_ms, ctypes.byref(tag), ctypes.byref(cam), ctypes.byref(st),
                               ctypes.byref(lat))
    if r < 0:
        raise SgmfError(-r, "sgmf_server_poll")
    return None if r == 0 else (tag.value, cam.value, st.value, lat.value)


def sgmf_server_stats(srv: int) -> dict:
    c = sgmf_server_counters()
    _check(lib().sgmf_server_stats(srv, ctypes.byref(c)), None)
    return {k: getattr(c, k) for k, _ in c._fields_}


def sgmf_server_destroy(srv: int | None) -> None:
    lib().sgmf_server_destroy(srv)


# ---- torch convenience wrapper ------------------------------------------------------

class Context:
    """Owns one sgmf context for a (width, height, max_disp) shape."""

    def __init__(self, width: int, height: int, max_disp: int, params: Params | None = None,
                 stream=None, max_batch: int = 1, band: int = 0):
        self.W, self.H, self.D = width, height, max_disp
        self.max_batch = max_batch
        self.band = band
        self.handle = (sgmf_create_banded(width, height, max_disp, band, max_batch) if band
                       else sgmf_create_batched(width, height, max_disp, max_batch))
        if params is not None:
            sgmf_set_params(self.handle, params)
        if stream is not None:
            self.set_stream(stream)

    def set_stream(self, stream) -> None:
        sgmf_set_stream(self.handle, getattr(stream, "cuda_stream", stream))

    def set_params(self, params: Params) -> None:
        sgmf_set_params(self.handle, params)

    def compute(self, left, right, lidar, out) -> None:
        """torch CUDA tensors: uint8 (H, W) or (n, H, W) x2, float32 of the same
        shape or None, int16 of the same shape."""
        shape = tuple(left.shape)
        if shape == (self.H, self.W):
            n = 1
        elif len(shape) == 3 and shape[1:] == (self.H, self.W) and 1 <= shape[0] <= self.max_batch:
            n = shape[0]
        else:
            raise ValueError(f"expected (H, W) = {(self.H, self.W)} or (n <= {self.max_batch}, H, W), got {shape}")
        for t, dt in ((left, "torch.uint8"), (right, "torch.uint8"), (out, "torch.int16")):
            if str(t.dtype) != dt or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != shape:
                raise ValueError(f"expected contiguous CUDA {dt} of shape {shape}")
        lp = None
        if lidar is not None:
            if str(lidar.dtype) != "torch.float32" or not lidar.is_cuda or not lidar.is_contiguous() \
                    or tuple(lidar.shape) != shape:
                raise ValueError(f"lidar must be a contiguous CUDA float32 {shape} tensor or None")
            lp = lidar.data_ptr()
        sgmf_compute_batch(self.handle, n, left.data_ptr(), right.data_ptr(), lp, out.data_ptr())

    def compute_banded(self, left, right, lidar, band_lo, out) -> None:
        """torch CUDA tensors as in compute(), plus band_lo: int16 (n, ceil(H/8), ceil(W/8))
        (or without the frame axis for one frame)."""
        shape = tuple(left.shape)
        n = 1 if len(shape) == 2 else shape[0]
        th, tw = (self.H + BAND_TILE - 1) // BAND_TILE, (self.W + BAND_TILE - 1) // BAND_TILE
        if str(band_lo.dtype) != "torch.int16" or not band_lo.is_cuda or not band_lo.is_contiguous() \
                or band_lo.numel() != n * th * tw:
            raise ValueError(f"band_lo must be a contiguous CUDA int16 tensor of {n} x {th} x {tw}")
        for t in (left, right, out):
            if not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != shape:
                raise ValueError("left, right and out must be contiguous CUDA tensors of one shape")
        sgmf_compute_banded(self.handle, n, left.data_ptr(), right.data_ptr(),
                            lidar.data_ptr() if lidar is not None else None, band_lo.data_ptr(), out.data_ptr())

    def compute_host(self, left, right, lidar, out) -> None:
        """numpy arrays (H, W) or (n, H, W); blocks until `out` holds the result."""
        import numpy as np
        shape = left.shape
        if shape == (self.H, self.W):
            n = 1
        elif len(shape) == 3 and shape[1:] == (self.H, self.W) and 1 <= shape[0] <= self.max_batch:
            n = shape[0]
        else:
            raise ValueError(f"expected (H, W) = {(self.H, self.W)} or (n <= {self.max_batch}, H, W), got {shape}")
        for a, dt in ((left, np.uint8), (right, np.uint8), (out, np.int16)):
            if a.dtype != dt or not a.flags["C_CONTIGUOUS"] or a.shape != shape:
                raise ValueError(f"expected C-contiguous {dt} of shape {shape}")
        lp = None
        if lidar is not None:
            if lidar.dtype != np.float32 or not lidar.flags["C_CONTIGUOUS"] or lidar.shape != shape:
                raise ValueError(f"lidar must be C-contiguous float32 {shape} or None")
            lp = lidar.ctypes.data
        sgmf_compute_host_batch(self.handle, n, left.ctypes.data, right.ctypes.data, lp, out.ctypes.data)

    def sync(self) -> None:
        sgmf_sync(self.handle)

    def stage(self, stage: int):
        """Copy an intermediate of the last compute to a numpy array."""
        import numpy as np
        shape2 = (self.H, self.W)
        spec = {
            SGMF_STAGE_DBAR: (np.int16, shape2), SGMF_STAGE_DHAT: (np.int16, shape2),
            SGMF_STAGE_DSTAR: (np.int16, shape2), SGMF_STAGE_DPRIME: (np.int16, shape2),
            SGMF_STAGE_DSUB: (np.int16, shape2),
            SGMF_STAGE_CENSUS_L: (np.uint64, shape2), SGMF_STAGE_CENSUS_R: (np.uint64, shape2),
            SGMF_STAGE_COST: (np.uint8, shape2 + (self.band or self.D,)),
            SGMF_STAGE_SUM: (np.uint16, shape2 + (self.band or self.D,)),
            SGMF_STAGE_BOX_S: (np.uint32, (mask_words(self.D),) + shape2),
            SGMF_STAGE_BOX_C: (np.uint32, (mask_words(self.D),) + shape2),
        }[stage]
        a = np.empty(spec[1], spec[0])
        sgmf_debug_stage(self.handle, stage, a.ctypes.data, a.nbytes)
        return a

    def set_debug(self, enable: bool) -> None:
        sgmf_set_debug(self.handle, enable)

    def launches_per_compute(self) -> int:
        return sgmf_launches_per_compute(self.handle)

    def set_profiling(self, enable: bool) -> None:
        sgmf_set_profiling(self.handle, enable)

    def kernel_times(self):
        return sgmf_kernel_times(self.handle)

    def device_bytes(self) -> int:
        return sgmf_device_bytes(self.handle)

    def close(self) -> None:
        if self.handle:
            sgmf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Multi:
    """A mixed-size batch replayed as one CUDA graph (resident buffers per frame)."""

    def __init__(self, shapes: list[tuple[int, int, int]], params: Params | None = None):
        self.shapes = [tuple(s) for s in shapes]
        self.handle = sgmf_multi_create(self.shapes, params)

    def frame_views(self, i: int):
        """torch tensors viewing frame i's resident device buffers: left, right, lidar, out."""
        import torch
        W, H, _ = self.shapes[i]
        lp, rp, dp, op = sgmf_multi_frame(self.handle, i)
        return (_device_view(lp, (H, W), torch.uint8), _device_view(rp, (H, W), torch.uint8),
                _device_view(dp, (H, W), torch.float32), _device_view(op, (H, W), torch.int16))

    def classes(self):
        return [sgmf_multi_class_info(self.handle, c) for c in range(sgmf_multi_classes(self.handle))]

    def autotune(self, reps: int = 3) -> None:
        sgmf_multi_autotune(self.handle, reps)

    def launch(self, stream=None) -> None:
        sgmf_multi_launch(self.handle, getattr(stream, "cuda_stream", stream))

    def sync(self) -> None:
        sgmf_multi_sync(self.handle)

    def launches(self) -> int:
        return sgmf_multi_launches(self.handle)

    def device_bytes(self) -> int:
        return sgmf_multi_device_bytes(self.handle)

    def close(self) -> None:
        if self.handle:
            sgmf_multi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _device_view(ptr: int, shape: tuple[int, ...], dtype):
    """A torch tensor over device memory owned by the library (no copy, no ownership)."""
    import torch

    class _Mem:
        def __init__(self, p, nbytes):
            self.__cuda_array_interface__ = {
                "shape": shape, "typestr": {torch.uint8: "|u1", torch.float32: "<f4", torch.int16: "<i2"}[dtype],
                "data": (p, False), "version": 3, "strides": None}

    n = 1
    for s in shape:
        n *= s
    return torch.as_tensor(_Mem(ptr, n), device="cuda")

