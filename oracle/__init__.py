"""CPU oracle for the stereo-LiDAR SGM pipeline (test infrastructure only).

This package wraps ``sgmf_oracle.c``: a plain, slow, single-threaded C
statement of the paper's pipeline (census/Hamming cost, DDC of Eq. 4,
semidensification of Eq. 5, the SGM path recursion of Eq. 2, WTA of Eq. 3
and the three-view consistency check of Eq. 6).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The CUDA library never calls it, shares no source
with it, and the product path fails if its own extension is missing instead
of falling back to this code.

Parity status: every stage is pinned by the CPU tests in
``tests/test_oracle_pins.py`` (brute-force dynamic programming, closed forms,
invariances and hand-computed values); see the docstring of each wrapper.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, asdict

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgmf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsgmf_oracle.so")
_lock = threading.Lock()
_lib = None

# consistency modes (Table V: stereo, camera-LiDAR, stereo-LiDAR) and census kinds
CHECK_STEREO_LIDAR, CHECK_STEREO, CHECK_LIDAR, CHECK_NONE = 0, 1, 2, 3
CENSUS_CS9X7, CENSUS_9X7 = 0, 1
INVALID = -1

# The eight path directions r = (rx, ry) of Sec. III; L_r(p) is built from L_r(p - r).
DIRECTIONS = [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1), (1, -1), (-1, 1)]


@dataclass
class Params:
    """Table II of the paper, plus the readings for what it leaves open."""

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
    census: int = CENSUS_CS9X7
    semidense: int = 1
    consistency: int = CHECK_STEREO_LIDAR
    num_paths: int = 8
    subpixel: int = 0


class _CParams(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int32) for k in (
        "p1", "p2", "q1", "q2", "alpha_num", "alpha_den", "ts", "rs", "tc", "rc",
        "lr_max_diff", "census", "semidense", "consistency", "num_paths", "subpixel")]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build`` (no GPU needed)."""
    with _lock:
        if (not force and os.path.exists(_SO)
                and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
            return _SO
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
        return _SO


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i = ctypes.c_int
        L.sgmfo_lidar.argtypes = [i, i, i, P, P]
        L.sgmfo_census.argtypes = [i, i, P, i, P]
        L.sgmfo_census_bits.argtypes = [i]
        L.sgmfo_census_bits.restype = i
        L.sgmfo_hamming.argtypes = [i, i, i, P, P, i, P]
        L.sgmfo_semidense.argtypes = [i, i, i, P, P, i, i, P]
        L.sgmfo_ddc.argtypes = [i, i, i, P, P, i, i, i, i, P]
        L.sgmfo_path.argtypes = [i, i, i, P, i, i, i, i, P]
        L.sgmfo_aggregate.argtypes = [i, i, i, P, i, i, i, P]
        L.sgmfo_aggregate.restype = i
        L.sgmfo_wta.argtypes = [i, i, i, P, P, P]
        L.sgmfo_subpixel.argtypes = [i, i, i, P, P, P]
        L.sgmfo_consistency.argtypes = [i, i, P, P, P, i, i, i, i, P]
        L.sgmfo_compute.argtypes = [ctypes.POINTER(_CParams), i, i, i, P, P, P, P,
                                    P, P, P, P, P, P, P, P]
        L.sgmfo_compute.restype = i
        L.sgmfo_path_banded.argtypes = [i, i, i, i, P, P, i, i, i, i, P]
        L.sgmfo_aggregate_banded.argtypes = [i, i, i, i, P, P, i, i, i, P]
        L.sgmfo_aggregate_banded.restype = i
        L.sgmfo_wta_banded.argtypes = [i, i, i, i, P, P, P, P]
        L.sgmfo_compute_banded.argtypes = [ctypes.POINTER(_CParams), i, i, i, i, P, P, P, P, P, P, P, P]
        L.sgmfo_compute_banded.restype = i
        _lib = L
    return _lib


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# stage wrappers (numpy in, numpy out)

def lidar(lidar_f32: np.ndarray | None, D: int, shape=None) -> np.ndarray:
    """Sparse map d-bar (int16, -1 invalid) from a float map (0 = no return)."""
    if lidar_f32 is None:
        H, W = shape
        src = None
    else:
        src = _c(lidar_f32, np.float32)
        H, W = src.shape
    out = np.empty((H, W), np.int16)
    lib().sgmfo_lidar(W, H, D, _p(src), _p(out))
    return out


def census(img: np.ndarray, kind: int = CENSUS_CS9X7) -> np.ndarray:
    """Census image (uint64, bit k = k-th offset of the 9x7 window in raster order)."""
    src = _c(img, np.uint8)
    H, W = src.shape
    out = np.empty((H, W), np.uint64)
    lib().sgmfo_census(W, H, _p(src), kind, _p(out))
    return out


def census_bits(kind: int) -> int:
    return lib().sgmfo_census_bits(kind)


def hamming(cl: np.ndarray, cr: np.ndarray, D: int, nbits: int) -> np.ndarray:
    """H(p, d) as an int32 volume (H, W, D)."""
    cl = _c(cl, np.uint64)
    cr = _c(cr, np.uint64)
    H, W = cl.shape
    out = np.empty((H, W, D), np.int32)
    lib().sgmfo_hamming(W, H, D, _p(cl), _p(cr), nbits, _p(out))
    return out


def semidense(dbar: np.ndarray, hv: np.ndarray, ts: int, rs: int) -> np.ndarray:
    """d-hat of Eq. 5 (int16, -1 invalid)."""
    dbar = _c(dbar, np.int16)
    hv = _c(hv, np.int32)
    H, W, D = hv.shape
    out = np.empty((H, W), np.int16)
    lib().sgmfo_semidense(W, H, D, _p(dbar), _p(hv), ts, rs, _p(out))
    return out


def ddc(hv: np.ndarray, prior: np.ndarray, q1: int, q2: int, a: int, b: int) -> np.ndarray:
    """C-bar of Eq. 4 (int32 volume)."""
    hv = _c(hv, np.int32)
    prior = _c(prior, np.int16)
    H, W, D = hv.shape
    out = np.empty((H, W, D), np.int32)
    lib().sgmfo_ddc(W, H, D, _p(hv), _p(prior), q1, q2, a, b, _p(out))
    return out


def path(cv: np.ndarray, p1: int, p2: int, rx: int, ry: int) -> np.ndarray:
    """L_r of Eq. 2 for one direction r = (rx, ry) (int32 volume)."""
    cv = _c(cv, np.int32)
    H, W, D = cv.shape
    out = np.empty((H, W, D), np.int32)
    lib().sgmfo_path(W, H, D, _p(cv), p1, p2, rx, ry, _p(out))
    return out


def aggregate(cv: np.ndarray, p1: int, p2: int, num_paths: int = 8) -> np.ndarray:
    """S = sum_r L_r (int32 volume)."""
    cv = _c(cv, np.int32)
    H, W, D = cv.shape
    out = np.empty((H, W, D), np.int32)
    if lib().sgmfo_aggregate(W, H, D, _p(cv), p1, p2, num_paths, _p(out)) != 0:
        raise MemoryError("oracle aggregate: allocation failed")
    return out


def wta(sv: np.ndarray):
    """(d*, d') of Eq. 3 and the diagonal search of the other view."""
    sv = _c(sv, np.int32)
    H, W, D = sv.shape
    ds = np.empty((H, W), np.int16)
    dp = np.empty((H, W), np.int16)
    lib().sgmfo_wta(W, H, D, _p(sv), _p(ds), _p(dp))
    return ds, dp


def subpixel(sv: np.ndarray, dstar: np.ndarray) -> np.ndarray:
    """Sub-pixel disparity of the parabola fit (Sec. III), int16 in 1/16 px."""
    sv = _c(sv, np.int32)
    dstar = _c(dstar, np.int16)
    H, W, D = sv.shape
    out = np.empty((H, W), np.int16)
    lib().sgmfo_subpixel(W, H, D, _p(sv), _p(dstar), _p(out))
    return out


def consistency(dstar, dprime, dbar, tc: int, rc: int, lr_max_diff: int = 1,
                mode: int = CHECK_STEREO_LIDAR) -> np.ndarray:
    """D^{c*} of Eq. 6 (int16, -1 invalid)."""
    dstar = _c(dstar, np.int16)
    dprime = _c(dprime, np.int16)
    dbar = _c(dbar, np.int16)
    H, W = dstar.shape
    out = np.empty((H, W), np.int16)
    lib().sgmfo_consistency(W, H, _p(dstar), _p(dprime), _p(dbar), tc, rc, lr_max_diff,
                            mode, _p(out))
    return out


@dataclass
class Result:
    out: np.ndarray
    dbar: np.ndarray | None = None
    census_l: np.ndarray | None = None
    census_r: np.ndarray | None = None
    dhat: np.ndarray | None = None
    cost: np.ndarray | None = None
    sum: np.ndarray | None = None
    dstar: np.ndarray | None = None
    dprime: np.ndarray | None = None


def compute(left: np.ndarray, right: np.ndarray, lidar_f32: np.ndarray | None, D: int,
            params: Params | None = None, dumps: bool = True, volumes: bool = False) -> Result:
    """The whole pipeline (Fig. 1).  ``dumps`` returns the per-pixel maps,
    ``volumes`` also the C-bar and S volumes (int32, H x W x D)."""
    params = params or Params()
    left = _c(left, np.uint8)
    right = _c(right, np.uint8)
    H, W = left.shape
    assert right.shape == (H, W)
    li = None if lidar_f32 is None else _c(lidar_f32, np.float32)
    if li is not None:
        assert li.shape == (H, W)
    cp = _CParams(**asdict(params))
    out = np.empty((H, W), np.int16)
    r = Result(out=out)
    if dumps:
        r.dbar = np.empty((H, W), np.int16)
        r.census_l = np.empty((H, W), np.uint64)
        r.census_r = np.empty((H, W), np.uint64)
        r.dhat = np.empty((H, W), np.int16)
        r.dstar = np.empty((H, W), np.int16)
        r.dprime = np.empty((H, W), np.int16)
    if volumes:
        r.cost = np.empty((H, W, D), np.int32)
        r.sum = np.empty((H, W, D), np.int32)
    rc = lib().sgmfo_compute(ctypes.byref(cp), W, H, D, _p(left), _p(right), _p(li), _p(out),
                             _p(r.dbar), _p(r.census_l), _p(r.census_r), _p(r.dhat),
                             _p(r.cost), _p(r.sum), _p(r.dstar), _p(r.dprime))
    if rc != 0:
        raise MemoryError("oracle compute: allocation failed")
    return r


# ---- banded SGM (not in the paper: the method restricted to per-pixel bands) ----

ABSENT = 1 << 29


def expand_tiles(lo_tiles: np.ndarray, W: int, H: int, tile: int = 16) -> np.ndarray:
    """Per-pixel band starts from per-tile ones ([ceil(H/tile)][ceil(W/tile)])."""
    lo_tiles = np.asarray(lo_tiles)
    ys = np.arange(H) // tile
    xs = np.arange(W) // tile
    return np.ascontiguousarray(lo_tiles[ys[:, None], xs[None, :]].astype(np.int16))


def path_banded(cv: np.ndarray, lo: np.ndarray, B: int, p1: int, p2: int, rx: int, ry: int) -> np.ndarray:
    cv = _c(cv, np.int32)
    lo = _c(lo, np.int16)
    H, W, D = cv.shape
    out = np.empty_like(cv)
    lib().sgmfo_path_banded(W, H, D, B, _p(lo), _p(cv), p1, p2, rx, ry, _p(out))
    return out


def aggregate_banded(cv: np.ndarray, lo: np.ndarray, B: int, p1: int, p2: int, num_paths: int = 8) -> np.ndarray:
    cv = _c(cv, np.int32)
    lo = _c(lo, np.int16)
    H, W, D = cv.shape
    out = np.empty_like(cv)
    if lib().sgmfo_aggregate_banded(W, H, D, B, _p(lo), _p(cv), p1, p2, num_paths, _p(out)) != 0:
        raise MemoryError("oracle aggregate_banded: allocation failed")
    return out


def wta_banded(sv: np.ndarray, lo: np.ndarray, B: int):
    sv = _c(sv, np.int32)
    lo = _c(lo, np.int16)
    H, W, D = sv.shape
    ds = np.empty((H, W), np.int16)
    dp = np.empty((H, W), np.int16)
    lib().sgmfo_wta_banded(W, H, D, B, _p(lo), _p(sv), _p(ds), _p(dp))
    return ds, dp


def compute_banded(left, right, lidar_f32, D: int, B: int, lo: np.ndarray, params: Params | None = None,
                   volumes: bool = False) -> Result:
    """The pipeline with aggregation, WTA and check on the bands [lo, lo + B)."""
    params = params or Params()
    left = _c(left, np.uint8)
    right = _c(right, np.uint8)
    H, W = left.shape
    lo = _c(lo, np.int16)
    assert lo.shape == (H, W)
    li = None if lidar_f32 is None else _c(lidar_f32, np.float32)
    cp = _CParams(**asdict(params))
    r = Result(out=np.empty((H, W), np.int16))
    r.dstar = np.empty((H, W), np.int16)
    r.dprime = np.empty((H, W), np.int16)
    if volumes:
        r.sum = np.empty((H, W, D), np.int32)
    rc = lib().sgmfo_compute_banded(ctypes.byref(cp), W, H, D, B, _p(lo), _p(left), _p(right), _p(li), _p(r.out),
                                    _p(r.sum), _p(r.dstar), _p(r.dprime))
    if rc != 0:
        raise MemoryError("oracle compute_banded: allocation failed")
    return r

