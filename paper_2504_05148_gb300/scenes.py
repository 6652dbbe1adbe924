"""Seeded synthetic stereo + LiDAR scenes shaped like the paper's workloads.

The paper evaluates on KITTI 141, CARLA and Middlebury (Sec. V-A).  None of
them is available here, so every input is generated: a rectified uint8 stereo
pair, a float32 sparse disparity map aligned with the left view (0 = no
return) and the true left-view disparity.  This module holds no step of the
method itself (no census, cost, aggregation or check); it only draws inputs,
and both the CUDA path and the CPU oracle consume what it returns.

Scene model.  A scene is a list of planar layers, each with a region in the
left image and a disparity d(x, y) = a + bx * x + by * y.  The visible layer
at a left pixel is the one with the largest disparity (front-most).  The left
image is a blurred-noise texture.  A right pixel x' shows the front-most layer
whose back-projection x = x' + d lands on a left pixel of that same layer; it
takes the left texture there (linear interpolation along the row).  Right
pixels that no layer reaches are occluded in the left view and take fresh
texture.  Gaussian noise is added and the result rounded to uint8.

Recipes (all seeded with numpy PCG64):
  tiny(seed)            256x128, D=64: background at d=4 and 3 slanted planes
                        with d in [4, 60]; LiDAR on 16 evenly spaced rows,
                        every 4th column, truth + N(0, 0.3), 2 % outliers
                        uniform in [0, 64).
  kitti(seed, beams)    1242x375, D=128: sky/far layer, ground plane with d
                        rising linearly below the horizon (about 0 to 100),
                        20 slanted planar objects; 64-beam LiDAR on rows of
                        the lower 60 % spaced densely toward the horizon, each
                        column of a beam row kept with p = 0.29 (about 5 %
                        density), truth + N(0, 0.3), 1 % of the returns near a
                        depth edge take the other side's disparity.
                        beams = 64/32/16/8 keeps every 1/2/4/8-th beam.
  indoor(seed)          640x480, D=64: room of box-like planes with large walls
                        of constant intensity +-1 noise, textured boxes.
  lowlight(seed)        1280x720, D=192: the KITTI-like layout scaled up,
                        intensities in 0..40 and N(0, 3) noise.
  random_small(seed, W, H, D)  arbitrary small shapes for edge-case parity.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Scene:
    name: str
    seed: int
    D: int
    left: np.ndarray        # uint8 (H, W)
    right: np.ndarray       # uint8 (H, W)
    lidar: np.ndarray       # float32 (H, W), 0 = no return
    truth: np.ndarray       # float32 (H, W) left-view disparity

    @property
    def shape(self):
        return self.left.shape

    @property
    def W(self):
        return self.left.shape[1]

    @property
    def H(self):
        return self.left.shape[0]


@dataclass
class Layer:
    a: float
    bx: float
    by: float
    region: np.ndarray      # bool (H, W), in left-image coordinates
    texture: np.ndarray | None = None   # optional per-layer texture (float, H x W)

    def disp(self, x, y):
        return self.a + self.bx * x + self.by * y


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian_blur(img: np.ndarray, sigma: float = 1.5, radius: int = 5) -> np.ndarray:
    """Separable Gaussian blur with reflected borders (float64 out)."""
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    k /= k.sum()
    a = np.pad(img.astype(np.float64), radius, mode="reflect")
    h = sum(k[i] * a[:, i:i + img.shape[1]] for i in range(2 * radius + 1))
    v = sum(k[i] * h[i:i + img.shape[0], :] for i in range(2 * radius + 1))
    return v


def texture(rng: np.random.Generator, H: int, W: int, lo: float = 0.0, hi: float = 255.0) -> np.ndarray:
    """Uniform 0..255 noise, Gaussian-blurred (sigma 1.5 px), contrast-stretched
    so that mean +- 2.5 std spans [lo, hi], clipped (float64)."""
    t = gaussian_blur(rng.uniform(0.0, 255.0, size=(H, W)))
    t = (t - t.mean()) / max(t.std(), 1e-9)
    mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo)
    return np.clip(mid + t * (half / 2.5), lo, hi)


def _compose(layers: list[Layer], H: int, W: int):
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    best = np.full((H, W), -np.inf)
    label = np.full((H, W), -1, np.int32)
    for k, L in enumerate(layers):
        d = L.disp(xs, ys)
        m = L.region & (d > best)
        best[m] = d[m]
        label[m] = k
    if (label < 0).any():
        raise ValueError("layers do not cover the image")
    return label, best


def _sample_row_linear(tex: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    W = tex.shape[1]
    x0 = np.clip(np.floor(x).astype(np.int64), 0, W - 1)
    x1 = np.clip(x0 + 1, 0, W - 1)
    f = np.clip(x - x0, 0.0, 1.0)
    return (1.0 - f) * tex[y, x0] + f * tex[y, x1]


def render(rng: np.random.Generator, layers: list[Layer], H: int, W: int,
           base_tex: np.ndarray, fill_tex: np.ndarray, sigma_n: float,
           lo: float = 0.0, hi: float = 255.0):
    """Left/right uint8 images and the true left disparity of a layered scene."""
    label, truth = _compose(layers, H, W)
    left_f = base_tex.copy()
    for k, L in enumerate(layers):
        if L.texture is not None:
            m = label == k
            left_f[m] = L.texture[m]
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    yi = ys.astype(np.int64)
    best = np.full((H, W), -np.inf)
    right_f = fill_tex.copy()
    for k, L in enumerate(layers):
        denom = 1.0 - L.bx
        xk = (xs + L.a + L.by * ys) / denom          # left x seen at right x' via layer k
        inside = (xk >= 0.0) & (xk <= W - 1)
        xr = np.clip(np.rint(xk).astype(np.int64), 0, W - 1)
        ok = inside & (label[yi, xr] == k)
        dk = L.disp(xk, ys)
        m = ok & (dk > best)
        if not m.any():
            continue
        best[m] = dk[m]
        right_f[m] = _sample_row_linear(left_f, xk[m], yi[m])
    right_f = right_f + rng.normal(0.0, sigma_n, size=(H, W))
    left = np.clip(np.rint(left_f), lo, hi).astype(np.uint8)
    right = np.clip(np.rint(right_f), lo, hi).astype(np.uint8)
    return left, right, truth.astype(np.float32)


def _slanted_rect(rng, H, W, x0, y0, w, h, dc, dmin, dmax, slope):
    region = np.zeros((H, W), bool)
    xa, xb = max(0, int(x0)), min(W, int(x0 + w))
    ya, yb = max(0, int(y0)), min(H, int(y0 + h))
    region[ya:yb, xa:xb] = True
    cx, cy = 0.5 * (xa + xb - 1), 0.5 * (ya + yb - 1)
    bx, by = rng.uniform(-slope, slope, size=2)
    # keep the plane inside [dmin, dmax] over its rectangle
    span = abs(bx) * 0.5 * max(xb - xa, 1) + abs(by) * 0.5 * max(yb - ya, 1)
    room = min(dc - dmin, dmax - dc)
    if span > room and span > 0:
        s = max(room, 0.0) / span
        bx, by = bx * s, by * s
    return Layer(a=dc - bx * cx - by * cy, bx=bx, by=by, region=region)


def _beam_rows(H: int, n: int, top_frac: float = 0.4, power: float = 1.6) -> np.ndarray:
    top = int(round(top_frac * H))
    t = np.linspace(0.0, 1.0, n)
    rows = np.rint(top + (H - 1 - top) * t ** power).astype(np.int64)
    for i in range(1, n):                         # strictly increasing
        rows[i] = max(rows[i], rows[i - 1] + 1)
    return rows[rows < H]


def _beam_lidar(rng, truth, n_beams: int, keep_every: int, p_col: float,
                misproj_frac: float, D: int, top_frac: float = 0.4) -> np.ndarray:
    H, W = truth.shape
    rows = _beam_rows(H, n_beams, top_frac)[::keep_every]
    lid = np.zeros((H, W), np.float32)
    mask = np.zeros((H, W), bool)
    for r in rows:
        mask[r] = rng.random(W) < p_col
    vals = truth + rng.normal(0.0, 0.3, size=(H, W))
    # misprojections near depth edges: the other side's disparity
    pad = np.pad(truth, 3, mode="edge")
    win = np.lib.stride_tricks.sliding_window_view(pad, (7, 7))
    dmax, dmin = win.max(axis=(2, 3)), win.min(axis=(2, 3))
    near = mask & ((dmax - dmin) > 2.0)
    n_ret = int(mask.sum())
    cand = np.flatnonzero(near.ravel())
    k = min(len(cand), int(round(misproj_frac * n_ret)))
    if k > 0:
        pick = rng.choice(cand, size=k, replace=False)
        own = truth.ravel()[pick]
        hi_, lo_ = dmax.ravel()[pick], dmin.ravel()[pick]
        other = np.where(hi_ - own > own - lo_, hi_, lo_)
        vals.ravel()[pick] = other + rng.normal(0.0, 0.3, size=k)
    vals = np.clip(vals, 0.05, D - 1 + 0.45)
    lid[mask] = vals[mask]
    return lid.astype(np.float32)


def tiny(seed: int = 1000) -> Scene:
    """256x128, D=64 (the small case)."""
    rng = _rng(seed)
    H, W, D = 128, 256, 64
    layers = [Layer(a=4.0, bx=0.0, by=0.0, region=np.ones((H, W), bool))]
    for _ in range(3):
        w, h = rng.uniform(40, 120), rng.uniform(30, 80)
        x0, y0 = rng.uniform(0, W - w), rng.uniform(0, H - h)
        layers.append(_slanted_rect(rng, H, W, x0, y0, w, h, rng.uniform(10, 54), 4.0, 60.0, 0.08))
    base = texture(rng, H, W)
    fill = texture(rng, H, W)
    left, right, truth = render(rng, layers, H, W, base, fill, 2.0)
    lid = np.zeros((H, W), np.float32)
    rows = np.rint((np.arange(16) + 0.5) * H / 16).astype(np.int64)
    cols = np.arange(0, W, 4)
    yy, xx = np.meshgrid(rows, cols, indexing="ij")
    v = truth[yy, xx] + rng.normal(0.0, 0.3, size=yy.shape)
    out = rng.random(yy.shape) < 0.02
    v[out] = rng.uniform(0.0, 64.0, size=int(out.sum()))
    lid[yy, xx] = v
    return Scene("tiny_256x128_d64", seed, D, left, right, lid.astype(np.float32), truth)


def _street_layers(rng, H, W, dmax_ground, n_obj, obj_dmax):
    horizon = int(0.4 * H)
    layers = [Layer(a=1.5, bx=rng.uniform(-3e-4, 3e-4), by=0.0, region=np.ones((H, W), bool))]
    g = dmax_ground / (H - 1 - horizon)
    ground = np.zeros((H, W), bool)
    ground[horizon + 1:] = True
    layers.append(Layer(a=-g * horizon, bx=0.0, by=g, region=ground))
    for _ in range(n_obj):
        yb = rng.uniform(horizon + 8, H - 1)
        d0 = float(np.clip(g * (yb - horizon) + rng.uniform(1.0, 12.0), 3.0, obj_dmax))
        h = rng.uniform(0.6, 1.4) * (1.6 * d0 + 10.0)
        w = rng.uniform(0.5, 2.0) * h
        x0 = rng.uniform(-0.2 * w, W - 0.8 * w)
        layers.append(_slanted_rect(rng, H, W, x0, yb - h, w, h, d0, 1.0, obj_dmax + 5.0, 0.04))
    return layers


def kitti(seed: int = 2000, beams: int = 64) -> Scene:
    """1242x375, D=128, KITTI-shaped street scene with 64/32/16/8-beam LiDAR."""
    if beams not in (64, 32, 16, 8):
        raise ValueError("beams must be 64, 32, 16 or 8")
    rng = _rng(seed)
    H, W, D = 375, 1242, 128
    layers = _street_layers(rng, H, W, 100.0, 20, 115.0)
    base = texture(rng, H, W)
    fill = texture(rng, H, W)
    left, right, truth = render(rng, layers, H, W, base, fill, 2.0)
    lid = _beam_lidar(rng, truth, 64, 64 // beams, 0.29, 0.01, D)
    return Scene(f"kitti_1242x375_d128_{beams}beam", seed, D, left, right, lid, truth)


def street(seed: int, W: int, H: int, D: int, beams: int = 64) -> Scene:
    """The KITTI-shaped street scene at any size: ground-plane and object
    disparities scale with D / 128 (the band proposal's training pairs at
    1242 x 375 D = 128 and its evaluation pairs at 1920 x 1080 D = 256)."""
    rng = _rng(seed)
    s = D / 128.0
    layers = _street_layers(rng, H, W, 100.0 * s, 20, 115.0 * s)
    base = texture(rng, H, W)
    fill = texture(rng, H, W)
    left, right, truth = render(rng, layers, H, W, base, fill, 2.0)
    lid = _beam_lidar(rng, truth, 64, 64 // beams, 0.29, 0.01, D)
    return Scene(f"street_{W}x{H}_d{D}", seed, D, left, right, lid, truth)


def lowlight(seed: int = 3300) -> Scene:
    """1280x720, D=192, low-light pair: intensities 0..40, N(0, 3) noise."""
    rng = _rng(seed)
    H, W, D = 720, 1280, 192
    layers = _street_layers(rng, H, W, 150.0, 20, 180.0)
    base = texture(rng, H, W, 0.0, 40.0)
    fill = texture(rng, H, W, 0.0, 40.0)
    left, right, truth = render(rng, layers, H, W, base, fill, 3.0, 0.0, 40.0)
    lid = _beam_lidar(rng, truth, 64, 1, 0.29, 0.01, D)
    return Scene("lowlight_1280x720_d192", seed, D, left, right, lid, truth)


def indoor(seed: int = 3200) -> Scene:
    """640x480, D=64, box-like room with near-untextured walls."""
    rng = _rng(seed)
    H, W, D = 480, 640, 64
    full = np.ones((H, W), bool)
    ys, xs = np.mgrid[0:H, 0:W]

    def flat(level):
        return level + rng.integers(-1, 2, size=(H, W)).astype(np.float64)

    back = Layer(a=8.0, bx=rng.uniform(-2e-3, 2e-3), by=0.0, region=full, texture=flat(rng.uniform(90, 170)))
    floor_y = int(0.65 * H)
    gf = 30.0 / (H - 1 - floor_y)
    floor = Layer(a=8.0 - gf * floor_y, bx=0.0, by=gf, region=ys > floor_y, texture=texture(rng, H, W))
    lw = int(0.15 * W)
    gl = 20.0 / lw
    left_wall = Layer(a=28.0, bx=-gl, by=0.0, region=xs < lw, texture=flat(rng.uniform(60, 200)))
    right_wall = Layer(a=8.0 - gl * (W - 1 - lw), bx=gl, by=0.0, region=xs > W - 1 - lw,
                       texture=flat(rng.uniform(60, 200)))
    layers = [back, floor, left_wall, right_wall]
    for _ in range(6):
        w, h = rng.uniform(50, 200), rng.uniform(40, 160)
        x0, y0 = rng.uniform(0, W - w), rng.uniform(0.2 * H, H - h)
        L = _slanted_rect(rng, H, W, x0, y0, w, h, rng.uniform(15, 55), 12.0, 60.0, 0.05)
        L.texture = texture(rng, H, W)
        layers.append(L)
    base = texture(rng, H, W)
    fill = texture(rng, H, W)
    left, right, truth = render(rng, layers, H, W, base, fill, 2.0)
    lid = _beam_lidar(rng, truth, 64, 1, 0.29, 0.01, D, top_frac=0.05)
    return Scene("indoor_640x480_d64", seed, D, left, right, lid, truth)


MIXED_SHAPES = ((640, 480, 64), (1242, 375, 128), (1280, 720, 192), (1920, 1080, 256))


def mixed(seed: int, W: int, H: int, D: int) -> Scene:
    """A pair of any size built like the small case (fronto-parallel background
    and three slanted planes, blurred-noise texture, N(0, 2) sensor noise),
    with a 64-beam LiDAR model: the frames of the mixed-size batch."""
    rng = _rng(seed)
    s = D / 64.0
    layers = [Layer(a=4.0 * s, bx=0.0, by=0.0, region=np.ones((H, W), bool))]
    for _ in range(3):
        w, h = rng.uniform(0.15, 0.45) * W, rng.uniform(0.2, 0.6) * H
        x0, y0 = rng.uniform(0, W - w), rng.uniform(0, H - h)
        layers.append(_slanted_rect(rng, H, W, x0, y0, w, h, rng.uniform(10, 54) * s, 4.0 * s,
                                    min(60.0 * s, D - 1.0), 0.08))
    base = texture(rng, H, W)
    fill = texture(rng, H, W)
    left, right, truth = render(rng, layers, H, W, base, fill, 2.0)
    lid = _beam_lidar(rng, truth, 64, 1, 0.29, 0.01, D)
    return Scene(f"mixed_{W}x{H}_d{D}", seed, D, left, right, lid, truth)


def mixed_batch(n_per_shape: int = 12, distinct: int = 12, base_seed: int = 4000) -> list[Scene]:
    """The mixed-size batch: n_per_shape pairs of each of MIXED_SHAPES (48 by
    default).  `distinct` < n_per_shape reuses that many generated pairs per
    shape cyclically (generation of the largest pairs takes seconds each)."""
    out = []
    for j, (W, H, D) in enumerate(MIXED_SHAPES):
        made = [mixed(base_seed + 100 * j + i, W, H, D) for i in range(min(distinct, n_per_shape))]
        out += [made[i % len(made)] for i in range(n_per_shape)]
    return out


def random_small(seed: int, W: int, H: int, D: int, n_planes: int = 2,
                 density: float = 0.08) -> Scene:
    """Small random scene of any shape (edge cases: ragged and tiny sizes)."""
    rng = _rng(seed)
    dlo = min(2.0, D - 1.0)
    dhi = max(dlo, D - 1.0)
    layers = [Layer(a=float(rng.uniform(dlo, dhi)) if D > 1 else 0.0, bx=0.0, by=0.0,
                    region=np.ones((H, W), bool))]
    for _ in range(n_planes):
        w, h = rng.uniform(1, W + 1), rng.uniform(1, H + 1)
        x0, y0 = rng.uniform(-0.3 * w, W - 0.7 * w), rng.uniform(-0.3 * h, H - 0.7 * h)
        layers.append(_slanted_rect(rng, H, W, x0, y0, w, h, float(rng.uniform(dlo, dhi)),
                                    0.0, max(D - 1.0, 0.0), 0.1))
    base = texture(rng, H, W) if min(H, W) > 5 else rng.uniform(0, 255, size=(H, W))
    fill = texture(rng, H, W) if min(H, W) > 5 else rng.uniform(0, 255, size=(H, W))
    left, right, truth = render(rng, layers, H, W, base, fill, 2.0)
    lid = np.zeros((H, W), np.float32)
    m = rng.random((H, W)) < density
    v = truth + rng.normal(0.0, 0.3, size=(H, W))
    bad = rng.random((H, W)) < 0.05
    v[bad] = rng.uniform(-2.0, D + 2.0, size=int(bad.sum()))
    lid[m] = v[m]
    # a few non-finite and negative entries exercise the ingest rules
    if H * W >= 4:
        idx = rng.choice(H * W, size=min(4, H * W), replace=False)
        lid.ravel()[idx] = np.array([np.nan, np.inf, -3.0, 0.0], np.float32)[:len(idx)]
    return Scene(f"random_{W}x{H}_d{D}", seed, D, left, right, lid.astype(np.float32), truth)


def by_name(name: str, seed: int | None = None) -> Scene:
    """Named workloads: tiny, kitti[64|32|16|8], indoor, lowlight."""
    if name == "tiny":
        return tiny(1000 if seed is None else seed)
    if name.startswith("kitti"):
        beams = int(name[5:] or 64)
        return kitti(2000 if seed is None else seed, beams)
    if name == "indoor":
        return indoor(3200 if seed is None else seed)
    if name == "lowlight":
        return lowlight(3300 if seed is None else seed)
    raise KeyError(name)
