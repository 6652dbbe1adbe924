"""CPU reference of the band-proposal network (TEST INFRASTRUCTURE ONLY).

Not part of the paper: a small CNN that proposes, from the quarter-resolution
left image and the semidensified LiDAR map d-hat, a disparity band per pixel
for the banded mode.  This module is the plain float64 statement of what the
CUDA kernels compute, used by the tests to check them; the library never
imports it.

Network: quarter-resolution input x (H4 x W4 x 32, channels 0..2 used, the
rest zero), five 3x3 convolutions with 32 output channels, bias and ReLU,
then a sixth 3x3 convolution with 32 outputs of which 0..2 are read: centre
c = D * o0, half-width w = 8 + 40 * sigmoid(o1), confidence q = sigmoid(o2).
Convolutions use zero padding.  Storage precision follows the GPU path:
weights and stored activations are bfloat16 values; arithmetic here is
float64 (the GPU accumulates in float32).

Layouts: activations [n][h][w][32]; weights [co][ky][kx][ci] (ky, kx = 0..2
for offsets -1..1); bias [co].
"""
from __future__ import annotations

import numpy as np

C = 32            # channels of every layer
LAYERS = 6


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray | None) -> np.ndarray:
    """y[n, y, x, co] = b[co] + sum_{ky, kx, ci} w[co, ky, kx, ci] x[n, y+ky-1, x+kx-1, ci]."""
    n, h, wd, ci = x.shape
    xp = np.zeros((n, h + 2, wd + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((n, h, wd, w.shape[0]))
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("nhwc,oc->nhwo", xp[:, ky:ky + h, kx:kx + wd], w[:, ky, kx, :])
    if b is not None:
        y += b
    return y


def conv3x3_dgrad(dy: np.ndarray, w: np.ndarray) -> np.ndarray:
    """dx of conv3x3 for the output gradient dy (no bias term)."""
    n, h, wd, co = dy.shape
    dyp = np.zeros((n, h + 2, wd + 2, co))
    dyp[:, 1:-1, 1:-1] = dy
    dx = np.zeros((n, h, wd, w.shape[3]))
    # x[p + o] feeds y[p] through w[:, 1+oy, 1+ox]: dx[q] = sum_o dy[q - o] w[:, 1+oy, 1+ox]
    for ky in range(3):
        for kx in range(3):
            oy, ox = ky - 1, kx - 1
            dx += np.einsum("nhwo,oc->nhwc", dyp[:, 1 - oy:1 - oy + h, 1 - ox:1 - ox + wd], w[:, ky, kx, :])
    return dx


def conv3x3_wgrad(x: np.ndarray, dy: np.ndarray):
    """(dw, db) of conv3x3 for input x and output gradient dy."""
    n, h, wd, ci = x.shape
    xp = np.zeros((n, h + 2, wd + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    dw = np.zeros((dy.shape[3], 3, 3, ci))
    for ky in range(3):
        for kx in range(3):
            dw[:, ky, kx, :] = np.einsum("nhwo,nhwc->oc", dy, xp[:, ky:ky + h, kx:kx + wd])
    return dw, dy.sum(axis=(0, 1, 2))


def forward(x: np.ndarray, ws: list, bs: list, round_acts: bool = True):
    """Activations of every layer: acts[0] = x, acts[l] = bf16(relu(conv)) for
    l = 1..5 (no rounding with round_acts=False), and the float64 outputs of
    layer 6."""
    acts = [x]
    for l in range(LAYERS - 1):
        a = np.maximum(conv3x3(acts[-1], ws[l], bs[l]), 0.0)
        acts.append(bf16_round(a) if round_acts else a)
    out = conv3x3(acts[-1], ws[-1], bs[-1])
    return acts, out


def heads(out: np.ndarray, D: int):
    """centre, half-width, confidence from the last layer's channels 0..2."""
    sig = lambda v: 1.0 / (1.0 + np.exp(-v))
    return D * out[..., 0], 8.0 + 40.0 * sig(out[..., 1]), sig(out[..., 2])


def loss_and_grad(out: np.ndarray, lo_t: np.ndarray, hi_t: np.ndarray, valid: np.ndarray, D: int,
                  lam_c: float = 1.0, lam_w: float = 0.25):
    """Band loss and its gradient with respect to the last layer's outputs.

    For each labelled quarter pixel (valid), with the plain method's disparity
    range [lo_t, hi_t] over its 4 x 4 block:
      centre target (lo_t + hi_t) / 2, half-width target clamp((hi_t - lo_t) / 2 + 2, 8, 48),
      L = lam_c |c - c_t| / D + lam_w |w - w_t| / D + BCE(q, y),
      y = 1 if [c - w, c + w] covers [lo_t, hi_t] (taken as a constant).
    The loss is the mean over labelled pixels."""
    c, w, q = heads(out, D)
    ct = 0.5 * (lo_t + hi_t)
    wt = np.clip(0.5 * (hi_t - lo_t) + 2.0, 8.0, 48.0)
    y = ((c - w <= lo_t) & (hi_t <= c + w)).astype(np.float64)
    nv = max(int(valid.sum()), 1)
    eps = 1e-12
    L = (lam_c * np.abs(c - ct) / D + lam_w * np.abs(w - wt) / D
         - (y * np.log(q + eps) + (1 - y) * np.log(1 - q + eps)))
    loss = float((L * valid).sum() / nv)
    g = np.zeros_like(out)
    s1 = (w - 8.0) / 40.0
    g[..., 0] = lam_c * np.sign(c - ct) * valid / nv                     # dc/do0 = D
    g[..., 1] = lam_w * np.sign(w - wt) / D * 40.0 * s1 * (1 - s1) * valid / nv
    g[..., 2] = (q - y) * valid / nv
    return loss, g


def backward(acts: list, ws: list, gout: np.ndarray):
    """Gradients (dws, dbs) of every layer for the output gradient gout.
    Stored activations are treated as the layers' outputs (the bf16 rounding
    passes the gradient through unchanged)."""
    dws, dbs = [None] * LAYERS, [None] * LAYERS
    g = gout
    for l in range(LAYERS - 1, -1, -1):
        dws[l], dbs[l] = conv3x3_wgrad(acts[l], g)
        if l > 0:
            g = conv3x3_dgrad(g, ws[l]) * (acts[l] > 0)
    return dws, dbs
