"""Band proposal for the banded mode: training and inference driver.

Not part of the paper.  A six-layer 3x3 CNN (32 channels, quarter resolution)
reads the left image and the semidensified LiDAR map d-hat and proposes per
pixel a disparity band (centre, half-width in [8, 48], confidence).  Every
computation runs in libsgmf kernels (tensor-core convolutions, loss, Adam,
band tiles); this module only allocates device memory and sequences the
calls.

Inference (LearnedSGM): the banded context's front half (ingest, census,
semidensification) gives d-hat; the network turns it into one band start
per 8 x 8 tile; if more than `fallback_frac` of the tiles are uncertain
(low confidence or a union of pixel bands wider than the band), the frame
falls back to the plain full-range method, else the banded back half
finishes it.
"""
from __future__ import annotations

import argparse
import os
import time

import numpy as np

from . import sgmf as S

C = 32
LAYERS = 6
WSZ = C * 9 * C          # weights of one layer
PSZ = WSZ + C            # weights + bias


def _q(n, v):
    return (v + n - 1) // n


class BandNet:
    """Parameters on the device: fp32 master copy (Adam state beside it), the
    bf16 copy the kernels read, and the packed tensor-core operand images."""

    def __init__(self, seed: int = 0):
        import torch
        rng = np.random.default_rng(seed)
        flat = np.zeros(LAYERS * PSZ, np.float32)
        for l in range(LAYERS):
            cin = 3 if l == 0 else C
            std = np.sqrt(2.0 / (9 * cin)) if l < LAYERS - 1 else 0.01
            w = rng.normal(scale=std, size=(C, 3, 3, C)).astype(np.float32)
            if l == 0:
                w[:, :, :, 3:] = 0.0
            if l == LAYERS - 1:
                w[3:] = 0.0
            flat[l * PSZ:l * PSZ + WSZ] = w.ravel()
        # start the heads near a useful point: centre 0.3 D, half-width ~24, confidence 0.5
        flat[(LAYERS - 1) * PSZ + WSZ + 0] = 0.3
        self.dev = torch.device("cuda")
        self.master = torch.from_numpy(flat).to(self.dev)
        self.m = torch.zeros_like(self.master)
        self.v = torch.zeros_like(self.master)
        self.grad = torch.zeros_like(self.master)
        self.wbf = torch.zeros(LAYERS * PSZ, dtype=torch.int16, device=self.dev)
        self.packed_f = torch.zeros((LAYERS, WSZ), dtype=torch.int16, device=self.dev)
        self.packed_d = torch.zeros((LAYERS, WSZ), dtype=torch.int16, device=self.dev)
        self.err = torch.zeros(1, dtype=torch.int32, device=self.dev)
        self.t = 0
        self._sync_bf16()

    def _sync_bf16(self):
        # bf16 copy of the master weights through a zero-rate Adam step is not
        # exact (it would move the moments): pack from a bf16 rounding instead
        import torch
        f = self.master.detach().cpu().numpy().astype(np.float32)
        u = f.view(np.uint32).astype(np.uint64)
        r = (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)
        self.wbf.copy_(torch.from_numpy(r.view(np.int16)))
        self.repack()

    def w_ptr(self, l):
        return self.wbf.data_ptr() + 2 * l * PSZ

    def b_ptr(self, l):
        return self.master.data_ptr() + 4 * (l * PSZ + WSZ)

    def repack(self, stream=None):
        for l in range(LAYERS):
            S.sgmf_bn_pack(self.w_ptr(l), self.packed_f[l].data_ptr(), self.packed_d[l].data_ptr(), stream)

    def forward(self, x, n, h, w, acts=None, out=None, stream=None):
        """x: bf16 [n][h][w][32] (int16 tensor).  Returns (acts, out f32)."""
        import torch
        if acts is None:
            acts = [x] + [torch.empty((n, h, w, C), dtype=torch.int16, device=self.dev) for _ in range(LAYERS - 1)]
        else:
            acts[0] = x
        if out is None:
            out = torch.empty((n, h, w, C), dtype=torch.float32, device=self.dev)
        for l in range(LAYERS):
            last = l == LAYERS - 1
            S.sgmf_bn_conv(n, h, w, acts[l].data_ptr(), self.packed_f[l].data_ptr(), self.b_ptr(l), not last, None,
                           None if last else acts[l + 1].data_ptr(), out.data_ptr() if last else None,
                           self.err.data_ptr(), stream)
        return acts, out

    def backward(self, acts, gout, n, h, w, gbuf=None, stream=None):
        """Accumulates parameter gradients into self.grad (zeroed first)."""
        import torch
        self.grad.zero_()
        if gbuf is None:
            gbuf = [torch.empty((n, h, w, C), dtype=torch.int16, device=self.dev) for _ in range(2)]
        g = gout
        for l in range(LAYERS - 1, -1, -1):
            dw = self.grad.data_ptr() + 4 * l * PSZ
            S.sgmf_bn_wgrad(n, h, w, acts[l].data_ptr(), g.data_ptr(), dw, dw + 4 * WSZ, self.err.data_ptr(), stream)
            if l > 0:
                nxt = gbuf[l % 2]
                S.sgmf_bn_conv(n, h, w, g.data_ptr(), self.packed_d[l].data_ptr(), None, False, acts[l].data_ptr(),
                               nxt.data_ptr(), None, self.err.data_ptr(), stream)
                g = nxt
        # (input channels 3..31 are zero, so their weight gradients are zero too)

    def step(self, lr, b1=0.9, b2=0.999, eps=1e-8, stream=None):
        self.t += 1
        S.sgmf_bn_adam(LAYERS * PSZ, self.master.data_ptr(), self.m.data_ptr(), self.v.data_ptr(),
                       self.grad.data_ptr(), lr, b1, b2, eps, self.t, self.wbf.data_ptr(), stream)
        self.repack(stream)

    def check(self):
        import torch
        torch.cuda.synchronize()
        if int(self.err.item()) != 0:
            raise RuntimeError("a bounded wait in a network kernel gave up")

    def save(self, path):
        np.savez(path, master=self.master.cpu().numpy())

    def load(self, path):
        import torch
        self.master.copy_(torch.from_numpy(np.load(path)["master"]))
        self._sync_bf16()


# ---- training data ----------------------------------------------------------------------

def _gen(args):
    from . import scenes
    seed, W, H, D = args
    s = scenes.street(seed, W, H, D)
    return s.left, s.right, s.lidar


def build_training_set(n_pairs: int, seed0: int = 100000, W: int = 1242, H: int = 375, D: int = 128,
                       batch: int = 16, workers: int = 0, pool=None):
    """Quarter-resolution inputs and labels of n_pairs generated street pairs,
    labelled by the plain method's output (run on the GPU).  Returns device
    tensors x [N][H4][W4][32] bf16, lohi [N][H4][W4][2] and per-pair label
    counts (host)."""
    import torch
    dev = torch.device("cuda")
    H4, W4 = _q(4, H), _q(4, W)
    x_all = torch.empty((n_pairs, H4, W4, C), dtype=torch.int16, device=dev)
    lohi_all = torch.empty((n_pairs, H4, W4, 2), dtype=torch.int16, device=dev)
    counts = np.zeros(n_pairs, np.int64)
    ctx = S.Context(W, H, D, max_batch=batch)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    jobs = [(seed0 + i, W, H, D) for i in range(n_pairs)]
    it = pool.imap(_gen, jobs, chunksize=4) if pool is not None else map(_gen, jobs)
    try:
        done = 0
        while done < n_pairs:
            nb = min(batch, n_pairs - done)
            got = [next(it) for _ in range(nb)]
            l = torch.from_numpy(np.stack([g[0] for g in got])).to(dev)
            r = torch.from_numpy(np.stack([g[1] for g in got])).to(dev)
            li = torch.from_numpy(np.stack([g[2] for g in got])).to(dev)
            out = torch.empty((nb, H, W), dtype=torch.int16, device=dev)
            ctx.compute(l, r, li, out)
            S.sgmf_bn_input(nb, W, H, D, l.data_ptr(), S.sgmf_prior_device(ctx.handle),
                            x_all[done].data_ptr())
            for i in range(nb):
                cnt.zero_()
                S.sgmf_bn_labels(1, W, H, out[i].data_ptr(), lohi_all[done + i].data_ptr(), cnt.data_ptr())
                torch.cuda.synchronize()
                counts[done + i] = int(cnt.item())
            ctx.sync()
            done += nb
    finally:
        ctx.close()
    return x_all, lohi_all, counts


def train(net: BandNet, x_all, lohi_all, counts, steps: int, batch: int = 16, lr: float = 2e-3, seed: int = 0,
          log_every: int = 100, D: int = 128):
    """Adam on the band loss; returns the loss history (one value per step)."""
    import torch
    dev = torch.device("cuda")
    N, H4, W4, _ = x_all.shape
    rng = np.random.default_rng(seed)
    acts = [None] + [torch.empty((batch, H4, W4, C), dtype=torch.int16, device=dev) for _ in range(LAYERS - 1)]
    out = torch.empty((batch, H4, W4, C), dtype=torch.float32, device=dev)
    grad = torch.empty((batch, H4, W4, C), dtype=torch.int16, device=dev)
    gbuf = [torch.empty((batch, H4, W4, C), dtype=torch.int16, device=dev) for _ in range(2)]
    xb = torch.empty((batch, H4, W4, C), dtype=torch.int16, device=dev)
    lb = torch.empty((batch, H4, W4, 2), dtype=torch.int16, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    hist = []
    for st in range(steps):
        idx = rng.choice(N, size=batch, replace=False)
        ti = torch.from_numpy(idx).to(dev)
        torch.index_select(x_all, 0, ti, out=xb)
        torch.index_select(lohi_all, 0, ti, out=lb)
        cnt.fill_(int(counts[idx].sum()))
        loss.zero_()
        net.forward(xb, batch, H4, W4, acts, out)
        S.sgmf_bn_loss(batch * H4 * W4, D, out.data_ptr(), lb.data_ptr(), cnt.data_ptr(), grad.data_ptr(),
                       loss.data_ptr())
        net.backward(acts, grad, batch, H4, W4, gbuf)
        cur = lr if st < 0.7 * steps else lr * 0.2
        net.step(cur)
        if st % 10 == 0 or st == steps - 1:
            hist.append((st, float(loss.item())))
            if log_every and st % log_every == 0:
                print(f"step {st} loss {hist[-1][1]:.4f}", flush=True)
    net.check()
    return hist


def evaluate(net: BandNet, x_all, lohi_all, counts, batch: int = 16, D: int = 128) -> float:
    """Mean band loss over the whole set (labelled pixels weighted equally)."""
    import torch
    dev = torch.device("cuda")
    N, H4, W4, _ = x_all.shape
    out = torch.empty((batch, H4, W4, C), dtype=torch.float32, device=dev)
    grad = torch.empty((batch, H4, W4, C), dtype=torch.int16, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    total, labelled = 0.0, 0
    for i in range(0, N, batch):
        nb = min(batch, N - i)
        c = int(counts[i:i + nb].sum())
        cnt.fill_(c)
        loss.zero_()
        _, o = net.forward(x_all[i:i + nb], nb, H4, W4, out=out[:nb])
        S.sgmf_bn_loss(nb * H4 * W4, D, o.data_ptr(), lohi_all[i:i + nb].data_ptr(), cnt.data_ptr(),
                       grad.data_ptr(), loss.data_ptr())
        total += float(loss.item()) * c
        labelled += c
    net.check()
    return total / max(labelled, 1)


# ---- inference ------------------------------------------------------------------------

class LearnedSGM:
    """The banded method driven by the network, with the plain method as the
    per-frame fallback."""

    def __init__(self, W: int, H: int, D: int, net: BandNet, band: int = 64, params=None, max_batch: int = 1,
                 conf_min: float = 0.5, fallback_frac: float = 0.02, sweep: bool | None = None):
        import torch
        self.W, self.H, self.D, self.band = W, H, D, band
        self.net = net
        self.conf_min, self.fallback_frac = conf_min, fallback_frac
        self.banded = S.Context(W, H, D, params, band=band, max_batch=max_batch)
        # the cluster sweep for the banded walks where it fits; it needs several
        # frames per call to fill the GPU (one cluster per frame and direction)
        if sweep if sweep is not None else max_batch >= 4:
            try:
                S.sgmf_set_tuning(self.banded.handle, 4, 128, 1)
            except S.SgmfError:
                pass
        self.plain = S.Context(W, H, D, params, max_batch=max_batch)
        dev = torch.device("cuda")
        self.H4, self.W4 = _q(4, H), _q(4, W)
        self.th, self.tw = _q(S.BAND_TILE, H), _q(S.BAND_TILE, W)
        n = max_batch
        self.x = torch.empty((n, self.H4, self.W4, C), dtype=torch.int16, device=dev)
        self.acts = [None] + [torch.empty((n, self.H4, self.W4, C), dtype=torch.int16, device=dev)
                              for _ in range(LAYERS - 1)]
        self.out = torch.empty((n, self.H4, self.W4, C), dtype=torch.float32, device=dev)
        self.lo = torch.empty((n, self.th, self.tw), dtype=torch.int16, device=dev)
        self.unc = torch.zeros(1, dtype=torch.int32, device=dev)
        self.stats = {"frames": 0, "fallback_frames": 0, "uncertain_tiles": 0, "tiles": 0}
        self.marks = None          # set to a list to receive (name, cuda event) pairs per compute

    def compute(self, left, right, lidar, out):
        """left/right uint8, lidar float32, out int16: (n, H, W) CUDA tensors.
        Returns True when the batch fell back to the plain method."""
        import torch
        n = left.shape[0] if left.dim() == 3 else 1

        def mark(name):
            if self.marks is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record()
                self.marks.append((name, e))

        mark("start")
        S.sgmf_compute_front(self.banded.handle, n, left.data_ptr(), right.data_ptr(),
                             lidar.data_ptr() if lidar is not None else None)
        mark("front")
        S.sgmf_bn_input(n, self.W, self.H, self.D, left.data_ptr(), S.sgmf_prior_device(self.banded.handle),
                        self.x.data_ptr())
        self.acts[0] = self.x
        for l in range(LAYERS):
            last = l == LAYERS - 1
            S.sgmf_bn_conv(n, self.H4, self.W4, self.acts[l].data_ptr(), self.net.packed_f[l].data_ptr(),
                           self.net.b_ptr(l), not last, None, None if last else self.acts[l + 1].data_ptr(),
                           self.out.data_ptr() if last else None, self.net.err.data_ptr())
        self.unc.zero_()
        S.sgmf_bn_tiles(n, self.W, self.H, self.D, self.band, self.conf_min, self.out.data_ptr(), self.lo.data_ptr(),
                        self.unc.data_ptr())
        mark("network")
        unc = int(self.unc.item())     # waits for the proposal
        tiles = n * self.th * self.tw
        self.stats["frames"] += n
        self.stats["uncertain_tiles"] += unc
        self.stats["tiles"] += tiles
        if unc > self.fallback_frac * tiles:
            self.stats["fallback_frames"] += n
            self.plain.compute(left, right, lidar, out)
            return True
        S.sgmf_compute_banded_back(self.banded.handle, n, self.lo.data_ptr(), out.data_ptr())
        mark("back")
        return False

    def sync(self):
        self.banded.sync()
        self.plain.sync()
        self.net.check()

    def close(self):
        self.banded.close()
        self.plain.close()


def disagreement(learned: np.ndarray, plain: np.ndarray) -> float:
    """Fraction of the plain method's valid pixels where the learned-band
    output is invalid or differs by more than one disparity."""
    v = plain >= 0
    if not v.any():
        return 0.0
    bad = (learned < 0) | (np.abs(learned.astype(np.int64) - plain.astype(np.int64)) > 1)
    return float((bad & v).sum() / v.sum())


def main(argv=None):
    ap = argparse.ArgumentParser(description="train the band-proposal network on generated street pairs")
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=1500)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                                                  "bandnet_street.npz"))
    args = ap.parse_args(argv)
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.workers) as pool:
        from . import build as _build
        _build.build()
        t0 = time.time()
        x_all, lohi_all, counts = build_training_set(args.pairs, pool=pool)
        print(f"training set: {args.pairs} pairs in {time.time() - t0:.0f} s", flush=True)
    net = BandNet(seed=1)
    t0 = time.time()
    hist = train(net, x_all, lohi_all, counts, args.steps, args.batch, args.lr)
    print(f"trained {args.steps} steps in {time.time() - t0:.1f} s; loss {hist[0][1]:.4f} -> {hist[-1][1]:.4f}",
          flush=True)
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    net.save(args.out)
    print("saved", args.out, flush=True)


if __name__ == "__main__":
    main()
