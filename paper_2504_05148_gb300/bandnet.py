"""Band proposal for the banded mode: training and inference driver.

Not part of the paper.  A six-layer 3x3 CNN (32 channels, quarter resolution)
reads the left image and the semidensified LiDAR map d-hat and proposes per
pixel a disparity band (centre, half-width in [8, 48], confidence).  Every
computation runs in libsgmf kernels (tensor-core convolutions, loss, Adam,
band tiles); this module only allocates device memory and sequences the
calls.

Inference (LearnedSGM): the banded context's front half (ingest, census,
semidensification) gives d-hat; the network turns it into one band start
per 8 x 8 tile for each band width; per frame a kernel picks the narrowest
width with at most `fallback_frac` uncertain tiles (low confidence or a
union of pixel bands wider than the band), else the plain full-range
method; each context then runs only its frames (per-frame gates on the
device, no host round trip).
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
        # the bf16 copy of the master weights (a library kernel), then the operand images
        S.sgmf_bn_to_bf16(LAYERS * PSZ, self.master.data_ptr(), self.wbf.data_ptr())
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
        """The fp32 master weights and the optimiser state (Adam moments and
        step count), so that training can resume exactly where it stopped."""
        np.savez(path, master=self.master.cpu().numpy(), adam_m=self.m.cpu().numpy(), adam_v=self.v.cpu().numpy(),
                 adam_t=np.int64(self.t))

    def load(self, path):
        """Weights, and the optimiser state when the file holds it (older
        files hold the weights only: the moments start at zero)."""
        import torch
        z = np.load(path)
        self.master.copy_(torch.from_numpy(z["master"]))
        if "adam_m" in z.files:
            self.m.copy_(torch.from_numpy(z["adam_m"]))
            self.v.copy_(torch.from_numpy(z["adam_v"]))
            self.t = int(z["adam_t"])
        else:
            self.m.zero_()
            self.v.zero_()
            self.t = 0
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


def batch_indices(seed: int, step: int, n: int, batch: int) -> np.ndarray:
    """The training pairs of one step: a function of (seed, step) alone, so a
    run resumed at any step draws the batches an uninterrupted one would."""
    return np.random.default_rng([seed, step]).choice(n, size=batch, replace=False)


def train(net: BandNet, x_all, lohi_all, counts, steps: int, batch: int = 16, lr: float = 2e-3, seed: int = 0,
          log_every: int = 100, D: int = 128, start: int = 0, stop: int | None = None):
    """Adam on the band loss over steps [start, stop) of a run of `steps`
    steps (the learning-rate schedule follows `steps`); returns the loss
    history.  With the optimiser state saved by BandNet.save, a run stopped
    at step k and resumed with start = k gives the uninterrupted run's weights."""
    import torch
    dev = torch.device("cuda")
    N, H4, W4, _ = x_all.shape
    stop = steps if stop is None else stop
    acts = [None] + [torch.empty((batch, H4, W4, C), dtype=torch.int16, device=dev) for _ in range(LAYERS - 1)]
    out = torch.empty((batch, H4, W4, C), dtype=torch.float32, device=dev)
    grad = torch.empty((batch, H4, W4, C), dtype=torch.int16, device=dev)
    gbuf = [torch.empty((batch, H4, W4, C), dtype=torch.int16, device=dev) for _ in range(2)]
    xb = torch.empty((batch, H4, W4, C), dtype=torch.int16, device=dev)
    lb = torch.empty((batch, H4, W4, 2), dtype=torch.int16, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    ti = torch.empty(batch, dtype=torch.int32, device=dev)
    xrow, lrow = H4 * W4 * C * 2, H4 * W4 * 2 * 2
    hist = []
    for st in range(start, stop):
        idx = batch_indices(seed, st, N, batch)
        ti.copy_(torch.from_numpy(idx.astype(np.int32)))
        S.sgmf_bn_gather(batch, ti.data_ptr(), N, xrow, x_all.data_ptr(), xb.data_ptr())
        S.sgmf_bn_gather(batch, ti.data_ptr(), N, lrow, lohi_all.data_ptr(), lb.data_ptr())
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
    """The banded method driven by the network.  Every frame takes the
    narrowest band width whose proposal it trusts (at most `fallback_frac`
    of its tiles uncertain) and falls back to the plain full-range method
    when none qualifies.  The choice is made per frame by a kernel; every
    context then runs only its own frames (sgmf_set_gate), so a call never
    waits for the proposal on the host."""

    def __init__(self, W: int, H: int, D: int, net: BandNet, band: int = 64, params=None, max_batch: int = 1,
                 conf_min: float = 0.5, fallback_frac: float = 0.02, sweep: bool | None = None,
                 bands: tuple | None = None):
        import torch
        self.W, self.H, self.D = W, H, D
        self.bands = tuple(sorted(bands if bands is not None else (band,)))
        self.band = self.bands[0]
        self.net = net
        self.conf_min, self.fallback_frac = conf_min, fallback_frac
        # one banded context per width (gate value = its index), the plain one last
        self.ctxs = [S.Context(W, H, D, params, band=b, max_batch=max_batch) for b in self.bands]
        self.banded = self.ctxs[0]          # runs the front half that feeds the network
        # the cluster sweep for the banded walks where it fits; it needs several
        # frames per call to fill the GPU (one cluster per frame and direction)
        if sweep if sweep is not None else max_batch >= 4:
            for c in self.ctxs:
                try:
                    S.sgmf_set_tuning(c.handle, 4, 128, 1)
                except S.SgmfError:
                    pass
        self.plain = S.Context(W, H, D, params, max_batch=max_batch)
        self.PLAIN = len(self.bands)
        dev = torch.device("cuda")
        self.H4, self.W4 = _q(4, H), _q(4, W)
        self.th, self.tw = _q(S.BAND_TILE, H), _q(S.BAND_TILE, W)
        n = max_batch
        self.x = torch.empty((n, self.H4, self.W4, C), dtype=torch.int16, device=dev)
        self.acts = [None] + [torch.empty((n, self.H4, self.W4, C), dtype=torch.int16, device=dev)
                              for _ in range(LAYERS - 1)]
        self.out = torch.empty((n, self.H4, self.W4, C), dtype=torch.float32, device=dev)
        self.lo = [torch.empty((n, self.th, self.tw), dtype=torch.int16, device=dev) for _ in self.bands]
        self.unc = torch.zeros((len(self.bands), n), dtype=torch.int32, device=dev)
        self.gate = torch.zeros(n, dtype=torch.int32, device=dev)
        self.marks = None          # set to a list to receive (name, cuda event) pairs per compute
        self.last_n = 0

    def compute(self, left, right, lidar, out):
        """left/right uint8, lidar float32, out int16: (n, H, W) CUDA tensors.
        Enqueues everything; the per-frame choice stays on the device."""
        import torch
        n = left.shape[0] if left.dim() == 3 else 1
        tiles = self.th * self.tw

        def mark(name):
            if self.marks is not None:
                e = torch.cuda.Event(enable_timing=True)
                e.record()
                self.marks.append((name, e))

        mark("start")
        for c in self.ctxs:                 # the front half runs on every frame
            S.sgmf_set_gate(c.handle, None, 0)
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
        for i, b in enumerate(self.bands):
            S.sgmf_bn_tiles(n, self.W, self.H, self.D, b, self.conf_min, self.out.data_ptr(), self.lo[i].data_ptr(),
                            self.unc[i].data_ptr())
        # widest band first (else the plain method), then narrower ones replace it where acceptable
        for i in range(len(self.bands) - 1, -1, -1):
            S.sgmf_bn_decide(n, tiles, self.fallback_frac, self.unc[i].data_ptr(), i,
                             self.PLAIN if i == len(self.bands) - 1 else -1, self.gate.data_ptr())
        mark("network")
        for i, c in enumerate(self.ctxs):
            if i > 0:                       # the other widths run their own front half on their frames
                S.sgmf_set_gate(c.handle, self.gate.data_ptr(), i)
                S.sgmf_compute_front(c.handle, n, left.data_ptr(), right.data_ptr(),
                                     lidar.data_ptr() if lidar is not None else None)
            S.sgmf_set_gate(c.handle, self.gate.data_ptr(), i)
            S.sgmf_compute_banded_back(c.handle, n, self.lo[i].data_ptr(), out.data_ptr())
        if self.fallback_frac < 1.0:         # else no frame can fall back: nothing to launch
            S.sgmf_set_gate(self.plain.handle, self.gate.data_ptr(), self.PLAIN)
            self.plain.compute(left, right, lidar, out)
        mark("back")
        self.last_n = n

    def decision(self):
        """(width index or PLAIN per frame, uncertain tiles per width and frame)
        of the last call; waits for it."""
        n = self.last_n
        return self.gate[:n].cpu().numpy().copy(), self.unc[:, :n].cpu().numpy().copy()

    def sync(self):
        for c in self.ctxs:
            c.sync()
        self.plain.sync()
        self.net.check()

    def close(self):
        for c in self.ctxs:
            c.close()
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
    ap.add_argument("--pairs", type=int, default=20000)
    ap.add_argument("--heldout", type=int, default=256, help="pairs of unseen seeds for the held-out loss")
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0, help="batch-order seed")
    ap.add_argument("--checkpoint-every", type=int, default=1000)
    ap.add_argument("--resume", action="store_true", help="continue the run saved in --out (weights + Adam state)")
    ap.add_argument("--workers", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                                                  "bandnet_street.npz"))
    args = ap.parse_args(argv)
    import json
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.workers) as pool:
        from . import build as _build
        _build.build()
        t0 = time.time()
        x_all, lohi_all, counts = build_training_set(args.pairs, pool=pool)
        gen_s = time.time() - t0
        print(f"training set: {args.pairs} pairs in {gen_s:.0f} s", flush=True)
        x_h, lohi_h, counts_h = build_training_set(args.heldout, seed0=200000, pool=pool)
    net = BandNet(seed=1)
    start = 0
    if args.resume and os.path.exists(args.out):
        net.load(args.out)
        start = net.t
        print(f"resuming at step {start}", flush=True)
    held0 = evaluate(net, x_h, lohi_h, counts_h)
    t0 = time.time()
    hist = []
    for a in range(start, args.steps, args.checkpoint_every):
        b = min(args.steps, a + args.checkpoint_every)
        hist += train(net, x_all, lohi_all, counts, args.steps, args.batch, args.lr, seed=args.seed, start=a, stop=b)
        os.makedirs(os.path.dirname(args.out), exist_ok=True)
        net.save(args.out)
        print(f"checkpoint at step {b}: held-out loss {evaluate(net, x_h, lohi_h, counts_h):.4f}", flush=True)
    train_s = time.time() - t0
    held = evaluate(net, x_h, lohi_h, counts_h)
    log = {"pairs": args.pairs, "heldout_pairs": args.heldout, "steps": args.steps, "batch": args.batch, "lr": args.lr,
           "seed": args.seed, "generation_s": round(gen_s, 1), "train_s": round(train_s, 1),
           "heldout_loss_start": held0, "heldout_loss_end": held,
           "loss_every_10_steps": [[int(st), round(v, 5)] for st, v in hist]}
    with open(os.path.splitext(args.out)[0] + "_train.json", "w") as fh:
        json.dump(log, fh)
    print(f"trained {args.steps - start} steps in {train_s:.1f} s; held-out loss {held0:.4f} -> {held:.4f}", flush=True)
    print("saved", args.out, flush=True)


if __name__ == "__main__":
    main()
