"""Simulated cameras feeding the request loop of the C ABI (sgmf_server_*).

Each camera delivers frames of one shape at a mean rate with Poisson jitter
(exponential inter-arrival times).  One submitter thread replays the merged
arrival schedule in real time; one poller thread collects finished requests.
The request loop itself (admission by device memory, continuous batching,
per-shape resident slots) is native code in the library; this module only
generates load and gathers latencies.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import sgmf


@dataclass
class Camera:
    W: int
    H: int
    D: int
    rate_hz: float
    frames: list            # scenes (left, right, lidar) cycled through


@dataclass
class RunResult:
    latencies_ms: dict = field(default_factory=dict)    # camera -> list
    outputs: dict = field(default_factory=dict)         # (camera, k) -> int16 array (if kept)
    statuses: list = field(default_factory=list)
    wall_s: float = 0.0
    submitted: int = 0
    stats: dict = field(default_factory=dict)

    def all_latencies(self) -> np.ndarray:
        return np.array([v for vs in self.latencies_ms.values() for v in vs], np.float64)

    def summary(self) -> dict:
        lat = self.all_latencies()
        return {"frames": int(lat.size), "frames_per_s": lat.size / self.wall_s if self.wall_s else 0.0,
                "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
                "max_ms": float(lat.max()) if lat.size else None}


def poisson_schedule(rate_hz: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times in [0, duration_s) with exponential gaps of mean 1 / rate_hz."""
    rng = np.random.default_rng(seed)
    n = int(rate_hz * duration_s * 2 + 20)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
    while t[-1] < duration_s:
        t = np.concatenate([t, t[-1] + np.cumsum(rng.exponential(1.0 / rate_hz, size=n))])
    return t[t < duration_s]


def _pinned(a: np.ndarray) -> np.ndarray:
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


def run(cameras: list[Camera], duration_s: float | None = None, schedule: list | None = None,
        params: sgmf.Params | None = None, budget_bytes: int = 8 << 30, max_batch: int = 8,
        max_slots_per_shape: int = 2, seed: int = 0, keep_outputs: bool = False,
        use_lidar: bool = True, serial: bool = False) -> RunResult:
    """Replay camera arrivals against a fresh server.  `schedule` (a list of
    (time_s, camera, frame_index)) overrides the Poisson arrivals; `serial`
    submits each request only after the previous one came back (every frame
    alone on the GPU)."""
    srv = sgmf.sgmf_server_create(params, budget_bytes, max_batch, max_slots_per_shape)
    res = RunResult()
    try:
        ids = [sgmf.sgmf_server_add_camera(srv, c.W, c.H, c.D) for c in cameras]
        inputs = [[(_pinned(f.left), _pinned(f.right), _pinned(f.lidar)) for f in c.frames] for c in cameras]
        if schedule is None:
            ev = []
            for ci, c in enumerate(cameras):
                for k, t in enumerate(poisson_schedule(c.rate_hz, duration_s, seed * 1000 + ci)):
                    ev.append((float(t), ci, k))
            schedule = sorted(ev)
        outs = {}
        pending = {}
        free = [[] for _ in cameras]          # pinned output buffers ready for reuse, per camera
        lock = threading.Lock()
        total = len(schedule)
        res.latencies_ms = {ci: [] for ci in range(len(cameras))}
        done = threading.Event()
        returned = threading.Semaphore(0)

        def poller():
            got = 0
            while got < total:
                r = sgmf.sgmf_server_poll(srv, 100)
                if r is None:
                    continue
                tag, cam, st, lat = r
                got += 1
                with lock:
                    key = pending.pop(tag)
                    res.statuses.append(st)
                    res.latencies_ms[cam].append(lat)
                    if keep_outputs:
                        res.outputs[key] = outs[tag].copy()
                    free[key[0]].append(outs.pop(tag))
                returned.release()
            done.set()

        th = threading.Thread(target=poller, daemon=True)
        th.start()
        t0 = time.perf_counter()
        for tag, (t, ci, k) in enumerate(schedule):
            delay = t - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            c = cameras[ci]
            l, r, li = inputs[ci][k % len(inputs[ci])]
            with lock:
                o = free[ci].pop() if free[ci] else None
            if o is None:
                o = _pinned(np.empty((c.H, c.W), np.int16))
            with lock:
                outs[tag] = o
                pending[tag] = (ci, k)
            sgmf.sgmf_server_submit(srv, ids[ci], l.ctypes.data, r.ctypes.data,
                                    li.ctypes.data if use_lidar else None, o.ctypes.data, tag)
            res.submitted += 1
            if serial:
                returned.acquire()
        done.wait()
        res.wall_s = time.perf_counter() - t0
        res.stats = sgmf.sgmf_server_stats(srv)
    finally:
        sgmf.sgmf_server_destroy(srv)
    return res


def run_closed(cameras: list[Camera], duration_s: float, depth: int = 4, params: sgmf.Params | None = None,
               budget_bytes: int = 8 << 30, max_batch: int = 8, max_slots_per_shape: int = 2) -> RunResult:
    """Saturation: every camera keeps `depth` requests outstanding (a new one
    is submitted as soon as one comes back) for `duration_s`."""
    srv = sgmf.sgmf_server_create(params, budget_bytes, max_batch, max_slots_per_shape)
    res = RunResult()
    try:
        ids = [sgmf.sgmf_server_add_camera(srv, c.W, c.H, c.D) for c in cameras]
        inputs = [[(_pinned(f.left), _pinned(f.right), _pinned(f.lidar)) for f in c.frames] for c in cameras]
        bufs = {}
        res.latencies_ms = {ci: [] for ci in range(len(cameras))}
        next_tag = [0]
        count = [0] * len(cameras)

        def submit(ci, o):
            c = cameras[ci]
            l, r, li = inputs[ci][count[ci] % len(inputs[ci])]
            count[ci] += 1
            tag = next_tag[0]
            next_tag[0] += 1
            bufs[tag] = (ci, o)
            sgmf.sgmf_server_submit(srv, ids[ci], l.ctypes.data, r.ctypes.data, li.ctypes.data, o.ctypes.data, tag)
            res.submitted += 1

        t0 = time.perf_counter()
        for ci, c in enumerate(cameras):
            for _ in range(depth):
                submit(ci, _pinned(np.empty((c.H, c.W), np.int16)))
        outstanding = depth * len(cameras)
        while outstanding:
            r = sgmf.sgmf_server_poll(srv, 100)
            if r is None:
                continue
            tag, cam, st, lat = r
            outstanding -= 1
            res.statuses.append(st)
            res.latencies_ms[cam].append(lat)
            ci, o = bufs.pop(tag)
            if time.perf_counter() - t0 < duration_s:
                submit(ci, o)
                outstanding += 1
        res.wall_s = time.perf_counter() - t0
        res.stats = sgmf.sgmf_server_stats(srv)
    finally:
        sgmf.sgmf_server_destroy(srv)
    return res
