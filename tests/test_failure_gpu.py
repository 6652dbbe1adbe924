"""Failure handling, made to happen without faulting the GPU.

* A bounded device wait that runs out: the census kernel's wait for its TMA
  tiles gets a limit of zero polls, every CTA takes the timeout path (waits
  again with the default limit for its own copy, then returns), sgmf_sync
  reports SGMF_ERR_TIMEOUT, and the same context then computes the oracle's
  result again.
* An allocation that fails on the host side (sgmf_debug_fail_alloc): every
  allocation of sgmf_create in turn; each failure returns SGMF_ERR_OOM and
  leaves the device's free memory as it was.
* A camera producer of the request loop that stalls, and one that dies:
  the other camera is served at its own pace meanwhile, every submitted
  request comes back with the oracle's result, and the server shuts down.
"""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_2504_05148_gb300 import scenes
from paper_2504_05148_gb300 import sgmf as S

pytestmark = pytest.mark.gpu


def _run(ctx, s, dev):
    import torch
    out = torch.empty(s.shape, dtype=torch.int16, device=dev)
    ctx.compute(torch.from_numpy(s.left).to(dev), torch.from_numpy(s.right).to(dev),
                torch.from_numpy(s.lidar).to(dev), out)
    return out


def test_census_wait_that_runs_out_reports_timeout_and_recovers(gpu):
    s = scenes.tiny(1900)
    want = oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out
    ctx = S.Context(s.W, s.H, s.D)
    try:
        for _ in range(2):
            S.sgmf_set_wait_limit(ctx.handle, S.SGMF_WAIT_CENSUS, 0)
            _run(ctx, s, gpu)
            with pytest.raises(S.SgmfError) as e:
                ctx.sync()
            assert e.value.status == S.SGMF_ERR_TIMEOUT
            # the flag was cleared by that sync; the default limit computes the result again
            S.sgmf_set_wait_limit(ctx.handle, S.SGMF_WAIT_CENSUS, -1)
            out = _run(ctx, s, gpu)
            ctx.sync()
            np.testing.assert_array_equal(out.cpu().numpy(), want)
    finally:
        ctx.close()


def test_wait_limit_rejects_unknown_wait(gpu):
    ctx = S.Context(64, 32, 64)
    try:
        with pytest.raises(S.SgmfError) as e:
            S.sgmf_set_wait_limit(ctx.handle, 7, 10)
        assert e.value.status == S.SGMF_ERR_ARG
    finally:
        ctx.close()


def _free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("banded", [False, True])
def test_failed_allocation_in_create_leaks_nothing(gpu, banded):
    W, H, D, nb = 640, 480, 128, 2
    create = (lambda: S.sgmf_create_banded(W, H, D, 64, nb)) if banded else (lambda: S.sgmf_create_batched(W, H, D, nb))
    S.sgmf_destroy(create())                  # module loading and first-use state outside the comparison
    n = 1
    while True:
        before = _free_bytes()
        S.sgmf_debug_fail_alloc(n)
        try:
            h = create()
        except S.SgmfError as e:
            assert e.status == S.SGMF_ERR_OOM, str(e)
            assert "out of memory" in str(e)
            assert _free_bytes() == before, f"allocation {n}: device memory not returned"
            n += 1
            continue
        finally:
            S.sgmf_debug_fail_alloc(0)
        S.sgmf_destroy(h)                     # past the last allocation: the hook never fired
        break
    assert n > 10                             # every one of create's allocations failed once


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_failed_staging_allocation_keeps_the_context_usable(gpu, n):
    s = scenes.tiny(1901)
    want = oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out
    ctx = S.Context(s.W, s.H, s.D)
    try:
        out = np.empty(s.shape, np.int16)
        before = _free_bytes()
        S.sgmf_debug_fail_alloc(n)            # the n-th of the host entry point's four staging buffers
        try:
            with pytest.raises(S.SgmfError) as e:
                ctx.compute_host(s.left, s.right, s.lidar, out)
            assert e.value.status == S.SGMF_ERR_OOM
        finally:
            S.sgmf_debug_fail_alloc(0)
        assert _free_bytes() == before        # the staging buffers it did get were returned
        ctx.compute_host(s.left, s.right, s.lidar, out)
        np.testing.assert_array_equal(out, want)
    finally:
        ctx.close()


def _pinned(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


class _Loop:
    """Two cameras of the tiny shape, a producer thread per camera and one
    poller; producer `victim` stalls for `stall_s` after its third frame, or
    dies there (raises) when `die` is set."""

    def __init__(self, victim_frames, other_frames, rate_hz, stall_s=0.0, die=False):
        self.frames = [[scenes.tiny(7000 + k) for k in range(2)], [scenes.tiny(7100 + k) for k in range(2)]]
        self.inputs = [[(_pinned(f.left), _pinned(f.right), _pinned(f.lidar)) for f in fs] for fs in self.frames]
        self.counts = [victim_frames, other_frames]
        self.rate = rate_hz
        self.stall_s, self.die = stall_s, die
        self.lock = threading.Lock()
        self.sent = {}          # tag -> (camera, frame index, submit time, output buffer)
        self.got = {}           # tag -> (status, completion time)
        self.stall_window = None
        self.errors = []

    def run(self):
        srv = S.sgmf_server_create(None, 8 << 30, 4, 2)
        try:
            cams = [S.sgmf_server_add_camera(srv, 256, 128, 64) for _ in range(2)]
            next_tag = [0]

            def producer(ci):
                try:
                    for k in range(self.counts[ci]):
                        if ci == 0 and k == 3:
                            if self.die:
                                raise RuntimeError("camera 0 producer dies")
                            t0 = time.perf_counter()
                            time.sleep(self.stall_s)
                            self.stall_window = (t0, time.perf_counter())
                        l, r, li = self.inputs[ci][k % 2]
                        o = _pinned(np.full((128, 256), -7, np.int16))
                        with self.lock:
                            tag = next_tag[0]
                            next_tag[0] += 1
                            self.sent[tag] = (ci, k % 2, time.perf_counter(), o)
                        S.sgmf_server_submit(srv, cams[ci], l.ctypes.data, r.ctypes.data, li.ctypes.data,
                                             o.ctypes.data, tag)
                        time.sleep(1.0 / self.rate)
                except RuntimeError as e:
                    self.errors.append(str(e))

            ths = [threading.Thread(target=producer, args=(ci,)) for ci in range(2)]
            for th in ths:
                th.start()
            deadline = time.perf_counter() + 30.0
            while time.perf_counter() < deadline:
                r = S.sgmf_server_poll(srv, 50)
                if r is not None:
                    tag, cam, st, lat = r
                    with self.lock:
                        self.got[tag] = (st, time.perf_counter())
                alive = any(th.is_alive() for th in ths)
                with self.lock:
                    if not alive and len(self.got) == len(self.sent):
                        break
            for th in ths:
                th.join(timeout=5.0)
            stats = S.sgmf_server_stats(srv)
        finally:
            t0 = time.perf_counter()
            S.sgmf_server_destroy(srv)
            self.destroy_s = time.perf_counter() - t0
        return stats

    def check_results(self):
        assert set(self.got) == set(self.sent), "every submitted request comes back"
        want = [[oracle.compute(f.left, f.right, f.lidar, f.D, dumps=False).out for f in fs] for fs in self.frames]
        for tag, (ci, k, _, o) in self.sent.items():
            assert self.got[tag][0] == S.SGMF_OK
            np.testing.assert_array_equal(o, want[ci][k], err_msg=f"camera {ci} frame {k}")


def test_stalled_producer_does_not_hold_back_the_other_camera(gpu):
    loop = _Loop(victim_frames=8, other_frames=40, rate_hz=40.0, stall_s=1.0)
    stats = loop.run()
    loop.check_results()
    assert loop.stall_window is not None
    a, b = loop.stall_window
    during = [tag for tag, (ci, _, t, _) in loop.sent.items() if ci == 1 and a <= t and t + 0.2 <= b]
    assert len(during) >= 10, "the other camera kept submitting during the stall"
    for tag in during:
        assert loop.got[tag][1] < b, "a request of the other camera waited for the stalled one"
    assert stats["submitted"] == stats["completed"] == 48
    assert loop.destroy_s < 5.0


def test_dead_producer_leaves_the_server_serving(gpu):
    loop = _Loop(victim_frames=8, other_frames=20, rate_hz=40.0, die=True)
    stats = loop.run()
    assert loop.errors == ["camera 0 producer dies"]
    loop.check_results()
    assert sum(1 for ci, *_ in loop.sent.values() if ci == 0) == 3
    assert stats["submitted"] == stats["completed"] == 23
    assert loop.destroy_s < 5.0
