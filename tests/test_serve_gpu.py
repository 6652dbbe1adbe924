"""The request loop (sgmf_server_*): continuous batching must not change
results, admission must respect the device-memory budget, and simulated
cameras must all be served with their latencies recorded."""
import numpy as np
import pytest

import oracle
from paper_2504_05148_gb300 import scenes, serving
from paper_2504_05148_gb300 import sgmf as S

pytestmark = pytest.mark.gpu

SHAPES = [(96, 40, 16), (96, 40, 16), (71, 29, 100), (71, 29, 100), (130, 40, 200), (256, 128, 64)]


def _cameras(rate=20.0, per_cam=3):
    cams = []
    for ci, (W, H, D) in enumerate(SHAPES):
        frames = [scenes.random_small(8000 + 10 * ci + k, W, H, D) if (W, H) != (256, 128) else scenes.tiny(8000 + k)
                  for k in range(per_cam)]
        cams.append(serving.Camera(W, H, D, rate, frames))
    return cams


def test_each_result_is_the_same_alone_and_in_the_mix(gpu):
    cams = _cameras()
    sched = [(0.0, ci, k) for k in range(3) for ci in range(len(cams))]      # everything at once
    alone = serving.run(cams, schedule=sched, keep_outputs=True, serial=True, max_batch=4)
    mix = serving.run(cams, schedule=sched, keep_outputs=True, max_batch=4)
    assert all(st == S.SGMF_OK for st in alone.statuses + mix.statuses)
    assert alone.stats["largest_batch"] == 1
    assert mix.stats["largest_batch"] > 1                 # requests were batched together
    assert mix.stats["max_concurrent_batches"] >= 2       # and ran side by side
    assert set(alone.outputs) == set(mix.outputs) == {(ci, k) for ci in range(len(cams)) for k in range(3)}
    for key in alone.outputs:
        np.testing.assert_array_equal(mix.outputs[key], alone.outputs[key], err_msg=str(key))
        ci, k = key
        f = cams[ci].frames[k]
        want = oracle.compute(f.left, f.right, f.lidar, f.D, dumps=False).out
        np.testing.assert_array_equal(mix.outputs[key], want, err_msg=f"oracle {key}")


def test_admission_by_device_memory(gpu):
    probe = S.sgmf_server_create(None, 1 << 40, 4, 2)
    try:
        S.sgmf_server_add_camera(probe, 96, 40, 16)
        slot = S.sgmf_server_stats(probe)["device_bytes"]
    finally:
        S.sgmf_server_destroy(probe)
    budget = int(slot * 1.5)
    srv = S.sgmf_server_create(None, budget, 4, 2)
    try:
        c0 = S.sgmf_server_add_camera(srv, 96, 40, 16)
        c1 = S.sgmf_server_add_camera(srv, 96, 40, 16)          # same shape: shares the slot
        with pytest.raises(S.SgmfError) as e:
            S.sgmf_server_add_camera(srv, 640, 480, 64)         # a second shape does not fit
        assert e.value.status == S.SGMF_ERR_OOM
        frames = [scenes.random_small(8100 + k, 96, 40, 16) for k in range(6)]
        outs = [np.empty((40, 96), np.int16) for _ in frames]
        for k, f in enumerate(frames):
            S.sgmf_server_submit(srv, (c0, c1)[k % 2], f.left.ctypes.data, f.right.ctypes.data,
                                 f.lidar.ctypes.data, outs[k].ctypes.data, k)
        seen = set()
        while len(seen) < len(frames):
            r = S.sgmf_server_poll(srv, 1000)
            assert r is not None
            assert r[2] == S.SGMF_OK
            seen.add(r[0])
        st = S.sgmf_server_stats(srv)
        assert st["slots"] == 1 and st["peak_device_bytes"] <= budget
        for k, f in enumerate(frames):
            np.testing.assert_array_equal(outs[k], oracle.compute(f.left, f.right, f.lidar, f.D, dumps=False).out)
    finally:
        S.sgmf_server_destroy(srv)


def test_simulated_cameras_are_all_served(gpu):
    cams = _cameras(per_cam=2)
    for ci, c in enumerate(cams):
        c.rate_hz = 10.0 + 4 * ci                           # 10 .. 30 Hz
    r = serving.run(cams, duration_s=1.5, seed=5)
    s = r.summary()
    assert r.submitted == s["frames"] > 0
    assert all(st == S.SGMF_OK for st in r.statuses)
    assert 0.0 < s["p50_ms"] <= s["p99_ms"] < 1000.0
