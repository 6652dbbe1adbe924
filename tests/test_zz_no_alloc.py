"""The allocation-free consistency entry point (sgmf_check_static).

Callers that cannot allocate device memory at the call site (a pool they do
not own, a real-time loop without cudaMalloc after start-up, a plugin host
that hands out only input and output buffers) use this entry point; its
working masks live in a static device array.  It must give exactly the
output of the ordinary pipeline's last stage: fed the pipeline's own d* and
d' and the same LiDAR map, the result equals sgmf_compute's output bit for
bit (the stage is integer arithmetic).  Two calls in a row, on different
frame sizes and modes, check that nothing carries over through the shared
array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2504_05148_gb300 import scenes
from paper_2504_05148_gb300 import sgmf as S

pytestmark = pytest.mark.gpu


def _pipeline(scene, params):
    """sgmf_compute's output and its d*, d' (ordinary entry point, with a context)."""
    import torch
    dev = torch.device("cuda:0")
    ctx = S.Context(scene.W, scene.H, scene.D, params)
    try:
        out = torch.empty(scene.shape, dtype=torch.int16, device=dev)
        ctx.compute(torch.from_numpy(scene.left).to(dev), torch.from_numpy(scene.right).to(dev),
                    torch.from_numpy(scene.lidar).to(dev), out)
        ctx.sync()
        return out.cpu().numpy(), ctx.stage(S.SGMF_STAGE_DSTAR), ctx.stage(S.SGMF_STAGE_DPRIME)
    finally:
        ctx.close()


def _pipeline_nolidar(scene, params):
    """As _pipeline with no LiDAR map (NULL)."""
    import torch
    dev = torch.device("cuda:0")
    ctx = S.Context(scene.W, scene.H, scene.D, params)
    try:
        out = torch.empty(scene.shape, dtype=torch.int16, device=dev)
        ctx.compute(torch.from_numpy(scene.left).to(dev), torch.from_numpy(scene.right).to(dev), None, out)
        ctx.sync()
        return out.cpu().numpy(), ctx.stage(S.SGMF_STAGE_DSTAR), ctx.stage(S.SGMF_STAGE_DPRIME)
    finally:
        ctx.close()


def _static(scene, params, dstar, dprime, lidar=True, free_check=False):
    import torch
    dev = torch.device("cuda:0")
    ds = torch.from_numpy(dstar).to(dev)
    dp = torch.from_numpy(dprime).to(dev)
    li = torch.from_numpy(scene.lidar).to(dev)
    out = torch.full(scene.shape, 12345, dtype=torch.int16, device=dev)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    S.sgmf_check_static(scene.W, scene.H, scene.D, params, ds.data_ptr(), dp.data_ptr(),
                        li.data_ptr() if lidar else None, out.data_ptr(), None)
    torch.cuda.synchronize()
    if free_check:
        # nothing was allocated on the device by the call
        assert torch.cuda.mem_get_info()[0] == free0
    return out.cpu().numpy()


def test_static_check_equals_pipeline_on_consecutive_calls(gpu):
    cases = [
        (scenes.kitti(2300), S.Params(), True),                                   # 1242 x 375, D = 128
        (scenes.tiny(1200), S.Params(consistency=S.SGMF_CHECK_LIDAR), True),      # 256 x 128, D = 64
        (scenes.kitti(2301), S.Params(tc=4, rc=9), True),
        (scenes.street(2310, 640, 480, 192), S.Params(), True),                   # 6 mask words a pixel
        (scenes.street(2311, 640, 480, 256), S.Params(rc=7), True),               # 8 mask words a pixel
        (scenes.kitti(2302), S.Params(consistency=S.SGMF_CHECK_STEREO), True),    # no box-OR
        (scenes.tiny(1202), S.Params(consistency=S.SGMF_CHECK_NONE), True),
        (scenes.kitti(2303), S.Params(), False),                                  # no LiDAR map
    ]
    for i, (scene, params, lidar) in enumerate(cases):
        want, dstar, dprime = _pipeline(scene, params) if lidar else _pipeline_nolidar(scene, params)
        got = _static(scene, params, dstar, dprime, lidar, free_check=i > 0)
        np.testing.assert_array_equal(got, want, err_msg=f"case {i}: {scene.name}")


def test_static_check_rejects_frames_beyond_its_array(gpu):
    s = scenes.tiny(1201)
    with pytest.raises(S.SgmfError) as e:
        # 1920 x 1080 with D = 256 needs 3 * 8 * 2073600 words, more than the array holds
        S.sgmf_check_static(1920, 1080, 256, S.Params(), 1, 1, None, 1, None)
    assert e.value.status == S.SGMF_ERR_SHAPE
    with pytest.raises(S.SgmfError) as e:
        S.sgmf_check_static(s.W, s.H, s.D, S.Params(p1=9, p2=3), 1, 1, None, 1, None)
    assert e.value.status == S.SGMF_ERR_PARAM
