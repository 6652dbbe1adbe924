"""The box-OR masks of Eq. 5 (radius r_s) and Eq. 6 (radius r_c): bit d of a
pixel's mask is set when some pixel of its clipped (2r+1)^2 window has
d-bar = d.  The expected masks are a SciPy maximum filter over the one-hot
planes of the oracle's d-bar, packed into 32-bit words: independent of the
kernels' sparse row pass and van Herk / Gil-Werman column pass."""
import numpy as np
import pytest

import oracle
from paper_2504_05148_gb300 import scenes
from paper_2504_05148_gb300 import sgmf as S

pytestmark = pytest.mark.gpu


def _want(dbar, D, r):
    from scipy.ndimage import maximum_filter
    H, W = dbar.shape
    MW = S.mask_words(D)
    hot = np.zeros((32 * MW, H, W), np.uint8)
    ys, xs = np.nonzero(dbar >= 0)
    hot[dbar[ys, xs], ys, xs] = 1
    box = maximum_filter(hot, size=(1, 2 * r + 1, 2 * r + 1), mode="constant", cval=0)
    bits = box.reshape(MW, 32, H, W).astype(np.uint64)
    return (bits << np.arange(32, dtype=np.uint64)[None, :, None, None]).sum(axis=1).astype(np.uint32)


def _masks(scene, params):
    import torch
    dev = torch.device("cuda:0")
    ctx = S.Context(scene.W, scene.H, scene.D, params)
    try:
        out = torch.empty(scene.shape, dtype=torch.int16, device=dev)
        ctx.compute(torch.from_numpy(scene.left).to(dev), torch.from_numpy(scene.right).to(dev),
                    torch.from_numpy(scene.lidar).to(dev), out)
        ctx.sync()
        return ctx.stage(S.SGMF_STAGE_BOX_S), ctx.stage(S.SGMF_STAGE_BOX_C)
    finally:
        ctx.close()


@pytest.mark.parametrize("W,H,D,rs,rc,density", [
    (1242, 75, 128, 6, 20, 0.05),      # the default radii on a KITTI-wide strip
    (97, 130, 256, 3, 40, 0.3),        # 8 word planes, windows taller than a column tile
    (33, 17, 64, 0, 1, 1.0),           # a LiDAR value at every pixel
    (300, 200, 192, 255, 100, 0.02),   # the largest radius
    (200, 90, 128, 16, 16, 0.1),       # equal radii
    (130, 70, 256, 16, 3, 0.2),        # r_s above r_c, 8 word planes
    (150, 33, 128, 17, 4, 0.1),        # column segments of 32 rows and a ragged last one
    (1, 70, 16, 2, 5, 0.5),            # one column
    (70, 1, 100, 5, 7, 0.5),           # one row
])
def test_box_masks_match_a_max_filter(gpu, W, H, D, rs, rc, density):
    s = scenes.random_small(W + 3 * H + D + rs, W, H, D, density=density)
    p = S.Params(rs=rs, rc=rc)
    box_s, box_c = _masks(s, p)
    dbar = oracle.lidar(s.lidar, D)
    np.testing.assert_array_equal(box_s, _want(dbar, D, rs), err_msg="r_s")
    np.testing.assert_array_equal(box_c, _want(dbar, D, rc), err_msg="r_c")


def test_only_the_wanted_radius(gpu):
    s = scenes.random_small(9700, 150, 60, 128)
    dbar = oracle.lidar(s.lidar, s.D)
    import torch
    dev = torch.device("cuda:0")
    for p, stage, r in [(S.Params(semidense=0), S.SGMF_STAGE_BOX_C, 20),
                        (S.Params(consistency=S.SGMF_CHECK_STEREO), S.SGMF_STAGE_BOX_S, 6)]:
        ctx = S.Context(s.W, s.H, s.D, p)
        try:
            out = torch.empty(s.shape, dtype=torch.int16, device=dev)
            ctx.compute(torch.from_numpy(s.left).to(dev), torch.from_numpy(s.right).to(dev),
                        torch.from_numpy(s.lidar).to(dev), out)
            ctx.sync()
            np.testing.assert_array_equal(ctx.stage(stage), _want(dbar, s.D, r))
            other = S.SGMF_STAGE_BOX_S if stage == S.SGMF_STAGE_BOX_C else S.SGMF_STAGE_BOX_C
            with pytest.raises(S.SgmfError):
                ctx.stage(other)
        finally:
            ctx.close()


@pytest.mark.parametrize("n", [1, 20, 32])
def test_box_masks_in_a_batch(gpu, n):
    """Batches of 256 x 300 frames at D = 128: the column pass streams row
    segments of 32, 64 or 128 rows, the longest whose grid still fills the
    device (on 152 SMs these batch sizes give the three lengths).  Frame 0's
    masks must equal the max filter; the outputs of the first, middle and
    last frame, which go through both masks, must equal the oracle's."""
    import torch
    W, H, D = 256, 300, 128
    scs = [scenes.random_small(9900 + i, W, H, D, density=0.08) for i in range(n)]
    dev = torch.device("cuda:0")
    ctx = S.Context(W, H, D, max_batch=n)
    try:
        out = torch.empty((n, H, W), dtype=torch.int16, device=dev)
        ctx.compute(torch.from_numpy(np.stack([s.left for s in scs])).to(dev),
                    torch.from_numpy(np.stack([s.right for s in scs])).to(dev),
                    torch.from_numpy(np.stack([s.lidar for s in scs])).to(dev), out)
        ctx.sync()
        box_s, box_c = ctx.stage(S.SGMF_STAGE_BOX_S), ctx.stage(S.SGMF_STAGE_BOX_C)
        got = out.cpu().numpy()
    finally:
        ctx.close()
    dbar = oracle.lidar(scs[0].lidar, D)
    np.testing.assert_array_equal(box_s, _want(dbar, D, 6), err_msg="r_s")
    np.testing.assert_array_equal(box_c, _want(dbar, D, 20), err_msg="r_c")
    for i in sorted({0, n // 2, n - 1}):
        s = scs[i]
        np.testing.assert_array_equal(got[i], oracle.compute(s.left, s.right, s.lidar, D, dumps=False).out,
                                      err_msg=f"frame {i}")
