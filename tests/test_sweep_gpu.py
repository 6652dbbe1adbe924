"""The row-synchronous sweep (tuning sweep = 1): one cluster per frame and
sweep direction carries the vertical and both diagonal directions of Eq. 2
row by row, exchanging edge vectors between groups and CTAs.  Its S, d*, d'
and output must equal the oracle's bit for bit on clusters of one to eight
CTAs with ragged last strips and groups, every lane width, the u16 path-cost
range, sub-pixel output and batches; where it does not fit, the context keeps
the line kernels and refuses the tuning.  (Its banded mode is tested with the
other banded cases.)"""
import numpy as np
import pytest

import oracle
from paper_2504_05148_gb300 import scenes
from paper_2504_05148_gb300 import sgmf as S

pytestmark = pytest.mark.gpu


def _run(scene, params=None, sweep=1, debug=True):
    import torch
    dev = torch.device("cuda:0")
    ctx = S.Context(scene.W, scene.H, scene.D, params)
    try:
        S.sgmf_set_tuning(ctx.handle, 4, 128, sweep)
        ctx.set_debug(debug)
        out = torch.empty(scene.shape, dtype=torch.int16, device=dev)
        ctx.compute(torch.from_numpy(scene.left).to(dev), torch.from_numpy(scene.right).to(dev),
                    torch.from_numpy(scene.lidar).to(dev), out)
        ctx.sync()
        res = {"out": out.cpu().numpy(), "dstar": ctx.stage(S.SGMF_STAGE_DSTAR),
               "dprime": ctx.stage(S.SGMF_STAGE_DPRIME)}
        if debug:
            res["sum"] = ctx.stage(S.SGMF_STAGE_SUM)
        res["launches"] = S.sgmf_launches_per_compute(ctx.handle)
        return res
    finally:
        ctx.close()


def _check(scene, params=None):
    p = params or S.Params()
    g = _run(scene, p)
    o = oracle.compute(scene.left, scene.right, scene.lidar, scene.D, oracle.Params(**vars(p)), volumes=True)
    bad = np.argwhere(g["sum"].astype(np.int64)[:, :, :scene.D] != o.sum[:, :, :scene.D])
    assert len(bad) == 0, f"{scene.name}: S differs at {len(bad)} cells, first {bad[:4].tolist()}"
    for name in ("dstar", "dprime", "out"):
        np.testing.assert_array_equal(g[name], getattr(o, name), err_msg=f"{scene.name} {name}")
    return g


# (W, H, D): clusters of 8 to 16 CTAs with a ragged last strip (1242, 2040),
# full CTAs (1280 at Dp = 64), the two wide lane widths at their widest rows
# (1280 at Dp = 256), ragged groups inside one CTA, one-pixel-wide and
# one-row frames
SHAPES = [(1242, 24, 128), (2040, 6, 128), (1280, 12, 64), (1280, 6, 256), (640, 14, 256), (300, 30, 192),
          (161, 21, 128), (17, 9, 100), (1, 5, 16), (2, 3, 3), (9, 1, 64), (33, 40, 64)]


@pytest.mark.parametrize("W,H,D", SHAPES)
def test_sweep_matches_oracle(gpu, W, H, D):
    s = scenes.random_small(W * 7 + H * 3 + D, W, H, D)
    g = _check(s)
    assert g["launches"] == 8             # one sweep launch instead of three line launches


@pytest.mark.parametrize("case", ["u16_range", "subpixel", "dsgm", "census_full", "no_check"])
def test_sweep_parameter_variants(gpu, case):
    s = scenes.random_small(9400, 203, 37, 128)
    p = {"u16_range": S.Params(p2=300), "subpixel": S.Params(subpixel=1), "dsgm": S.Params(semidense=0),
         "census_full": S.Params(census=S.SGMF_CENSUS_9X7),
         "no_check": S.Params(consistency=S.SGMF_CHECK_NONE)}[case]
    _check(s, p)


def test_sweep_equals_line_kernels_at_full_size(gpu):
    s = scenes.kitti(2750)
    a = _run(s, sweep=1)
    b = _run(s, sweep=0)
    for name in ("sum", "dstar", "dprime", "out"):
        np.testing.assert_array_equal(a[name], b[name], err_msg=name)
    want = oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out
    np.testing.assert_array_equal(a["out"], want)


def test_sweep_batch(gpu):
    import torch
    dev = torch.device("cuda:0")
    scs = [scenes.random_small(9500 + i, 410, 33, 128) for i in range(3)]
    ctx = S.Context(410, 33, 128, max_batch=3)
    try:
        S.sgmf_set_tuning(ctx.handle, 4, 128, 1)
        out = torch.empty((3, 33, 410), dtype=torch.int16, device=dev)
        ctx.compute(torch.from_numpy(np.stack([s.left for s in scs])).to(dev),
                    torch.from_numpy(np.stack([s.right for s in scs])).to(dev),
                    torch.from_numpy(np.stack([s.lidar for s in scs])).to(dev), out)
        ctx.sync()
        got = out.cpu().numpy()
    finally:
        ctx.close()
    for i, s in enumerate(scs):
        np.testing.assert_array_equal(got[i], oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out,
                                      err_msg=f"frame {i}")


def test_four_paths_keep_the_line_kernel(gpu):
    s = scenes.random_small(9600, 120, 30, 64)
    p = S.Params(num_paths=4)
    g = _run(s, p, debug=False)
    want = oracle.compute(s.left, s.right, s.lidar, s.D, oracle.Params(**vars(p)), dumps=False).out
    np.testing.assert_array_equal(g["out"], want)


def test_sweep_refused_where_it_does_not_fit(gpu):
    # a row wider than sixteen CTAs of 128 pixels (Dp = 128)
    ctx = S.Context(3200, 8, 128)
    try:
        assert S.sgmf_get_tuning(ctx.handle)[2] == 0
        with pytest.raises(S.SgmfError) as e:
            S.sgmf_set_tuning(ctx.handle, 4, 128, 1)
        assert e.value.status == S.SGMF_ERR_ARG
    finally:
        ctx.close()
    # a banded context takes the sweep (off by default)
    h = S.sgmf_create_banded(256, 32, 128, 64, 1)
    try:
        assert S.sgmf_get_tuning(h)[2] == 0
        S.sgmf_set_tuning(h, 4, 128, 1)
        assert S.sgmf_get_tuning(h)[2] == 1
    finally:
        S.sgmf_destroy(h)


def test_split_batch_matches_oracle(gpu):
    """16 frames of a 1242-pixel row: the batch splits into a first part of
    whole sweep waves, whose row kernel runs on the second stream beside the
    rest's sweep; every frame must equal the oracle, and the result must not
    depend on the split (a one-frame context gives the same output)."""
    import torch
    dev = torch.device("cuda:0")
    W, H, D, n = 1242, 10, 128, 16
    scs = [scenes.random_small(9800 + i, W, H, D) for i in range(n)]
    ctx = S.Context(W, H, D, max_batch=n)
    try:
        S.sgmf_set_tuning(ctx.handle, 4, 128, 1)
        assert S.sgmf_tuning_of(ctx.handle).parts == 1
        out = torch.empty((n, H, W), dtype=torch.int16, device=dev)
        for _ in range(2):                 # twice: the events and the second stream are reused
            out.fill_(-7)
            ctx.compute(torch.from_numpy(np.stack([s.left for s in scs])).to(dev),
                        torch.from_numpy(np.stack([s.right for s in scs])).to(dev),
                        torch.from_numpy(np.stack([s.lidar for s in scs])).to(dev), out)
            ctx.sync()
        got = out.cpu().numpy()
        # the whole batch in one launch per kernel gives the same output
        S.sgmf_set_tuning(ctx.handle, 4, 128, 1, 0)
        out.fill_(-7)
        ctx.compute(torch.from_numpy(np.stack([s.left for s in scs])).to(dev),
                    torch.from_numpy(np.stack([s.right for s in scs])).to(dev),
                    torch.from_numpy(np.stack([s.lidar for s in scs])).to(dev), out)
        ctx.sync()
        np.testing.assert_array_equal(out.cpu().numpy(), got)
        with pytest.raises(S.SgmfError):
            S.sgmf_set_tuning(ctx.handle, 4, 128, 1, 2)
    finally:
        ctx.close()
    for i, s in enumerate(scs):
        np.testing.assert_array_equal(got[i], oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out,
                                      err_msg=f"frame {i}")


def test_bench_configuration_at_full_size(gpu):
    """The timed configuration: 32 KITTI-shaped frames in one call through the
    sweep (in parts of one sweep wave, row kernels on the second stream).
    Every frame equals the line-kernel path's; the first frame, the first of
    the second part and the last also equal the oracle."""
    import torch
    dev = torch.device("cuda:0")
    n = 32
    scs = [scenes.kitti(12000 + i) for i in range(n)]
    l = torch.from_numpy(np.stack([s.left for s in scs])).to(dev)
    r = torch.from_numpy(np.stack([s.right for s in scs])).to(dev)
    li = torch.from_numpy(np.stack([s.lidar for s in scs])).to(dev)
    got = {}
    for sweep in (1, 0):
        ctx = S.Context(1242, 375, 128, max_batch=n)
        try:
            S.sgmf_set_tuning(ctx.handle, 4, 128, sweep)
            out = torch.empty((n, 375, 1242), dtype=torch.int16, device=dev)
            ctx.compute(l, r, li, out)
            ctx.sync()
            got[sweep] = out.cpu().numpy()
        finally:
            ctx.close()
    np.testing.assert_array_equal(got[1], got[0])
    for i in (0, 13, n - 1):
        s = scs[i]
        np.testing.assert_array_equal(got[1][i], oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out,
                                      err_msg=f"frame {i}")
