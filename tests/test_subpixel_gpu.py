"""Parity of the sub-pixel output (parabola fit after Eq. 3, in 1/16 px).

The fit is integer arithmetic on S(d*-1), S(d*), S(d*+1), so the CUDA path's
sub-pixel map and its output must equal the oracle's bit for bit: the whole
map with the check off, and every pixel (kept or -1) with it on.
"""
import numpy as np
import pytest

import oracle
from paper_2504_05148_gb300 import scenes
from paper_2504_05148_gb300 import sgmf as S

pytestmark = pytest.mark.gpu


def _gpu(scene, params):
    import torch
    dev = torch.device("cuda:0")
    ctx = S.Context(scene.W, scene.H, scene.D, params)
    try:
        out = torch.empty(scene.shape, dtype=torch.int16, device=dev)
        ctx.compute(torch.from_numpy(scene.left).to(dev), torch.from_numpy(scene.right).to(dev),
                    torch.from_numpy(scene.lidar).to(dev), out)
        ctx.sync()
        return out.cpu().numpy(), ctx.stage(S.SGMF_STAGE_DSUB), ctx.stage(S.SGMF_STAGE_DSTAR)
    finally:
        ctx.close()


def _check(scene, params):
    out, dsub, dstar = _gpu(scene, params)
    o = oracle.compute(scene.left, scene.right, scene.lidar, scene.D, oracle.Params(**vars(params)),
                       volumes=True)
    np.testing.assert_array_equal(dstar, o.dstar, err_msg=f"{scene.name}: d*")
    want = oracle.subpixel(o.sum, o.dstar)
    bad = np.argwhere(dsub != want)
    assert len(bad) == 0, f"{scene.name}: sub-pixel map differs at {len(bad)} px, first {bad[:4].tolist()}"
    np.testing.assert_array_equal(out, o.out, err_msg=f"{scene.name}: output")
    return out, o


def test_tiny_no_check_whole_map(gpu):
    out, o = _check(scenes.tiny(1500), S.Params(subpixel=1, consistency=S.SGMF_CHECK_NONE))
    assert (out >= 0).all()
    assert (out % 16 != 0).mean() > 0.3          # many pixels land between integers


def test_tiny_with_check(gpu):
    _check(scenes.tiny(1501), S.Params(subpixel=1))


@pytest.mark.parametrize("W,H,D", [(9, 7, 3), (33, 17, 16), (64, 16, 37), (71, 29, 100), (65, 20, 128),
                                   (97, 23, 193), (50, 30, 256)])
def test_shapes(gpu, W, H, D):
    _check(scenes.random_small(W * 7 + H + D, W, H, D), S.Params(subpixel=1, consistency=S.SGMF_CHECK_NONE))


@pytest.mark.parametrize("case", ["u16_spill", "census_full", "four_paths"])
def test_parameter_variants(gpu, case):
    p = {"u16_spill": S.Params(subpixel=1, p2=300), "census_full": S.Params(subpixel=1, census=S.SGMF_CENSUS_9X7),
         "four_paths": S.Params(subpixel=1, num_paths=4)}[case]
    _check(scenes.random_small(88, 71, 29, 100), p)


def test_kitti_full_size(gpu):
    out, o = _check(scenes.kitti(2500), S.Params(subpixel=1))
    assert (out >= 0).mean() > 0.5


def test_integer_output_unchanged_when_off(gpu):
    """subpixel = 0 keeps the integer output (the default path is untouched)."""
    s = scenes.tiny(1502)
    import torch
    dev = torch.device("cuda:0")
    res = []
    for sp in (0, 1):
        ctx = S.Context(s.W, s.H, s.D, S.Params(subpixel=sp))
        try:
            out = torch.empty(s.shape, dtype=torch.int16, device=dev)
            ctx.compute(torch.from_numpy(s.left).to(dev), torch.from_numpy(s.right).to(dev),
                        torch.from_numpy(s.lidar).to(dev), out)
            ctx.sync()
            res.append(out.cpu().numpy().astype(int))
            if sp == 0:
                with pytest.raises(S.SgmfError):
                    ctx.stage(S.SGMF_STAGE_DSUB)
        finally:
            ctx.close()
    np.testing.assert_array_equal(res[0], oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out)
    v = res[0] >= 0
    np.testing.assert_array_equal(res[1] >= 0, v)
    assert (np.abs(res[1][v] - 16 * res[0][v]) <= 8).all()


def test_batch(gpu):
    import torch
    dev = torch.device("cuda:0")
    scs = [scenes.tiny(1510 + i) for i in range(3)]
    p = S.Params(subpixel=1)
    ctx = S.Context(scs[0].W, scs[0].H, scs[0].D, p, max_batch=4)
    try:
        o = torch.empty((3,) + scs[0].shape, dtype=torch.int16, device=dev)
        ctx.compute(torch.from_numpy(np.stack([s.left for s in scs])).to(dev),
                    torch.from_numpy(np.stack([s.right for s in scs])).to(dev),
                    torch.from_numpy(np.stack([s.lidar for s in scs])).to(dev), o)
        ctx.sync()
        got = o.cpu().numpy()
    finally:
        ctx.close()
    for i, s in enumerate(scs):
        want = oracle.compute(s.left, s.right, s.lidar, s.D, oracle.Params(subpixel=1), dumps=False).out
        np.testing.assert_array_equal(got[i], want, err_msg=f"frame {i}")
