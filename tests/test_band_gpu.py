"""Parity of the banded mode (sgmf_create_banded / sgmf_compute_banded) with
the banded oracle: every map, the banded cost and the banded S bit for bit,
on random band tables (jumps at every tile edge), smooth ones, the
full-range band and batches."""
import numpy as np
import pytest

import oracle
from paper_2504_05148_gb300 import scenes
from paper_2504_05148_gb300 import sgmf as S

pytestmark = pytest.mark.gpu


def _tiles(W, H):
    return (H + S.BAND_TILE - 1) // S.BAND_TILE, (W + S.BAND_TILE - 1) // S.BAND_TILE


def _gpu(scene, B, lo_tiles, params=None, lidar=True, sweep=0):
    import torch
    dev = torch.device("cuda:0")
    ctx = S.Context(scene.W, scene.H, scene.D, params, band=B)
    try:
        if sweep:
            S.sgmf_set_tuning(ctx.handle, 4, 128, 1)     # the cluster sweep on the bands
        ctx.set_debug(True)          # keeps the banded S of the frame for the comparison
        out = torch.empty(scene.shape, dtype=torch.int16, device=dev)
        ctx.compute_banded(torch.from_numpy(scene.left).to(dev), torch.from_numpy(scene.right).to(dev),
                           torch.from_numpy(scene.lidar).to(dev) if lidar else None,
                           torch.from_numpy(np.ascontiguousarray(lo_tiles, np.int16)).to(dev), out)
        ctx.sync()
        return {"out": out.cpu().numpy(), "dstar": ctx.stage(S.SGMF_STAGE_DSTAR),
                "dprime": ctx.stage(S.SGMF_STAGE_DPRIME), "cost": ctx.stage(S.SGMF_STAGE_COST),
                "sum": ctx.stage(S.SGMF_STAGE_SUM)}
    finally:
        ctx.close()


def _check(scene, B, lo_tiles, params=None, lidar=True, sweep=0):
    params = params or S.Params()
    lo_c = np.clip(lo_tiles, 0, scene.D - B).astype(np.int16)
    g = _gpu(scene, B, lo_tiles, params, lidar, sweep)
    lo = oracle.expand_tiles(lo_c, scene.W, scene.H, S.BAND_TILE)
    o = oracle.compute_banded(scene.left, scene.right, scene.lidar if lidar else None, scene.D, B, lo,
                              oracle.Params(**vars(params)), volumes=True)
    plain = oracle.compute(scene.left, scene.right, scene.lidar if lidar else None, scene.D,
                           oracle.Params(**vars(params)), volumes=True)
    idx = lo[:, :, None].astype(np.int64) + np.arange(B)[None, None, :]
    want_cost = np.take_along_axis(plain.cost, idx, axis=2)
    np.testing.assert_array_equal(g["cost"].astype(np.int64), want_cost, err_msg=f"{scene.name} cost")
    want_sum = np.take_along_axis(o.sum, idx, axis=2)
    bad = np.argwhere(g["sum"].astype(np.int64) != want_sum)
    assert len(bad) == 0, f"{scene.name}: banded S differs at {len(bad)} cells, first {bad[:4].tolist()}"
    for name in ("dstar", "dprime", "out"):
        np.testing.assert_array_equal(g[name], getattr(o, name), err_msg=f"{scene.name} {name}")
    return g, o


@pytest.mark.parametrize("sweep", [0, 1])
@pytest.mark.parametrize("B", [64, 128])
@pytest.mark.parametrize("W,H,D", [(256, 128, 128), (71, 29, 200), (130, 40, 256), (33, 17, 128), (200, 50, 160),
                                   (1300, 20, 192)])
def test_random_band_tables(gpu, B, W, H, D, sweep):
    if B > D:
        pytest.skip("band wider than the range")
    s = scenes.random_small(W * 3 + H + D + B, W, H, D)
    rng = np.random.default_rng(W + H + D + B)
    lo = rng.integers(-5, D - B + 6, size=_tiles(W, H))          # out-of-range starts get clamped
    _check(s, B, lo, sweep=sweep)


@pytest.mark.parametrize("sweep", [0, 1])
def test_smooth_bands_from_the_truth(gpu, sweep):
    s = scenes.kitti(2700)
    B = 64
    th, tw = _tiles(s.W, s.H)
    lo = np.zeros((th, tw), np.int64)
    T = S.BAND_TILE
    for ty in range(th):
        for tx in range(tw):
            blk = s.truth[T * ty:T * ty + T, T * tx:T * tx + T]
            lo[ty, tx] = int(np.median(blk)) - B // 2
    g, o = _check(s, B, lo, sweep=sweep)
    assert (g["out"] >= 0).mean() > 0.5


def test_full_range_band_is_the_plain_method(gpu):
    s = scenes.random_small(9100, 150, 60, 128)
    lo = np.zeros(_tiles(150, 60), np.int16)
    g, _ = _check(s, 128, lo)
    want = oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out
    np.testing.assert_array_equal(g["out"], want)


@pytest.mark.parametrize("sweep", [0, 1])
@pytest.mark.parametrize("case", ["dsgm", "four_paths", "u16_spill", "no_lidar", "census_full"])
def test_parameter_variants(gpu, case, sweep):
    s = scenes.random_small(9200, 97, 45, 192)
    rng = np.random.default_rng(9)
    lo = rng.integers(0, 192 - 64 + 1, size=_tiles(97, 45))
    p = {"dsgm": S.Params(semidense=0), "four_paths": S.Params(num_paths=4), "u16_spill": S.Params(p2=300),
         "no_lidar": S.Params(), "census_full": S.Params(census=S.SGMF_CENSUS_9X7)}[case]
    _check(s, 64, lo, p, lidar=case != "no_lidar", sweep=sweep)


@pytest.mark.parametrize("sweep", [0, 1])
def test_batch(gpu, sweep):
    import torch
    dev = torch.device("cuda:0")
    scs = [scenes.random_small(9300 + i, 120, 50, 128) for i in range(3)]
    rng = np.random.default_rng(3)
    los = [rng.integers(0, 65, size=_tiles(120, 50)).astype(np.int16) for _ in scs]
    ctx = S.Context(120, 50, 128, band=64, max_batch=3)
    try:
        if sweep:
            S.sgmf_set_tuning(ctx.handle, 4, 128, 1)
        out = torch.empty((3, 50, 120), dtype=torch.int16, device=dev)
        ctx.compute_banded(torch.from_numpy(np.stack([s.left for s in scs])).to(dev),
                           torch.from_numpy(np.stack([s.right for s in scs])).to(dev),
                           torch.from_numpy(np.stack([s.lidar for s in scs])).to(dev),
                           torch.from_numpy(np.stack(los)).to(dev), out)
        ctx.sync()
        got = out.cpu().numpy()
    finally:
        ctx.close()
    for i, s in enumerate(scs):
        o = oracle.compute_banded(s.left, s.right, s.lidar, s.D, 64,
                                  oracle.expand_tiles(los[i], 120, 50, S.BAND_TILE))
        np.testing.assert_array_equal(got[i], o.out, err_msg=f"frame {i}")


def test_banded_context_rules(gpu):
    with pytest.raises(S.SgmfError):
        S.sgmf_create_banded(64, 32, 100, 96, 1)         # band must be 64 or 128
    with pytest.raises(S.SgmfError):
        S.sgmf_create_banded(64, 32, 100, 128, 1)        # band wider than the range
    h = S.sgmf_create_banded(64, 32, 128, 64, 1)
    try:
        assert S.sgmf_band_width(h) == 64
        with pytest.raises(S.SgmfError):
            S.sgmf_compute(h, 1, 1, None, 1)             # plain compute refuses a banded context
    finally:
        S.sgmf_destroy(h)
