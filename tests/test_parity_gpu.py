"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

All arithmetic of the method is integer, so every compared map must match
the oracle bit for bit: d-bar, both census images, d-hat, the uint8 cost
volume, the aggregate S (where kept), d*, d' and the output D^{c*}.
"""
import threading

import numpy as np
import pytest

import oracle
from paper_2504_05148_gb300 import scenes
from paper_2504_05148_gb300 import sgmf as S

pytestmark = pytest.mark.gpu

STAGES = {
    "dbar": S.SGMF_STAGE_DBAR, "census_l": S.SGMF_STAGE_CENSUS_L, "census_r": S.SGMF_STAGE_CENSUS_R,
    "dhat": S.SGMF_STAGE_DHAT, "cost": S.SGMF_STAGE_COST, "sum": S.SGMF_STAGE_SUM,
    "dstar": S.SGMF_STAGE_DSTAR, "dprime": S.SGMF_STAGE_DPRIME,
}


def _to_oracle_params(p: S.Params) -> oracle.Params:
    return oracle.Params(**vars(p))


def run_gpu(scene, params=None, lidar=True, debug=True, stream=None):
    import torch
    params = params or S.Params()
    H, W = scene.shape
    ctx = S.Context(W, H, scene.D, params)
    try:
        if stream is not None:
            ctx.set_stream(stream)
        if debug:
            ctx.set_debug(True)
        dev = torch.device("cuda:0")
        left = torch.from_numpy(scene.left).to(dev)
        right = torch.from_numpy(scene.right).to(dev)
        li = torch.from_numpy(scene.lidar).to(dev) if lidar else None
        out = torch.empty((H, W), dtype=torch.int16, device=dev)
        ctx.compute(left, right, li, out)
        ctx.sync()
        res = {"out": out.cpu().numpy()}
        for name, st in STAGES.items():
            if name == "sum" and not debug:
                continue
            res[name] = ctx.stage(st)
        return res
    finally:
        ctx.close()


def compare(scene, params=None, lidar=True, volumes=True):
    params = params or S.Params()
    g = run_gpu(scene, params, lidar=lidar, debug=volumes)
    o = oracle.compute(scene.left, scene.right, scene.lidar if lidar else None, scene.D,
                       _to_oracle_params(params), volumes=volumes)
    order = ["dbar", "census_l", "census_r", "dhat"]
    if volumes:
        order += ["cost", "sum"]
    order += ["dstar", "dprime", "out"]
    for name in order:
        a = g[name]
        b = getattr(o, name)
        if name in ("cost", "sum"):
            b = b.astype(np.int64)
            a = a.astype(np.int64)
        if not np.array_equal(a, b):
            bad = np.argwhere(a != b)
            raise AssertionError(f"{scene.name}: stage {name} differs at {len(bad)} places, first {bad[:5].tolist()} "
                                 f"gpu={a[tuple(bad[0])]} oracle={b[tuple(bad[0])]}")
    return g, o


def test_tiny_bit_exact(gpu):
    compare(scenes.tiny(1000))


@pytest.mark.parametrize("seed", [1001, 1002, 1003])
def test_tiny_seeds(gpu, seed):
    compare(scenes.tiny(seed), volumes=False)


def test_kitti_full_size_bit_exact(gpu):
    """1242 x 375, D = 128: the benchmark workload, compared on every output."""
    compare(scenes.kitti(2000), volumes=False)


def test_kitti_volumes_bit_exact(gpu):
    compare(scenes.kitti(2001), volumes=True)


@pytest.mark.parametrize("beams", [32, 16, 8])
def test_kitti_beam_sweep(gpu, beams):
    compare(scenes.kitti(2100 + beams, beams=beams), volumes=False)


def test_indoor(gpu):
    compare(scenes.indoor(3200), volumes=False)


def test_lowlight(gpu):
    compare(scenes.lowlight(3300), volumes=False)


@pytest.mark.parametrize("W,H,D", [
    (1, 1, 1), (2, 3, 2), (5, 4, 4), (8, 6, 9), (9, 7, 16), (17, 5, 3), (31, 33, 64), (33, 17, 37),
    (64, 16, 65), (65, 20, 128), (100, 40, 129), (70, 9, 192), (97, 23, 193), (50, 30, 256),
    (300, 8, 255), (130, 70, 100), (16, 100, 64), (256, 3, 200),
])
def test_random_shapes(gpu, W, H, D):
    compare(scenes.random_small(W * 1000 + H * 10 + D, W, H, D))


PARAM_CASES = {
    "dsgm": S.Params(semidense=0),
    "census_full": S.Params(census=S.SGMF_CENSUS_9X7),
    "four_paths": S.Params(num_paths=4),
    "stereo_check": S.Params(consistency=S.SGMF_CHECK_STEREO),
    "lidar_check": S.Params(consistency=S.SGMF_CHECK_LIDAR),
    "no_check": S.Params(consistency=S.SGMF_CHECK_NONE),
    "alpha0": S.Params(alpha_num=0),
    "u16_spill": S.Params(p2=300),
    "big_q": S.Params(q1=40, q2=300),
    "p1_eq_p2": S.Params(p1=50, p2=50),
    "zero_pen": S.Params(p1=0, p2=0),
    "ts9": S.Params(ts=9),
    "wide_windows": S.Params(rs=15, rc=40, tc=5),
    "huge_windows": S.Params(rs=50, rc=60, tc=3),          # the separable box-OR (radius > 48)
    "zero_windows": S.Params(rs=0, rc=0, tc=0),
    "lr2": S.Params(lr_max_diff=2),
    "full_census_big_p2": S.Params(census=S.SGMF_CENSUS_9X7, p2=1000, q2=200),
}


@pytest.mark.parametrize("case", sorted(PARAM_CASES))
def test_parameter_variants(gpu, case):
    compare(scenes.tiny(1010), PARAM_CASES[case])


@pytest.mark.parametrize("case", ["u16_spill", "census_full", "dsgm"])
def test_parameter_variants_ragged(gpu, case):
    compare(scenes.random_small(77, 71, 29, 100), PARAM_CASES[case])


def test_no_lidar_null_pointer(gpu):
    g, o = compare(scenes.tiny(1004), lidar=False)
    assert (g["dbar"] == -1).all()


def test_host_entry_point_matches_device(gpu):
    s = scenes.tiny(1005)
    g = run_gpu(s, debug=False)
    ctx = S.Context(s.W, s.H, s.D)
    try:
        out = np.empty(s.shape, np.int16)
        ctx.compute_host(s.left, s.right, s.lidar, out)
        np.testing.assert_array_equal(out, g["out"])
        out2 = np.empty(s.shape, np.int16)
        ctx.compute_host(s.left, s.right, None, out2)
        o = oracle.compute(s.left, s.right, None, s.D, dumps=False)
        np.testing.assert_array_equal(out2, o.out)
    finally:
        ctx.close()


def test_concurrent_streams_give_identical_results(gpu):
    import torch
    sc = [scenes.tiny(1020 + i) for i in range(4)]
    want = [oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out for s in sc]
    streams = [torch.cuda.Stream() for _ in sc]
    ctxs = [S.Context(s.W, s.H, s.D, stream=st) for s, st in zip(sc, streams)]
    dev = torch.device("cuda:0")
    try:
        outs = []
        for rep in range(3):
            outs = []
            for s, c, st in zip(sc, ctxs, streams):
                with torch.cuda.stream(st):
                    l = torch.from_numpy(s.left).to(dev, non_blocking=False)
                    r = torch.from_numpy(s.right).to(dev)
                    li = torch.from_numpy(s.lidar).to(dev)
                    o = torch.empty(s.shape, dtype=torch.int16, device=dev)
                    st.synchronize()
                    c.compute(l, r, li, o)
                    outs.append((o, l, r, li))
            for c in ctxs:
                c.sync()
            for (o, *_), w in zip(outs, want):
                np.testing.assert_array_equal(o.cpu().numpy(), w)
    finally:
        for c in ctxs:
            c.close()


def test_threads_with_host_entry_point(gpu):
    sc = [scenes.tiny(1030 + i) for i in range(3)]
    want = [oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out for s in sc]
    import torch
    streams = [torch.cuda.Stream() for _ in sc]
    ctxs = [S.Context(s.W, s.H, s.D, stream=st) for s, st in zip(sc, streams)]
    outs = [np.empty(s.shape, np.int16) for s in sc]
    errs = []

    def work(i):
        try:
            for _ in range(3):
                ctxs[i].compute_host(sc[i].left, sc[i].right, sc[i].lidar, outs[i])
        except Exception as e:  # pragma: no cover
            errs.append(e)

    th = [threading.Thread(target=work, args=(i,)) for i in range(len(sc))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    try:
        assert not errs, errs
        for o, w in zip(outs, want):
            np.testing.assert_array_equal(o, w)
    finally:
        for c in ctxs:
            c.close()


def test_bad_parameters_are_rejected(gpu):
    ctx = S.Context(32, 16, 16)
    try:
        for bad in (S.Params(p1=20, p2=10), S.Params(q1=9, q2=3), S.Params(alpha_num=11),
                    S.Params(alpha_den=0), S.Params(num_paths=5), S.Params(q2=400),
                    S.Params(p2=5000), S.Params(rs=-1), S.Params(consistency=7)):
            with pytest.raises(S.SgmfError) as e:
                ctx.set_params(bad)
            assert e.value.status == S.SGMF_ERR_PARAM
        # the previous parameters stay in force
        assert S.sgmf_get_params(ctx.handle) == S.Params()
        with pytest.raises(S.SgmfError) as e:
            S.sgmf_compute(ctx.handle, 0, 0, 0, 0)
        assert e.value.status == S.SGMF_ERR_ARG
        with pytest.raises(S.SgmfError):
            ctx.stage(S.SGMF_STAGE_SUM)      # debug not enabled
    finally:
        ctx.close()


def test_repeated_calls_reuse_scratch(gpu):
    """Nothing leaks between frames: run scene A, then B, then A again."""
    import torch
    a, b = scenes.tiny(1040), scenes.tiny(1041)
    ctx = S.Context(a.W, a.H, a.D)
    dev = torch.device("cuda:0")
    try:
        res = []
        for s in (a, b, a):
            o = torch.empty(s.shape, dtype=torch.int16, device=dev)
            ctx.compute(torch.from_numpy(s.left).to(dev), torch.from_numpy(s.right).to(dev),
                        torch.from_numpy(s.lidar).to(dev), o)
            ctx.sync()
            res.append(o.cpu().numpy())
        np.testing.assert_array_equal(res[0], res[2])
        np.testing.assert_array_equal(res[1], oracle.compute(b.left, b.right, b.lidar, b.D, dumps=False).out)
    finally:
        ctx.close()


def _batch_run(scs, params=None, lidar=True):
    import torch
    dev = torch.device("cuda:0")
    H, W, D = scs[0].H, scs[0].W, scs[0].D
    ctx = S.Context(W, H, D, params, max_batch=len(scs) + 1)
    try:
        l = torch.from_numpy(np.stack([s.left for s in scs])).to(dev)
        r = torch.from_numpy(np.stack([s.right for s in scs])).to(dev)
        li = torch.from_numpy(np.stack([s.lidar for s in scs])).to(dev) if lidar else None
        o = torch.empty((len(scs), H, W), dtype=torch.int16, device=dev)
        ctx.compute(l, r, li, o)
        ctx.sync()
        return o.cpu().numpy()
    finally:
        ctx.close()


@pytest.mark.parametrize("case", ["default", "dsgm", "u16_spill", "four_paths"])
def test_batch_matches_oracle_per_frame(gpu, case):
    params = S.Params() if case == "default" else PARAM_CASES[case]
    scs = [scenes.tiny(1100 + i) for i in range(3)]
    got = _batch_run(scs, params)
    for i, s in enumerate(scs):
        want = oracle.compute(s.left, s.right, s.lidar, s.D, _to_oracle_params(params), dumps=False).out
        np.testing.assert_array_equal(got[i], want, err_msg=f"frame {i}")


@pytest.mark.parametrize("W,H,D", [(71, 29, 100), (9, 7, 16), (130, 40, 200)])
def test_batch_ragged_shapes(gpu, W, H, D):
    scs = [scenes.random_small(5000 + i, W, H, D) for i in range(4)]
    got = _batch_run(scs)
    for i, s in enumerate(scs):
        np.testing.assert_array_equal(got[i], oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out)


def test_batch_full_size_and_host_batch(gpu):
    """Four 1242 x 375, D = 128 frames in one batch (the benchmark launch
    shape), through the device and the host batch entry points."""
    scs = [scenes.kitti(2200 + i) for i in range(4)]
    got = _batch_run(scs)
    want = [oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out for s in scs]
    for i in range(4):
        np.testing.assert_array_equal(got[i], want[i])
    ctx = S.Context(scs[0].W, scs[0].H, scs[0].D, max_batch=4)
    try:
        out = np.empty((4,) + scs[0].shape, np.int16)
        ctx.compute_host(np.stack([s.left for s in scs]), np.stack([s.right for s in scs]),
                         np.stack([s.lidar for s in scs]), out)
        for i in range(4):
            np.testing.assert_array_equal(out[i], want[i])
        with pytest.raises(S.SgmfError):
            S.sgmf_compute_batch(ctx.handle, 5, 1, 1, None, 1)
    finally:
        ctx.close()
