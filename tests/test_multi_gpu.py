"""Launch tuning, the autotuner and mixed-size batches in one CUDA graph.

Tuning changes launch shapes only, so every candidate must reproduce the
oracle bit for bit.  A mixed-size batch replays every class through the
same kernels inside one graph launch: each frame's output must equal the
oracle's, after the first (captured) launch and after replays with new
inputs written into the resident buffers.
"""
import numpy as np
import pytest

import oracle
from paper_2504_05148_gb300 import scenes
from paper_2504_05148_gb300 import sgmf as S

pytestmark = pytest.mark.gpu

# line kernels with each CTA shape, then the row-synchronous sweep
TUNINGS = [(w, px, 0) for w in (1, 2, 4, 8) for px in (32, 64, 128)] + [(4, px, 1) for px in (32, 64, 128)]


def _run(scene, params, tuning):
    import torch
    dev = torch.device("cuda:0")
    ctx = S.Context(scene.W, scene.H, scene.D, params)
    try:
        S.sgmf_set_tuning(ctx.handle, *tuning)
        assert S.sgmf_get_tuning(ctx.handle) == tuning
        out = torch.empty(scene.shape, dtype=torch.int16, device=dev)
        ctx.compute(torch.from_numpy(scene.left).to(dev), torch.from_numpy(scene.right).to(dev),
                    torch.from_numpy(scene.lidar).to(dev), out)
        ctx.sync()
        return out.cpu().numpy(), ctx.stage(S.SGMF_STAGE_COST), ctx.stage(S.SGMF_STAGE_DSTAR)
    finally:
        ctx.close()


@pytest.mark.parametrize("tuning", TUNINGS)
@pytest.mark.parametrize("shape", [(256, 128, 64), (71, 29, 100), (130, 40, 200), (9, 7, 3)])
def test_every_tuning_is_bit_exact(gpu, tuning, shape):
    W, H, D = shape
    s = scenes.tiny(1600) if shape == (256, 128, 64) else scenes.random_small(W + H + D, W, H, D)
    o = oracle.compute(s.left, s.right, s.lidar, s.D, volumes=True)
    out, cost, dstar = _run(s, S.Params(), tuning)
    np.testing.assert_array_equal(cost.astype(np.int64), o.cost, err_msg=f"cost {tuning}")
    np.testing.assert_array_equal(dstar, o.dstar, err_msg=f"d* {tuning}")
    np.testing.assert_array_equal(out, o.out, err_msg=f"out {tuning}")


def test_tunings_agree_at_full_size(gpu):
    s = scenes.kitti(2600)
    want = oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out
    for t in [(2, 32, 0), (8, 128, 0), (4, 64, 1), (4, 128, 1)]:
        np.testing.assert_array_equal(_run(s, S.Params(), t)[0], want, err_msg=str(t))


def test_bad_tuning_rejected(gpu):
    ctx = S.Context(64, 32, 32)
    try:
        assert S.sgmf_get_tuning(ctx.handle) == (4, 128, 0)      # line kernels by default
        for t in [(3, 128), (4, 100), (0, 0), (16, 64), (1, 16), (4, 128, 2), (4, 128, -1)]:
            with pytest.raises(S.SgmfError) as e:
                S.sgmf_set_tuning(ctx.handle, *t)
            assert e.value.status == S.SGMF_ERR_ARG
        assert S.sgmf_get_tuning(ctx.handle) == (4, 128, 0)
        S.sgmf_set_tuning(ctx.handle, 4, 128, 1)                  # the sweep fits this shape
        assert S.sgmf_get_tuning(ctx.handle) == (4, 128, 1)
    finally:
        ctx.close()


def test_autotune_keeps_results(gpu):
    import torch
    dev = torch.device("cuda:0")
    scs = [scenes.tiny(1610 + i) for i in range(3)]
    ctx = S.Context(256, 128, 64, max_batch=3)
    try:
        l = torch.from_numpy(np.stack([s.left for s in scs])).to(dev)
        r = torch.from_numpy(np.stack([s.right for s in scs])).to(dev)
        li = torch.from_numpy(np.stack([s.lidar for s in scs])).to(dev)
        o = torch.empty((3, 128, 256), dtype=torch.int16, device=dev)
        best, ms = S.sgmf_autotune(ctx.handle, 3, l.data_ptr(), r.data_ptr(), li.data_ptr(), o.data_ptr(), 2)
        assert best in TUNINGS and ms > 0.0
        assert S.sgmf_get_tuning(ctx.handle) == best
        o.fill_(7)
        ctx.compute(l, r, li, o)
        ctx.sync()
        got = o.cpu().numpy()
    finally:
        ctx.close()
    for i, s in enumerate(scs):
        np.testing.assert_array_equal(got[i], oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out)


def _fill(m, i, s):
    import torch
    lv, rv, dv, _ = m.frame_views(i)
    lv.copy_(torch.from_numpy(s.left))
    rv.copy_(torch.from_numpy(s.right))
    dv.copy_(torch.from_numpy(s.lidar))


def test_mixed_batch_graph_matches_oracle(gpu):
    import torch
    shapes = [(96, 40, 16), (71, 29, 100), (96, 40, 16), (130, 40, 200), (71, 29, 100), (50, 30, 256)]
    frames = [scenes.random_small(7000 + i, *sh) for i, sh in enumerate(shapes)]
    with S.Multi(shapes) as m:
        assert len(m.classes()) == 4
        assert [c[1] for c in m.classes()] == [2, 2, 1, 1]
        for i, s in enumerate(frames):
            _fill(m, i, s)
        torch.cuda.synchronize()
        m.launch()
        m.sync()
        for i, s in enumerate(frames):
            want = oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out
            np.testing.assert_array_equal(m.frame_views(i)[3].cpu().numpy(), want, err_msg=f"frame {i}")
        # replay the captured graph on new inputs written into the same buffers
        frames2 = [scenes.random_small(7100 + i, *sh) for i, sh in enumerate(shapes)]
        for i, s in enumerate(frames2):
            _fill(m, i, s)
        torch.cuda.synchronize()
        for _ in range(2):
            m.launch()
        m.sync()
        for i, s in enumerate(frames2):
            want = oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out
            np.testing.assert_array_equal(m.frame_views(i)[3].cpu().numpy(), want, err_msg=f"replay frame {i}")
        # 8 launches per class with the sweep, 10 with the three line kernels (Eq. 5 runs in the cost kernel)
        assert m.launches() == sum(8 if c[2][2] else 10 for c in m.classes())


def test_mixed_batch_autotune_then_replay(gpu):
    import torch
    shapes = [(256, 128, 64)] * 3 + [(71, 29, 100)] * 2
    frames = [scenes.tiny(1620 + i) for i in range(3)] + [scenes.random_small(7200 + i, 71, 29, 100) for i in range(2)]
    with S.Multi(shapes, S.Params(subpixel=1)) as m:
        for i, s in enumerate(frames):
            _fill(m, i, s)
        torch.cuda.synchronize()
        m.autotune(reps=1)
        for c in m.classes():
            assert c[2] in TUNINGS
        m.launch()
        m.sync()
        for i, s in enumerate(frames):
            want = oracle.compute(s.left, s.right, s.lidar, s.D, oracle.Params(subpixel=1), dumps=False).out
            np.testing.assert_array_equal(m.frame_views(i)[3].cpu().numpy(), want, err_msg=f"frame {i}")


def test_mixed_batch_full_sizes(gpu):
    """The four frame sizes of the mixed batch, three pairs each: every frame
    equals its single-context result, the first of each size also the oracle's."""
    import torch
    scs = scenes.mixed_batch(n_per_shape=3, distinct=2)
    shapes = [(s.W, s.H, s.D) for s in scs]
    dev = torch.device("cuda:0")
    with S.Multi(shapes) as m:
        for i, s in enumerate(scs):
            _fill(m, i, s)
        torch.cuda.synchronize()
        m.launch()
        m.launch()
        m.sync()
        got = [m.frame_views(i)[3].cpu().numpy() for i in range(len(scs))]
    for i, s in enumerate(scs):
        ctx = S.Context(s.W, s.H, s.D)
        try:
            out = torch.empty(s.shape, dtype=torch.int16, device=dev)
            ctx.compute(torch.from_numpy(s.left).to(dev), torch.from_numpy(s.right).to(dev),
                        torch.from_numpy(s.lidar).to(dev), out)
            ctx.sync()
            np.testing.assert_array_equal(got[i], out.cpu().numpy(), err_msg=f"frame {i} {s.name}")
        finally:
            ctx.close()
    for i in range(0, len(scs), 3):
        s = scs[i]
        want = oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out
        np.testing.assert_array_equal(got[i], want, err_msg=f"oracle {s.name}")
