"""Training and inference of the band proposal.

(1) One forward/backward pass of the whole network on the GPU against the
float64 reference (activations and inter-layer gradients are stored in
bf16 on the GPU, hence the relative tolerances); (2) training lowers the
loss; (3) the learned pipeline is exactly the banded method on the bands it
proposes (bit-exact with the banded oracle); (4) training is what makes the
proposal useful: the trained network's output disagrees with the plain
method far less than an untrained one's, without falling back."""
import numpy as np
import pytest

import oracle
from oracle import band_net as N
from paper_2504_05148_gb300 import bandnet, scenes
from paper_2504_05148_gb300 import sgmf as S

pytestmark = pytest.mark.gpu


def _host_params(net):
    flat = net.master.cpu().numpy().astype(np.float64)
    ws, bs = [], []
    for l in range(bandnet.LAYERS):
        w = flat[l * bandnet.PSZ:l * bandnet.PSZ + bandnet.WSZ].reshape(32, 3, 3, 32)
        ws.append(N.bf16_round(w))
        bs.append(flat[l * bandnet.PSZ + bandnet.WSZ:(l + 1) * bandnet.PSZ].astype(np.float32).astype(np.float64))
    return ws, bs


def test_network_pass_matches_reference(gpu):
    import torch
    net = bandnet.BandNet(seed=3)
    rng = np.random.default_rng(5)
    n, h, w = 2, 10, 17
    x = np.zeros((n, h, w, 32))
    x[..., :3] = N.bf16_round(rng.normal(scale=0.5, size=(n, h, w, 3)))
    xb = torch.from_numpy(((x.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)).view(np.int16)).cuda()
    acts, out = net.forward(xb, n, h, w)
    gout = N.bf16_round(rng.normal(scale=1e-2, size=(n, h, w, 32)))
    gb = torch.from_numpy(((gout.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)).view(np.int16)).cuda()
    net.backward(acts, gb, n, h, w)
    net.check()
    ws, bs = _host_params(net)
    racts, rout = N.forward(x, ws, bs)
    got = out.cpu().numpy().astype(np.float64)
    assert np.abs(got - rout).max() <= 2e-2 * np.abs(rout).max()
    dws, dbs = N.backward(racts, ws, gout)
    g = net.grad.cpu().numpy().astype(np.float64)
    for l in range(bandnet.LAYERS):
        gw = g[l * bandnet.PSZ:l * bandnet.PSZ + bandnet.WSZ].reshape(32, 3, 3, 32)
        gbias = g[l * bandnet.PSZ + bandnet.WSZ:(l + 1) * bandnet.PSZ]
        scale = max(np.abs(dws[l]).max(), 1e-12)
        assert np.abs(gw - dws[l]).max() <= 5e-2 * scale, l
        assert np.abs(gbias - dbs[l]).max() <= 5e-2 * max(np.abs(dbs[l]).max(), 1e-12), l


def _small_set(n_pairs, W=320, H=96, D=128, seed0=900000):
    return bandnet.build_training_set(n_pairs, seed0=seed0, W=W, H=H, D=D, batch=8)


@pytest.fixture(scope="module")
def trained():
    x_all, lohi, counts = _small_set(48)
    net = bandnet.BandNet(seed=1)
    before = bandnet.evaluate(net, x_all, lohi, counts, batch=8, D=128)
    bandnet.train(net, x_all, lohi, counts, steps=300, batch=8, lr=3e-3, log_every=0, D=128)
    after = bandnet.evaluate(net, x_all, lohi, counts, batch=8, D=128)
    return net, (before, after)


def test_training_lowers_the_loss(gpu, trained):
    _, (before, after) = trained
    assert after < 0.7 * before, (before, after)


def _run_learned(net, s, band, conf_min=0.0, fallback_frac=1.0):
    """One frame through the learned pipeline: (output, band starts, fell back to the plain method)."""
    import torch
    dev = torch.device("cuda")
    L = bandnet.LearnedSGM(s.W, s.H, s.D, net, band=band, conf_min=conf_min, fallback_frac=fallback_frac)
    try:
        out = torch.empty((1, s.H, s.W), dtype=torch.int16, device=dev)
        L.compute(torch.from_numpy(s.left[None]).to(dev), torch.from_numpy(s.right[None]).to(dev),
                  torch.from_numpy(s.lidar[None]).to(dev), out)
        L.sync()
        gate, _ = L.decision()
        return out[0].cpu().numpy(), L.lo[0][0].cpu().numpy(), bool(gate[0] == L.PLAIN), None
    finally:
        L.close()


def test_learned_pipeline_is_the_banded_method(gpu, trained):
    net, _ = trained
    s = scenes.street(910000, 320, 96, 128)
    got, lo_t, fell, _ = _run_learned(net, s, 64)
    assert not fell
    o = oracle.compute_banded(s.left, s.right, s.lidar, s.D, 64, oracle.expand_tiles(lo_t, s.W, s.H, S.BAND_TILE))
    np.testing.assert_array_equal(got, o.out)


def test_training_is_what_makes_the_bands_useful(gpu, trained):
    net, _ = trained
    fresh = bandnet.BandNet(seed=7)
    s = scenes.street(920000, 320, 96, 128)
    plain = oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out
    got_t, _, fell_t, _ = _run_learned(net, s, 64)
    got_u, _, fell_u, _ = _run_learned(fresh, s, 64)
    assert not fell_t and not fell_u
    dt, du = bandnet.disagreement(got_t, plain), bandnet.disagreement(got_u, plain)
    assert dt < 0.5 * du, (dt, du)


def test_fallback_runs_the_plain_method(gpu, trained):
    net, _ = trained
    s = scenes.street(930000, 320, 96, 128)
    got, _, fell, _ = _run_learned(net, s, 64, conf_min=1.1, fallback_frac=0.0)   # every tile uncertain
    assert fell
    np.testing.assert_array_equal(got, oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False).out)


def test_gates_split_a_batch_between_contexts(gpu):
    """Per-frame gates: one batch, a banded and a plain context sharing it by
    a device gate array (hand-set here, as sgmf_bn_decide would write it).
    Each frame's output is exactly the method its gate word names, and a
    context leaves the frames it skips untouched."""
    import torch
    dev = torch.device("cuda")
    frames = [scenes.street(940000 + i, 320, 96, 128) for i in range(4)]
    st = lambda k: torch.from_numpy(np.stack([getattr(f, k) for f in frames])).to(dev)
    gate_h = np.array([0, 1, 1, 0], np.int32)
    gate = torch.from_numpy(gate_h).to(dev)
    th, tw = (96 + S.BAND_TILE - 1) // S.BAND_TILE, (320 + S.BAND_TILE - 1) // S.BAND_TILE
    rng = np.random.default_rng(3)
    lo = rng.integers(0, 128 - 64 + 1, size=(4, th, tw)).astype(np.int16)
    banded = S.Context(320, 96, 128, band=64, max_batch=4)
    plain = S.Context(320, 96, 128, max_batch=4)
    try:
        out = torch.full((4, 96, 320), 7777, dtype=torch.int16, device=dev)
        S.sgmf_set_gate(banded.handle, gate.data_ptr(), 0)
        banded.compute_banded(st("left"), st("right"), st("lidar"), torch.from_numpy(lo).to(dev), out)
        banded.sync()
        only_banded = out.cpu().numpy().copy()
        S.sgmf_set_gate(plain.handle, gate.data_ptr(), 1)
        plain.compute(st("left"), st("right"), st("lidar"), out)
        plain.sync()
        got = out.cpu().numpy()
    finally:
        banded.close()
        plain.close()
    for i, f in enumerate(frames):
        if gate_h[i] == 1:
            assert (only_banded[i] == 7777).all(), "the banded context wrote a frame it skips"
            want = oracle.compute(f.left, f.right, f.lidar, f.D, dumps=False).out
        else:
            want = oracle.compute_banded(f.left, f.right, f.lidar, f.D, 64,
                                         oracle.expand_tiles(lo[i], f.W, f.H, S.BAND_TILE)).out
        np.testing.assert_array_equal(got[i], want, err_msg=f"frame {i}, gate {gate_h[i]}")


def test_learned_batch_frames_follow_their_decision(gpu, trained):
    """Two band widths in one learned call: every frame's output equals the
    banded oracle on the bands of the width its device-side decision chose
    (or the plain method where it fell back)."""
    import torch
    net, _ = trained
    dev = torch.device("cuda")
    frames = [scenes.street(941000 + i, 320, 96, 128) for i in range(3)]
    st = lambda k: torch.from_numpy(np.stack([getattr(f, k) for f in frames])).to(dev)
    L = bandnet.LearnedSGM(320, 96, 128, net, bands=(64, 128), conf_min=0.5, fallback_frac=0.5, max_batch=3)
    try:
        out = torch.empty((3, 96, 320), dtype=torch.int16, device=dev)
        L.compute(st("left"), st("right"), st("lidar"), out)
        L.sync()
        gate, unc = L.decision()
        got = out.cpu().numpy()
        los = [t.cpu().numpy() for t in L.lo]
    finally:
        L.close()
    tiles = L.th * L.tw
    for i, f in enumerate(frames):
        g = int(gate[i])
        want_g = 0 if unc[0, i] <= int(0.5 * tiles) else (1 if unc[1, i] <= int(0.5 * tiles) else L.PLAIN)
        assert g == want_g, (i, gate, unc)
        if g == L.PLAIN:
            want = oracle.compute(f.left, f.right, f.lidar, f.D, dumps=False).out
        else:
            B = L.bands[g]
            want = oracle.compute_banded(f.left, f.right, f.lidar, f.D, B,
                                         oracle.expand_tiles(los[g][i], f.W, f.H, S.BAND_TILE)).out
        np.testing.assert_array_equal(got[i], want, err_msg=f"frame {i}, path {g}")
