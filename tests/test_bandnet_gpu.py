"""The band-proposal network's kernels against the float64 reference
(oracle/band_net.py).  Inputs and weights are bfloat16 values on both sides,
so the forward and gradient GEMMs differ only by float32 accumulation
order: tolerances follow from 288-term (or pixel-count) float32 sums.
Shapes leave a ragged last tile of 128 pixels."""
import numpy as np
import pytest

from oracle import band_net as N
from paper_2504_05148_gb300 import sgmf as S

pytestmark = pytest.mark.gpu


def _bits(a64):
    """float64 array holding bf16 values -> uint16 bit patterns."""
    f = np.ascontiguousarray(a64, np.float32)
    return (f.view(np.uint32) >> 16).astype(np.uint16)


def _from_bits(u16):
    return (u16.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


_KEEP = []


def _dev(a):
    """Device copy kept alive until the test ends: a tensor freed right after
    data_ptr() would hand its memory to the next allocation before the
    asynchronous kernel that reads it has run."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    _KEEP.append(t)
    return t


@pytest.fixture(autouse=True)
def _release():
    yield
    import torch
    torch.cuda.synchronize()
    _KEEP.clear()


def _rand_bf16(rng, shape, scale=1.0):
    return N.bf16_round(rng.normal(scale=scale, size=shape))


class _Err:
    def __init__(self):
        import torch
        self.t = torch.zeros(1, dtype=torch.int32, device="cuda")

    @property
    def ptr(self):
        return self.t.data_ptr()

    def check(self):
        import torch
        torch.cuda.synchronize()
        assert int(self.t.item()) == 0, "a bounded wait gave up"


def _pack(w64):
    import torch
    wd = _dev(_bits(w64))
    pf = torch.empty(9216, dtype=torch.int16, device="cuda")
    pdg = torch.empty(9216, dtype=torch.int16, device="cuda")
    S.sgmf_bn_pack(wd.data_ptr(), pf.data_ptr(), pdg.data_ptr())
    return pf, pdg


@pytest.mark.parametrize("n,h,w", [(2, 13, 37), (1, 8, 16), (1, 1, 1), (3, 30, 41)])
def test_conv_forward(gpu, n, h, w):
    import torch
    rng = np.random.default_rng(n * 100 + h + w)
    x = _rand_bf16(rng, (n, h, w, 32))
    wt = _rand_bf16(rng, (32, 3, 3, 32), 0.1)
    b = rng.normal(size=32).astype(np.float32).astype(np.float64)
    pf, _ = _pack(wt)
    xd = _dev(_bits(x))
    yf = torch.empty((n, h, w, 32), dtype=torch.float32, device="cuda")
    yb = torch.empty((n, h, w, 32), dtype=torch.int16, device="cuda")
    err = _Err()
    S.sgmf_bn_conv(n, h, w, xd.data_ptr(), pf.data_ptr(), _dev(b.astype(np.float32)).data_ptr(), False, None,
                   None, yf.data_ptr(), err.ptr)
    S.sgmf_bn_conv(n, h, w, xd.data_ptr(), pf.data_ptr(), _dev(b.astype(np.float32)).data_ptr(), True, None,
                   yb.data_ptr(), None, err.ptr)
    err.check()
    ref = N.conv3x3(x, wt, b)
    got = yf.cpu().numpy().astype(np.float64)
    scale = N.conv3x3(np.abs(x), np.abs(wt), np.abs(b))          # sum of |terms| per output
    assert (np.abs(got - ref) <= 3e-5 * scale + 1e-7).all(), float(np.abs(got - ref).max())
    gb = _from_bits(yb.cpu().numpy().view(np.uint16))
    want = N.bf16_round(np.maximum(got, 0.0))                     # the bf16 store of the GPU's own f32
    np.testing.assert_array_equal(gb, want)


def test_conv_data_gradient_with_relu_mask(gpu):
    import torch
    rng = np.random.default_rng(7)
    n, h, w = 2, 11, 29
    dy = _rand_bf16(rng, (n, h, w, 32))
    act = N.bf16_round(np.maximum(rng.normal(size=(n, h, w, 32)), 0.0))   # about half the entries are 0
    wt = _rand_bf16(rng, (32, 3, 3, 32), 0.1)
    _, pdg = _pack(wt)
    out = torch.empty((n, h, w, 32), dtype=torch.float32, device="cuda")
    err = _Err()
    S.sgmf_bn_conv(n, h, w, _dev(_bits(dy)).data_ptr(), pdg.data_ptr(), None, False, _dev(_bits(act)).data_ptr(),
                   None, out.data_ptr(), err.ptr)
    err.check()
    ref = N.conv3x3_dgrad(dy, wt) * (act > 0)
    scale = N.conv3x3_dgrad(np.abs(dy), np.abs(wt))
    got = out.cpu().numpy().astype(np.float64)
    assert (np.abs(got - ref) <= 3e-5 * scale + 1e-7).all(), float(np.abs(got - ref).max())
    assert (got[act <= 0] == 0).all()


@pytest.mark.parametrize("n,h,w", [(2, 13, 37), (1, 40, 300), (1, 2, 3)])
def test_weight_gradient(gpu, n, h, w):
    import torch
    rng = np.random.default_rng(n + h + w)
    x = _rand_bf16(rng, (n, h, w, 32))
    dy = _rand_bf16(rng, (n, h, w, 32))
    dw = torch.zeros(32 * 288, dtype=torch.float32, device="cuda")
    db = torch.zeros(32, dtype=torch.float32, device="cuda")
    err = _Err()
    S.sgmf_bn_wgrad(n, h, w, _dev(_bits(x)).data_ptr(), _dev(_bits(dy)).data_ptr(), dw.data_ptr(), db.data_ptr(),
                    err.ptr)
    err.check()
    rw, rb = N.conv3x3_wgrad(x, dy)
    sw, sb = N.conv3x3_wgrad(np.abs(x), np.abs(dy))
    gw = dw.cpu().numpy().astype(np.float64).reshape(32, 3, 3, 32)
    gb = db.cpu().numpy().astype(np.float64)
    P = n * h * w
    tol = (P + 64) * 2.0 ** -23
    assert (np.abs(gw - rw) <= tol * sw + 1e-6).all(), float(np.abs(gw - rw).max())
    assert (np.abs(gb - rb) <= tol * sb + 1e-6).all()


def test_input_labels_loss_tiles_adam(gpu):
    import torch
    rng = np.random.default_rng(11)
    n, H, W, D = 2, 23, 45, 128
    left = rng.integers(0, 256, size=(n, H, W)).astype(np.uint8)
    dhat = np.where(rng.random((n, H, W)) < 0.2, rng.integers(0, D, size=(n, H, W)), -1).astype(np.int16)
    H4, W4 = (H + 3) // 4, (W + 3) // 4
    x = torch.empty((n, H4, W4, 32), dtype=torch.int16, device="cuda")
    S.sgmf_bn_input(n, W, H, D, _dev(left).data_ptr(), _dev(dhat).data_ptr(), x.data_ptr())
    gx = _from_bits(x.cpu().numpy().view(np.uint16))
    want = np.zeros((n, H4, W4, 32))
    for f in range(n):
        for qy in range(H4):
            for qx in range(W4):
                bl = left[f, 4 * qy:4 * qy + 4, 4 * qx:4 * qx + 4].astype(np.float64)
                bd = dhat[f, 4 * qy:4 * qy + 4, 4 * qx:4 * qx + 4]
                v = bd[bd >= 0]
                want[f, qy, qx, 0] = bl.mean() / 255.0 - 0.5
                want[f, qy, qx, 1] = v.mean() / D if v.size else 0.0
                want[f, qy, qx, 2] = v.size / 16.0
    np.testing.assert_allclose(gx, N.bf16_round(want), rtol=0, atol=2.0 ** -8)
    # labels from a disparity map
    disp = np.where(rng.random((n, H, W)) < 0.7, rng.integers(0, D, size=(n, H, W)), -1).astype(np.int16)
    lohi = torch.empty((n, H4, W4, 2), dtype=torch.int16, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.sgmf_bn_labels(n, W, H, _dev(disp).data_ptr(), lohi.data_ptr(), cnt.data_ptr())
    lh = lohi.cpu().numpy()
    nlab = 0
    for f in range(n):
        for qy in range(H4):
            for qx in range(W4):
                v = disp[f, 4 * qy:4 * qy + 4, 4 * qx:4 * qx + 4]
                v = v[v >= 0]
                exp = (v.min(), v.max()) if v.size else (-1, -1)
                nlab += bool(v.size)
                assert tuple(lh[f, qy, qx]) == exp
    assert int(cnt.item()) == nlab
    # loss and gradient
    out = rng.normal(size=(n, H4, W4, 32)).astype(np.float32)
    out[..., 0] = rng.uniform(0.05, 0.95, size=(n, H4, W4)).astype(np.float32)
    grad = torch.empty((n, H4, W4, 32), dtype=torch.int16, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    S.sgmf_bn_loss(n * H4 * W4, D, _dev(out).data_ptr(), lohi.data_ptr(), cnt.data_ptr(), grad.data_ptr(),
                   loss.data_ptr())
    valid = lh[..., 1] >= 0
    rl, rg = N.loss_and_grad(out.astype(np.float64), lh[..., 0].astype(np.float64), lh[..., 1].astype(np.float64),
                             valid, D)
    assert abs(float(loss.item()) - rl) <= 1e-4 * abs(rl)
    gg = _from_bits(grad.cpu().numpy().view(np.uint16))
    np.testing.assert_allclose(gg, N.bf16_round(rg), rtol=2.0 ** -7, atol=1e-9)
    # band starts per tile
    B, qmin = 64, 0.5
    T = S.BAND_TILE
    lo_t = torch.empty((n, (H + T - 1) // T, (W + T - 1) // T), dtype=torch.int16, device="cuda")
    unc = torch.zeros(n, dtype=torch.int32, device="cuda")           # one count per frame
    S.sgmf_bn_tiles(n, W, H, D, B, qmin, _dev(out).data_ptr(), lo_t.data_ptr(), unc.data_ptr())
    c, wv, q = N.heads(out.astype(np.float64), D)
    got = lo_t.cpu().numpy()
    nunc = np.zeros(n, np.int64)
    for f in range(n):
        for ty in range(got.shape[1]):
            for tx in range(got.shape[2]):
                Q = T // 4
                sl = (f, slice(Q * ty, Q * ty + Q), slice(Q * tx, Q * tx + Q))
                lo_u, hi_u = (c[sl] - wv[sl]).min(), (c[sl] + wv[sl]).max()
                mid = np.rint(0.5 * (lo_u + hi_u))
                assert abs(int(got[f, ty, tx]) - int(np.clip(mid - B // 2, 0, D - B))) <= 1
                nunc[f] += bool(q[sl].min() < qmin or hi_u - lo_u > B)
    assert np.abs(unc.cpu().numpy() - nunc).max() <= 1
    # the per-frame choice: value where the count is at most frac * tiles, else otherwise / kept
    tiles = got.shape[1] * got.shape[2]
    cnt_f = unc.cpu().numpy().astype(np.int64)
    gate = torch.full((n,), 9, dtype=torch.int32, device="cuda")
    for frac, value, other in ((0.5, 1, 2), (0.1, 0, -1)):
        S.sgmf_bn_decide(n, tiles, frac, unc.data_ptr(), value, other, gate.data_ptr())
    want = np.where(cnt_f <= int(0.1 * tiles), 0, np.where(cnt_f <= int(0.5 * tiles), 1, 2))
    np.testing.assert_array_equal(gate.cpu().numpy(), want)
    # Adam
    cnt_p = 1000
    wv0 = rng.normal(size=cnt_p).astype(np.float32)
    g = rng.normal(size=cnt_p).astype(np.float32)
    wd, md, vd = _dev(wv0.copy()), torch.zeros(cnt_p, device="cuda"), torch.zeros(cnt_p, device="cuda")
    wb = torch.empty(cnt_p, dtype=torch.int16, device="cuda")
    S.sgmf_bn_adam(cnt_p, wd.data_ptr(), md.data_ptr(), vd.data_ptr(), _dev(g).data_ptr(), 1e-2, 0.9, 0.999, 1e-8,
                   1, wb.data_ptr())
    m1 = 0.1 * g.astype(np.float64)
    v1 = 0.001 * g.astype(np.float64) ** 2
    want_w = wv0 - 1e-2 * (m1 / 0.1) / (np.sqrt(v1 / 0.001) + 1e-8)
    np.testing.assert_allclose(wd.cpu().numpy(), want_w, rtol=1e-5, atol=1e-6)
    np.testing.assert_array_equal(_from_bits(wb.cpu().numpy().view(np.uint16)),
                                  N.bf16_round(wd.cpu().numpy().astype(np.float64)))
