"""Pins of the CPU reference of the band-proposal network (float64), each
against something other than itself: a library correlation, adjoint
identities, central finite differences, hand values of bfloat16 rounding."""
import numpy as np
import pytest

from oracle import band_net as N


def test_bf16_rounding_hand_values():
    v = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, 1.0 + 2.0 ** -7 + 2.0 ** -8, -2.5, 0.0,
                  3.0e38])
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -6, -2.5, 0.0, 2.9993746e38])
    got = N.bf16_round(v)
    np.testing.assert_allclose(got[:6], want[:6], rtol=0, atol=0)
    assert abs(got[6] - 3.0e38) / 3.0e38 < 2 ** -8


def test_conv_matches_library_correlation():
    scipy_signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 7, 9, 4))
    w = rng.normal(size=(3, 3, 3, 4))
    b = rng.normal(size=3)
    y = N.conv3x3(x, w, b)
    for n in range(2):
        for co in range(3):
            ref = b[co] + sum(scipy_signal.correlate2d(x[n, :, :, ci], w[co, :, :, ci], mode="same")
                              for ci in range(4))
            np.testing.assert_allclose(y[n, :, :, co], ref, rtol=1e-12, atol=1e-12)


def test_dgrad_and_wgrad_are_adjoints():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 5, 6, 4))
    w = rng.normal(size=(3, 3, 3, 4))
    dy = rng.normal(size=(2, 5, 6, 3))
    y = N.conv3x3(x, w, None)
    lhs = float((y * dy).sum())
    assert abs(lhs - float((x * N.conv3x3_dgrad(dy, w)).sum())) < 1e-9 * max(1.0, abs(lhs))
    dw, db = N.conv3x3_wgrad(x, dy)
    assert abs(lhs - float((w * dw).sum())) < 1e-9 * max(1.0, abs(lhs))
    np.testing.assert_allclose(db, dy.sum(axis=(0, 1, 2)))


def _net(rng, cin=3):
    ws = [rng.normal(scale=0.3, size=(N.C, 3, 3, N.C)) for _ in range(N.LAYERS)]
    bs = [rng.normal(scale=0.1, size=N.C) for _ in range(N.LAYERS)]
    ws[0][:, :, :, cin:] = 0.0
    return ws, bs


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    ws, bs = _net(rng)
    x = np.zeros((1, 4, 5, N.C))
    x[..., :3] = rng.normal(size=(1, 4, 5, 3))
    gout = rng.normal(size=(1, 4, 5, N.C))
    acts, out = N.forward(x, ws, bs, round_acts=False)
    dws, dbs = N.backward(acts, ws, gout)
    f = lambda: float((N.forward(x, ws, bs, round_acts=False)[1] * gout).sum())
    h = 1e-6
    for l, (co, ky, kx, ci) in [(0, (5, 1, 2, 1)), (2, (7, 0, 0, 3)), (5, (2, 2, 1, 30)), (3, (31, 1, 1, 0))]:
        old = ws[l][co, ky, kx, ci]
        ws[l][co, ky, kx, ci] = old + h
        fp = f()
        ws[l][co, ky, kx, ci] = old - h
        fm = f()
        ws[l][co, ky, kx, ci] = old
        assert abs((fp - fm) / (2 * h) - dws[l][co, ky, kx, ci]) < 1e-5 * max(1.0, abs(dws[l][co, ky, kx, ci]))
    for l, co in [(1, 4), (5, 0)]:
        old = bs[l][co]
        bs[l][co] = old + h
        fp = f()
        bs[l][co] = old - h
        fm = f()
        bs[l][co] = old
        assert abs((fp - fm) / (2 * h) - dbs[l][co]) < 1e-5 * max(1.0, abs(dbs[l][co]))


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    D = 128
    out = rng.normal(size=(1, 3, 4, N.C))
    out[..., 0] = rng.uniform(0.1, 0.9, size=(1, 3, 4))
    lo = rng.integers(0, 100, size=(1, 3, 4)).astype(np.float64)
    hi = lo + rng.integers(0, 30, size=(1, 3, 4))
    valid = rng.random((1, 3, 4)) < 0.8
    loss, g = N.loss_and_grad(out, lo, hi, valid, D)
    h = 1e-7
    for idx in [(0, 0, 0, 0), (0, 1, 2, 1), (0, 2, 3, 2), (0, 1, 1, 0), (0, 0, 3, 2)]:
        o2 = out.copy()
        o2[idx] += h
        lp, _ = N.loss_and_grad(o2, lo, hi, valid, D)
        o2[idx] -= 2 * h
        lm, _ = N.loss_and_grad(o2, lo, hi, valid, D)
        assert abs((lp - lm) / (2 * h) - g[idx]) < 1e-5, idx
    # channels beyond the heads get no gradient
    assert (g[..., 3:] == 0).all()
