"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself or with the CUDA path: each
expected value comes from brute force over all labelings, a closed form, a
hand computation stored under tests/golden/, or an invariance the method must
have.  Runs on CPU only.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2504_05148_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(12345)


# ---------------------------------------------------------------------------
# LiDAR ingest (Sec. IV: d-bar is an integer disparity; reading: rint, half to even)

def test_lidar_rounding_and_validity():
    D = 8
    vals = np.array([[0.5, 1.5, 2.5, 3.5, 0.49999997, 0.0, -1.0, np.nan,
                      np.inf, -np.inf, 6.6, 7.4, 7.5, 8.0, 1e-30, 5.5]], np.float32)
    got = oracle.lidar(vals, D)
    want = np.array([[0, 2, 2, 4, 0, -1, -1, -1, -1, -1, 7, 7, -1, -1, 0, 6]], np.int16)
    np.testing.assert_array_equal(got, want)


def test_lidar_none_is_all_invalid():
    got = oracle.lidar(None, 16, shape=(3, 5))
    assert got.shape == (3, 5) and (got == -1).all()


# ---------------------------------------------------------------------------
# Census (Sec. IV-A).  Expected bit sets written out from the offset order:
# raster order over dy = -3..3 (outer), dx = -4..4 (inner), centre skipped.

def _bits(idx):
    v = 0
    for k in idx:
        v |= 1 << k
    return v


def test_census_constant_image_is_zero():
    img = np.full((20, 30), 77, np.uint8)
    for kind in (oracle.CENSUS_CS9X7, oracle.CENSUS_9X7):
        assert (oracle.census(img, kind) == 0).all()


def test_census_horizontal_ramp_closed_form():
    H, W = 15, 40
    img = np.tile(np.arange(W, dtype=np.uint8), (H, 1))          # I = x
    cs = oracle.census(img, oracle.CENSUS_CS9X7)
    full = oracle.census(img, oracle.CENSUS_9X7)
    # CS: bit set iff I(p+o) > I(p-o) iff dx > 0; among the 31 offsets before the
    # centre those are dx = 1..4 in rows dy = -3, -2, -1
    want_cs = _bits([5, 6, 7, 8, 14, 15, 16, 17, 23, 24, 25, 26])
    # full: I(p+o) > I(p) iff dx > 0, in all seven rows
    want_full = _bits([5, 6, 7, 8, 14, 15, 16, 17, 23, 24, 25, 26, 31, 32, 33, 34,
                       40, 41, 42, 43, 49, 50, 51, 52, 58, 59, 60, 61])
    inner = (slice(3, H - 3), slice(4, W - 4))
    assert (cs[inner] == want_cs).all()
    assert (full[inner] == want_full).all()


def test_census_vertical_ramp_closed_form():
    H, W = 20, 30
    img = np.tile(np.arange(H, dtype=np.uint8)[:, None], (1, W))  # I = y
    cs = oracle.census(img, oracle.CENSUS_CS9X7)
    full = oracle.census(img, oracle.CENSUS_9X7)
    inner = (slice(3, H - 3), slice(4, W - 4))
    # CS: I(p+o) > I(p-o) iff dy > 0, but every CS offset has dy <= 0
    assert (cs[inner] == 0).all()
    # full: dy > 0 are the last 27 offsets, bits 35..61
    assert (full[inner] == _bits(range(35, 62))).all()


def test_census_border_bits_are_zero():
    img = np.full((9, 11), 10, np.uint8)
    img[0, 0] = 5                                           # every neighbour is brighter
    full = oracle.census(img, oracle.CENSUS_9X7)
    # at (0,0) only offsets with dx >= 0 and dy >= 0 are inside: dy=0, dx=1..4 (bits
    # 31..34) and dy=1..3, dx=0..4 (bits 39..43, 48..52, 57..61)
    want = _bits(list(range(31, 35)) + list(range(39, 44)) + list(range(48, 53)) + list(range(57, 62)))
    assert int(full[0, 0]) == want
    # CS at (0,0): each pair needs p+o and p-o inside; p-o has -dx, -dy, so the
    # pair is inside only if dx = dy = 0 (the centre) -> no bit
    assert int(oracle.census(img, oracle.CENSUS_CS9X7)[0, 0]) == 0


def test_hamming_shift_and_left_border():
    H, W, D = 12, 40, 6
    left = RNG.integers(0, 256, size=(H, W), dtype=np.uint8)
    k = 3
    right = np.empty_like(left)
    right[:, :W - k] = left[:, k:]                          # right(x') = left(x' + k)
    right[:, W - k:] = RNG.integers(0, 256, size=(H, k), dtype=np.uint8)
    for kind in (oracle.CENSUS_CS9X7, oracle.CENSUS_9X7):
        nb = oracle.census_bits(kind)
        hv = oracle.hamming(oracle.census(left, kind), oracle.census(right, kind), D, nb)
        # closed form: windows coincide for 4 + k <= x <= W - 5 (rows clip alike)
        assert (hv[:, 4 + k:W - 4, k] == 0).all()
        # x - d < 0: the largest distance
        for d in range(D):
            assert (hv[:, :d, d] == nb).all()
        # elsewhere H is a popcount of census bits
        assert hv.min() >= 0 and hv.max() <= nb


# ---------------------------------------------------------------------------
# DDC, Eq. 4 (values worked by hand in tests/golden/ddc_values.txt)

def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "ddc_values.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_ddc_golden_values():
    rows = _golden_rows()
    assert len(rows) >= 5
    for h, a, b, q1, q2, cls, real, integer in rows:
        h, a, b, q1, q2, cls = map(int, (h, a, b, q1, q2, cls))
        D = 8
        prior = np.array([[3]], np.int16)
        d = {0: 3, 1: 4, 2: 6}[cls]
        hv = np.full((1, 1, D), h, np.int32)
        cv = oracle.ddc(hv, prior, q1, q2, a, b)
        assert int(cv[0, 0, d]) == int(integer)
        assert abs(cv[0, 0, d] - float(real)) <= 0.5


def test_ddc_rounding_bound_and_no_prior():
    D = 7
    for a, b in [(7, 10), (1, 3), (0, 5), (5, 5), (3, 8)]:
        for q1, q2 in [(5, 160), (0, 0), (9, 9), (1, 200)]:
            hv = np.tile(np.arange(63, dtype=np.int32)[:, None, None], (1, 1, D))  # H = 0..62
            prior = np.full((63, 1), 3, np.int16)
            cv = oracle.ddc(hv, prior, q1, q2, a, b)
            alpha = a / b
            for d in range(D):
                q = 0 if d == 3 else (q1 if abs(d - 3) == 1 else q2)
                real = (1 - alpha) * hv[:, 0, d] + alpha * q
                assert np.all(np.abs(cv[:, 0, d] - real) <= 0.5 + 1e-9)
            # invalid prior: no DDC, C-bar = H
            cv2 = oracle.ddc(hv, np.full((63, 1), -1, np.int16), q1, q2, a, b)
            np.testing.assert_array_equal(cv2, hv)


# ---------------------------------------------------------------------------
# Eq. 2 against brute-force minimisation of the chain energy of Eq. 1

def _brute_chain(C, p1, p2):
    """min over all labelings of sum C + P1 [|dd|=1] + P2 [|dd|>1], by final label."""
    n, D = C.shape
    best = np.full(D, np.inf)
    for lab in itertools.product(range(D), repeat=n):
        e = sum(int(C[i, lab[i]]) for i in range(n))
        for i in range(1, n):
            dd = abs(lab[i] - lab[i - 1])
            e += p1 if dd == 1 else (p2 if dd > 1 else 0)
        best[lab[-1]] = min(best[lab[-1]], e)
    return best


def _check_chain(Lchain, Cchain, p1, p2):
    """L(p_j, d) + sum_{k<j} m_k equals the brute-force chain minimum at every j."""
    acc = 0
    for j in range(len(Cchain)):
        want = _brute_chain(Cchain[:j + 1], p1, p2)
        np.testing.assert_array_equal(Lchain[j] + acc, want)
        acc += int(Lchain[j].min())


@pytest.mark.parametrize("seed", range(6))
def test_path_horizontal_equals_brute_force(seed):
    rng = np.random.default_rng(seed)
    n, D = int(rng.integers(2, 7)), int(rng.integers(2, 5))
    p1 = int(rng.integers(0, 15))
    p2 = int(rng.integers(p1, 40))
    cv = rng.integers(0, 41, size=(1, n, D)).astype(np.int32)
    Lr = oracle.path(cv, p1, p2, 1, 0)
    _check_chain(Lr[0], cv[0], p1, p2)
    Ll = oracle.path(cv, p1, p2, -1, 0)
    _check_chain(Ll[0, ::-1], cv[0, ::-1], p1, p2)


@pytest.mark.parametrize("seed", range(4))
def test_path_vertical_equals_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    n, D = int(rng.integers(2, 7)), int(rng.integers(2, 5))
    p1 = int(rng.integers(0, 15))
    p2 = int(rng.integers(p1, 40))
    cv = rng.integers(0, 41, size=(n, 1, D)).astype(np.int32)
    Ld = oracle.path(cv, p1, p2, 0, 1)
    _check_chain(Ld[:, 0], cv[:, 0], p1, p2)
    Lu = oracle.path(cv, p1, p2, 0, -1)
    _check_chain(Lu[::-1, 0], cv[::-1, 0], p1, p2)


@pytest.mark.parametrize("r", [(1, 1), (-1, -1), (1, -1), (-1, 1)])
def test_path_diagonals_equal_brute_force(r):
    rng = np.random.default_rng(7)
    H, W, D = 4, 5, 3
    p1, p2 = 4, 11
    cv = rng.integers(0, 30, size=(H, W, D)).astype(np.int32)
    L = oracle.path(cv, p1, p2, r[0], r[1])
    rx, ry = r
    # every pixel whose predecessor p - r is outside the image starts a chain
    for y in range(H):
        for x in range(W):
            if 0 <= x - rx < W and 0 <= y - ry < H:
                continue
            chain = []
            cx, cy = x, y
            while 0 <= cx < W and 0 <= cy < H:
                chain.append((cy, cx))
                cx, cy = cx + rx, cy + ry
            Cc = np.array([cv[a, b] for a, b in chain])
            Lc = np.array([L[a, b] for a, b in chain])
            _check_chain(Lc, Cc, p1, p2)


def test_single_row_sum_closed_form():
    """On a 1-row image the vertical and diagonal paths have length 1, so
    S = 6 C + L_right + L_left (8 paths) and S = 2 C + L_right + L_left (4 paths)."""
    rng = np.random.default_rng(3)
    W, D = 9, 6
    cv = rng.integers(0, 60, size=(1, W, D)).astype(np.int32)
    Lr = oracle.path(cv, 10, 120, 1, 0)
    Ll = oracle.path(cv, 10, 120, -1, 0)
    np.testing.assert_array_equal(oracle.aggregate(cv, 10, 120, 8), 6 * cv + Lr + Ll)
    np.testing.assert_array_equal(oracle.aggregate(cv, 10, 120, 4), 2 * cv + Lr + Ll)


def test_path_costs_bounded():
    """min{...} - m lies in [0, P2], so C <= L <= C + P2 (the uint8 bound of the GPU path)."""
    rng = np.random.default_rng(9)
    cv = rng.integers(0, 132, size=(6, 7, 9)).astype(np.int32)
    for rx, ry in oracle.DIRECTIONS:
        L = oracle.path(cv, 10, 120, rx, ry)
        assert (L >= cv).all() and (L <= cv + 120).all()


# ---------------------------------------------------------------------------
# WTA (Eq. 3) and the right-view diagonal search

def test_wta_argmin_ties_and_right_view():
    S = np.array([[[5, 3, 3, 9], [1, 1, 0, 4], [7, 2, 8, 2]]], np.int32)   # H=1, W=3, D=4
    ds, dp = oracle.wta(S)
    np.testing.assert_array_equal(ds, [[1, 2, 1]])
    # d'(x') = argmin_{d: x'+d < W} S(x'+d, d)
    # x'=0: S(0,0)=5, S(1,1)=1, S(2,2)=8 -> 1;  x'=1: S(1,0)=1, S(2,1)=2 -> 0;  x'=2: S(2,0)=7 -> 0
    np.testing.assert_array_equal(dp, [[1, 0, 0]])


def test_right_view_diagonal_closed_form():
    """Cell (x, d) of the left-based aggregate belongs to the right pixel
    x' = x - d.  Mark one cell per right pixel: d'(x') must return its d."""
    W, D = 11, 5
    rng = np.random.default_rng(17)
    S = np.full((2, W, D), 50, np.int32)
    target = np.zeros((2, W), int)
    for y in range(2):
        for xr in range(W):
            t = int(rng.integers(0, min(D, W - xr)))      # x' + t < W
            target[y, xr] = t
            S[y, xr + t, t] = 1
    _, dp = oracle.wta(S)
    np.testing.assert_array_equal(dp, target)


# ---------------------------------------------------------------------------
# Sub-pixel parabola fit (Sec. III, after Eq. 3); results in 1/16 px

def test_subpixel_recovers_the_vertex_of_a_sampled_parabola():
    """S sampled from a (16 d - V)^2 + c: the parabola through three samples is
    that parabola, so its vertex V / 16 comes back exactly, also when V / 16 is
    a half-integer (then d* and d* + 1 tie and d* is the smaller)."""
    rng = np.random.default_rng(31)
    W, D = 300, 24
    d = np.arange(D)
    V = rng.integers(24, 16 * (D - 2) + 1, size=W)
    a = rng.integers(1, 4, size=W)
    c = rng.integers(0, 50, size=W)
    S = (a[:, None] * (16 * d[None, :] - V[:, None]) ** 2 + c[:, None]).astype(np.int32)[None]
    ds, _ = oracle.wta(S)
    assert ((ds >= 1) & (ds <= D - 2)).all()
    np.testing.assert_array_equal(oracle.subpixel(S, ds)[0], V)


def test_subpixel_hand_values():
    # (S(d*-1), S(d*), S(d*+1)) -> offset 16 (S- - S+) / (2 (S- - 2 S* + S+)), rounded half up
    cases = [((5, 3, 3), 8),        # tie with d* + 1: the vertex is half-way
             ((17, 0, 15), 1),      # 32 / 64 = 0.5 sixteenths -> 1
             ((15, 0, 17), 0),      # -0.5 -> 0
             ((9, 1, 9), 0),        # symmetric
             ((40, 0, 8), 5),       # 16 * 32 / 96 = 5.33 -> 5
             ((8, 0, 40), -5),      # -5.33 -> -5
             ((2, 0, 200), -8)]     # 16 * -198 / 404 = -7.84 -> -8
    for (sm, s0, sp), want in cases:
        S = np.array([[[999, sm, s0, sp, 999]]], np.int32)
        ds, _ = oracle.wta(S)
        assert ds[0, 0] == 2
        assert oracle.subpixel(S, ds)[0, 0] == 32 + want, (sm, s0, sp)


def test_subpixel_at_the_ends_of_the_range_is_integer():
    S = np.array([[[0, 5, 9, 9], [9, 9, 5, 1], [4, 4, 4, 4]]], np.int32)
    ds, _ = oracle.wta(S)
    np.testing.assert_array_equal(ds, [[0, 3, 0]])
    np.testing.assert_array_equal(oracle.subpixel(S, ds), [[0, 48, 0]])


def test_subpixel_mirror_and_bounds():
    """Reversing the disparity axis mirrors the vertex: the two results add up
    to 16 (D - 1), plus 1 where the offset is an exact half (rounded up both
    times); every offset lies within half a pixel of d*."""
    rng = np.random.default_rng(32)
    H, W, D = 3, 200, 16
    S = rng.permutation(H * W * D).reshape(H, W, D).astype(np.int32)   # distinct values: no ties
    ds, _ = oracle.wta(S)
    got = oracle.subpixel(S, ds).astype(int)
    R = np.ascontiguousarray(S[:, :, ::-1])
    dr, _ = oracle.wta(R)
    np.testing.assert_array_equal(dr, D - 1 - ds)
    rev = oracle.subpixel(R, dr).astype(int)
    tot = got + rev - 16 * (D - 1)
    assert set(np.unique(tot)) <= {0, 1}
    inner = (ds > 0) & (ds < D - 1)
    assert (np.abs(got - 16 * ds.astype(int))[inner] <= 8).all()
    assert (got[~inner] == 16 * ds[~inner]).all()


def test_subpixel_pipeline_keeps_the_integer_check():
    """With the fit switched on, the check (on integer d*) keeps the same
    pixels, and each kept value lies within half a pixel of d*."""
    s = scenes.tiny(1400)
    r0 = oracle.compute(s.left, s.right, s.lidar, s.D, dumps=False)
    r1 = oracle.compute(s.left, s.right, s.lidar, s.D, oracle.Params(subpixel=1), dumps=False)
    np.testing.assert_array_equal(r1.out < 0, r0.out < 0)
    v = r0.out >= 0
    assert (np.abs(r1.out[v].astype(int) - 16 * r0.out[v].astype(int)) <= 8).all()
    assert (r1.out[v] != 16 * r0.out[v]).mean() > 0.5


# ---------------------------------------------------------------------------
# Semidensification (Eq. 5) hand cases

def test_semidense_hand_cases():
    H, W, D = 7, 7, 8
    dbar = np.full((H, W), -1, np.int16)
    dbar[3, 3] = 5
    hv = np.full((H, W, D), 9, np.int32)
    hv[3, 5, 5] = 0        # neighbour (3,5) matches disparity 5 perfectly
    hv[0, 0, 5] = 1
    # T_s = 2, r_s = 2: (3,5) sees q=(3,3) -> H=0 < 2 -> d-hat = 5
    dh = oracle.semidense(dbar, hv, 2, 2)
    assert dh[3, 5] == 5
    # (0,0) is outside the 5x5 window of (3,3): no candidate -> stays invalid
    assert dh[0, 0] == -1
    # (3,3) itself: H(p,5) = 9 >= T_s -> falls back to d-bar = 5
    assert dh[3, 3] == 5
    # everywhere else in the window the cost 9 is not below T_s -> d-bar (invalid)
    assert dh[1, 1] == -1
    # T_s = 0 or r_s = 0 leave d-bar unchanged
    np.testing.assert_array_equal(oracle.semidense(dbar, hv, 0, 2), dbar)
    np.testing.assert_array_equal(oracle.semidense(dbar, hv, 100, 0), dbar)
    # ties in H go to the smaller disparity; a valid d-bar_p can be replaced
    dbar2 = np.full((H, W), -1, np.int16)
    dbar2[2, 2], dbar2[2, 4], dbar2[3, 3] = 6, 2, 4
    hv2 = np.full((H, W, D), 9, np.int32)
    hv2[3, 3, 6] = 1
    hv2[3, 3, 2] = 1
    dh2 = oracle.semidense(dbar2, hv2, 2, 1)
    assert dh2[3, 3] == 2


def test_semidense_ts_zero_is_dsgm():
    s = scenes.tiny()
    p0 = oracle.Params(ts=0)
    pd = oracle.Params(semidense=0)
    a = oracle.compute(s.left, s.right, s.lidar, s.D, p0)
    b = oracle.compute(s.left, s.right, s.lidar, s.D, pd)
    np.testing.assert_array_equal(a.dhat, a.dbar)
    np.testing.assert_array_equal(a.out, b.out)


# ---------------------------------------------------------------------------
# Consistency check (Eq. 6)

def test_consistency_window_extent_and_threshold():
    H, W, D = 50, 60, 32
    dbar = np.full((H, W), -1, np.int16)
    dbar[20, 30] = 10
    rc, tc = 5, 2
    dp = np.full((H, W), 0, np.int16)                  # stereo term fails (d* = 10 vs 0)
    for dstar_val, ok_expected in [(10, True), (12, True), (8, True), (13, False), (7, False)]:
        ds = np.full((H, W), dstar_val, np.int16)
        out = oracle.consistency(ds, dp, dbar, tc, rc, 1, oracle.CHECK_LIDAR)
        ys, xs = np.mgrid[0:H, 0:W]
        inside = (np.abs(ys - 20) <= rc) & (np.abs(xs - 30) <= rc)
        want = np.where(inside & ok_expected, dstar_val, -1)
        np.testing.assert_array_equal(out, want)


def test_consistency_stereo_term_and_modes():
    H, W, D = 4, 20, 8
    k = 3
    ds = np.full((H, W), k, np.int16)
    dp = np.full((H, W), k, np.int16)
    dbar = np.full((H, W), -1, np.int16)
    st = oracle.consistency(ds, dp, dbar, 2, 3, 1, oracle.CHECK_STEREO)
    # q_m = (x - k, y) exists only for x >= k
    want = np.where(np.arange(W)[None, :] >= k, k, -1) * np.ones((H, 1), int)
    np.testing.assert_array_equal(st, want)
    # without LiDAR in any window, stereo-LiDAR = stereo
    np.testing.assert_array_equal(oracle.consistency(ds, dp, dbar, 2, 3, 1, oracle.CHECK_STEREO_LIDAR), st)
    # |d* - d'| <= 1 passes, 2 fails
    dp2 = dp.copy()
    dp2[:, :5] = k + 1
    dp2[:, 5:] = k + 2
    st2 = oracle.consistency(ds, dp2, dbar, 2, 3, 1, oracle.CHECK_STEREO)
    xm = np.arange(W) - k
    want2 = np.where((xm >= 0) & (xm < 5), k, -1) * np.ones((H, 1), int)
    np.testing.assert_array_equal(st2, want2)
    # no check
    np.testing.assert_array_equal(oracle.consistency(ds, dp2, dbar, 2, 3, 1, oracle.CHECK_NONE), ds)
    # T_c >= D: any LiDAR return in the window passes
    dbar[0, 0] = 0
    li = oracle.consistency(np.full((H, W), D - 1, np.int16), dp2, dbar, D, 3, 1, oracle.CHECK_LIDAR)
    ys, xs = np.mgrid[0:H, 0:W]
    np.testing.assert_array_equal(li >= 0, (ys <= 3) & (xs <= 3))


def test_consistency_predicate_symmetry():
    """|a - b| <= t is symmetric: swapping d* and the LiDAR value keeps the decision."""
    H, W = 5, 5
    rng = np.random.default_rng(4)
    for _ in range(20):
        a, b = int(rng.integers(0, 30)), int(rng.integers(0, 30))
        t = int(rng.integers(0, 5))
        dbar = np.full((H, W), -1, np.int16)
        dbar[2, 2] = b
        o1 = oracle.consistency(np.full((H, W), a, np.int16), np.zeros((H, W), np.int16), dbar, t, 1, 1,
                                oracle.CHECK_LIDAR)
        dbar[2, 2] = a
        o2 = oracle.consistency(np.full((H, W), b, np.int16), np.zeros((H, W), np.int16), dbar, t, 1, 1,
                                oracle.CHECK_LIDAR)
        assert (o1[2, 2] >= 0) == (o2[2, 2] >= 0) == (abs(a - b) <= t)


def _right_view_check(dstar, dprime, lr):
    """The stereo condition of Eq. 6 seen from the right view, by direct
    loops: right pixel x' keeps d'(x') when its match x' + d'(x') lies in
    the image and |d'(x') - d*(x' + d'(x'))| <= lr."""
    H, W = dstar.shape
    out = np.full((H, W), -1, np.int16)
    for y in range(H):
        for xr in range(W):
            d = int(dprime[y, xr])
            x = xr + d
            if 0 <= d and x < W and abs(d - int(dstar[y, x])) <= lr:
                out[y, xr] = d
    return out


def _consistent_maps(rng, H, W, D, jitter):
    """A left map d* of slanted planes (slope in [0, 1/2), no occlusion) and
    the right map d' it induces (x' = x - d*(x)), plus optional random
    jitter of d' in [-jitter, jitter]."""
    ds = np.zeros((H, W), np.int16)
    dp = np.zeros((H, W), np.int16)
    for y in range(H):
        a, b = rng.uniform(1, D // 2), rng.uniform(0.0, 0.49)
        row = np.minimum(np.rint(a + b * np.arange(W)), D - 1).astype(np.int64)
        ds[y] = row
        dp[y] = row[-1] if W else 0
        for x in range(W - 1, -1, -1):       # the leftmost x of each x' wins, as any would
            if x - row[x] >= 0:
                dp[y, x - row[x]] = row[x]
        if jitter:
            dp[y] = np.clip(dp[y] + rng.integers(-jitter, jitter + 1, size=W), 0, D - 1)
    return ds, dp


@pytest.mark.parametrize("lr", [0, 1, 2])
def test_consistency_mirror_identity(lr):
    """P-6(ii): the L-R check of Eq. 6 run with the views swapped and
    mirrored horizontally (the right map as d*, the left map as d', both
    mirrored) equals the check from the right view, mirrored back.  The
    maps are near-consistent (d' jittered by up to 2), so that a lookup of
    d' one pixel off q_m = (x - d*, y) changes many decisions."""
    rng = np.random.default_rng(60 + lr)
    for _ in range(6):
        H, W, D = int(rng.integers(1, 6)), int(rng.integers(8, 60)), int(rng.integers(4, 40))
        ds, dp = _consistent_maps(rng, H, W, D, 2)
        none = np.full((H, W), -1, np.int16)
        swapped = oracle.consistency(dp[:, ::-1], ds[:, ::-1], none, 2, 20, lr, oracle.CHECK_STEREO)
        np.testing.assert_array_equal(swapped[:, ::-1], _right_view_check(ds, dp, lr))


def test_consistency_passes_everywhere_on_consistent_maps():
    """P-6(ii): on occlusion-free, mutually consistent maps the L-R check
    keeps every pixel whose match lies in the image, and so does the check
    from the right view (for every right pixel that some left pixel maps to)."""
    rng = np.random.default_rng(66)
    for _ in range(6):
        H, W, D = 4, int(rng.integers(16, 80)), int(rng.integers(4, 40))
        ds, dp = _consistent_maps(rng, H, W, D, 0)
        none = np.full((H, W), -1, np.int16)
        out = oracle.consistency(ds, dp, none, 2, 20, 1, oracle.CHECK_STEREO)
        xs = np.arange(W)[None, :]
        inside = xs - ds >= 0
        np.testing.assert_array_equal(out[inside], ds[inside])
        assert (out[~inside] == -1).all()
        rv = _right_view_check(ds, dp, 1)
        hit = np.zeros((H, W), bool)
        for y in range(H):
            for x in range(W):
                if x - ds[y, x] >= 0:
                    hit[y, x - ds[y, x]] = True
        np.testing.assert_array_equal(rv[hit], dp[hit])


def test_consistency_uses_raw_sparse_map():
    s = scenes.tiny()
    r = oracle.compute(s.left, s.right, s.lidar, s.D)
    p = oracle.Params()
    want = oracle.consistency(r.dstar, r.dprime, r.dbar, p.tc, p.rc, p.lr_max_diff, oracle.CHECK_STEREO_LIDAR)
    np.testing.assert_array_equal(r.out, want)
    alt = oracle.consistency(r.dstar, r.dprime, r.dhat, p.tc, p.rc, p.lr_max_diff, oracle.CHECK_STEREO_LIDAR)
    assert (alt != r.out).any()          # the choice of map matters on this scene


# ---------------------------------------------------------------------------
# Whole-pipeline invariants

def test_no_lidar_reduces_to_census_sgm():
    s = scenes.random_small(5, 48, 24, 16)
    a = oracle.compute(s.left, s.right, None, s.D, volumes=True)
    z = oracle.compute(s.left, s.right, np.zeros_like(s.lidar), s.D, volumes=True)
    assert (a.dbar == -1).all() and (a.dhat == -1).all()
    nb = oracle.census_bits(oracle.CENSUS_CS9X7)
    hv = oracle.hamming(a.census_l, a.census_r, s.D, nb)
    np.testing.assert_array_equal(a.cost, hv)                      # C-bar = H
    for f in ("out", "dstar", "dprime", "cost", "sum"):
        np.testing.assert_array_equal(getattr(a, f), getattr(z, f))
    # the output is the stereo-only check of plain census SGM
    st = oracle.consistency(a.dstar, a.dprime, a.dbar, 2, 20, 1, oracle.CHECK_STEREO)
    np.testing.assert_array_equal(a.out, st)
    # alpha = 0 with LiDAR present also leaves C-bar = H
    b = oracle.compute(s.left, s.right, s.lidar, s.D, oracle.Params(alpha_num=0), volumes=True)
    np.testing.assert_array_equal(b.cost, hv)


def _numpy_sgm_reference(C, p1, p2, dirs):
    """Independent vectorised statement of Eq. 2: each direction is swept as a
    whole front (row, column or anti-diagonal band) at once."""
    H, W, D = C.shape
    S = np.zeros_like(C, dtype=np.int64)
    for rx, ry in dirs:
        L = np.zeros_like(C, dtype=np.int64)
        ys = range(H) if ry >= 0 else range(H - 1, -1, -1)
        xs = range(W) if rx >= 0 else range(W - 1, -1, -1)
        if ry == 0:
            order = [(None, x) for x in xs]
        else:
            order = [(y, None) for y in ys]
        for y, x in order:
            if ry == 0:
                cur = (slice(None), x)
                px = x - rx
                if not 0 <= px < W:
                    L[cur] = C[cur]
                    continue
                prev = L[:, px]
                c = C[:, x]
                m = prev.min(axis=1, keepdims=True)
                up = np.concatenate([prev[:, 1:], np.full((H, 1), np.iinfo(np.int64).max // 4)], 1)
                dn = np.concatenate([np.full((H, 1), np.iinfo(np.int64).max // 4), prev[:, :-1]], 1)
                L[:, x] = c + np.minimum.reduce([prev, up + p1, dn + p1, np.broadcast_to(m + p2, prev.shape)]) - m
            else:
                py = y - ry
                if not 0 <= py < H:
                    L[y] = C[y]
                    continue
                big = np.iinfo(np.int64).max // 4
                prev = np.full((W, D), big)
                src = np.arange(W) - rx
                ok = (src >= 0) & (src < W)
                prev[ok] = L[py, src[ok]]
                c = C[y]
                m = prev.min(axis=1, keepdims=True)
                up = np.concatenate([prev[:, 1:], np.full((W, 1), big)], 1)
                dn = np.concatenate([np.full((W, 1), big), prev[:, :-1]], 1)
                new = c + np.minimum.reduce([prev, up + p1, dn + p1, np.broadcast_to(m + p2, prev.shape)]) - m
                L[y] = np.where(ok[:, None], new, c)
        S += L
    return S


def test_aggregate_matches_independent_vectorised_sweep():
    rng = np.random.default_rng(21)
    C = rng.integers(0, 132, size=(13, 17, 9)).astype(np.int32)
    S = oracle.aggregate(C, 10, 120, 8)
    np.testing.assert_array_equal(S, _numpy_sgm_reference(C, 10, 120, oracle.DIRECTIONS))


def test_monotone_intensity_map_invariance():
    s = scenes.tiny(1001)
    left, right = s.left // 2, s.right // 2                 # values 0..127
    lut = np.sort(RNG.choice(256, size=128, replace=False)).astype(np.uint8)   # strictly increasing
    a = oracle.compute(left, right, s.lidar, s.D)
    b = oracle.compute(lut[left], lut[right], s.lidar, s.D)
    for f in ("census_l", "census_r", "dhat", "dstar", "dprime", "out"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))


def _plane_pair(H, W, k, seed):
    rng = np.random.default_rng(seed)
    left = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    right = np.empty_like(left)
    right[:, :W - k] = left[:, k:]
    right[:, W - k:] = rng.integers(0, 256, size=(H, k))
    return left, right


def test_exact_recovery_of_fronto_parallel_plane():
    H, W, D, k = 40, 120, 32, 9
    left, right = _plane_pair(H, W, k, 5)
    lid = np.zeros((H, W), np.float32)
    lid[::7, ::5] = k
    for li in (None, lid):
        r = oracle.compute(left, right, li, D, volumes=True)
        # H(p, k) = 0 wherever both 9x7 windows coincide: 4 + k <= x <= W - 5
        assert (r.cost[:, 4 + k:W - 4, k] == 0).all()
        # the truth wins well inside that band
        assert (r.dstar[:, 4 + k + 4:W - 4 - 4] == k).all()


def test_exact_recovery_two_planes():
    """Two fronto-parallel planes side by side (left half k1, right half k2 > k1)."""
    H, W, D, k1, k2 = 30, 160, 32, 4, 12
    rng = np.random.default_rng(8)
    left = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    split = 80
    right = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    # right pixel x' sees the left half at x = x' + k1 and the right half at x = x' + k2;
    # the front plane (k2) wins where both land
    for xr in range(W):
        xa, xb = xr + k1, xr + k2
        if xb < W and xb >= split:
            right[:, xr] = left[:, xb]
        elif xa < split:
            right[:, xr] = left[:, xa]
    r = oracle.compute(left, right, None, D)
    assert (r.dstar[:, 4 + k1 + 4:split - 4 - 8] == k1).all()
    assert (r.dstar[:, split + 8:W - 8] == k2).all()


@pytest.mark.slow
def test_lidar_improves_total_error_on_street_scene():
    """Sanity (not parity): counting invalid pixels as errors (>= 3 px,
    Sec. V-B), SDSGM beats stereo-only SGM on the KITTI-shaped scene."""
    s = scenes.kitti()
    err = {}
    for name, li in (("sdsgm", s.lidar), ("sgm", None)):
        r = oracle.compute(s.left, s.right, li, s.D, dumps=False)
        bad = (r.out < 0) | (np.abs(r.out.astype(np.float64) - s.truth) >= 3)
        err[name] = bad.mean()
    assert err["sdsgm"] < err["sgm"]
