"""Pins of the banded oracle (the method restricted to per-pixel disparity
bands, the form the learned band proposal drives; not part of the paper).

Each expectation comes from somewhere other than the banded code: the plain
method (full bands, or one constant band = the plain method on a slice of
the disparity axis), brute-force minimisation over all labelings that stay in
the bands, or hand cases.  CPU only.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2504_05148_gb300 import scenes


def test_full_band_is_the_plain_method():
    s = scenes.tiny(1700)
    lo = np.zeros(s.shape, np.int16)
    a = oracle.compute(s.left, s.right, s.lidar, s.D, volumes=True)
    for B in (s.D, s.D + 7):
        b = oracle.compute_banded(s.left, s.right, s.lidar, s.D, B, lo, volumes=True)
        np.testing.assert_array_equal(b.sum, a.sum)
        np.testing.assert_array_equal(b.dstar, a.dstar)
        np.testing.assert_array_equal(b.dprime, a.dprime)
        np.testing.assert_array_equal(b.out, a.out)


@pytest.mark.parametrize("a0,B", [(0, 16), (5, 20), (30, 34)])
def test_constant_band_is_the_plain_method_on_a_slice(a0, B):
    """One band [a, a+B) everywhere: S on the band equals the plain aggregate
    of the cost volume restricted to those disparities."""
    s = scenes.tiny(1701)
    r = oracle.compute(s.left, s.right, s.lidar, s.D, volumes=True)
    lo = np.full(s.shape, a0, np.int16)
    sv = oracle.aggregate_banded(r.cost, lo, B, 10, 120)
    want = oracle.aggregate(np.ascontiguousarray(r.cost[:, :, a0:a0 + B]), 10, 120)
    np.testing.assert_array_equal(sv[:, :, a0:a0 + B], want)
    assert (sv[:, :, :a0] == oracle.ABSENT).all() and (sv[:, :, a0 + B:] == oracle.ABSENT).all()
    ds, _ = oracle.wta_banded(sv, lo, B)
    np.testing.assert_array_equal(ds, a0 + np.argmin(want, axis=2))


def _brute_banded(C, bands, p1, p2):
    """min over labelings with label_i in bands[i] of the chain energy of
    Eq. 1 (P1 for a step of one disparity, P2 for a larger one), by final
    label: the unmodified energy, only the label sets are restricted."""
    n, D = C.shape
    best = np.full(D, np.inf)
    for lab in itertools.product(*[range(a, b) for a, b in bands]):
        e = sum(int(C[i, lab[i]]) for i in range(n))
        for i in range(1, n):
            dd = abs(lab[i] - lab[i - 1])
            e += p1 if dd == 1 else (p2 if dd > 1 else 0)
        best[lab[-1]] = min(best[lab[-1]], e)
    return best


@pytest.mark.parametrize("seed", range(8))
def test_banded_path_equals_brute_force(seed):
    rng = np.random.default_rng(400 + seed)
    n, D = int(rng.integers(2, 7)), int(rng.integers(3, 7))
    B = int(rng.integers(1, D))
    p1 = int(rng.integers(0, 12))
    p2 = int(rng.integers(p1, 40))
    cv = rng.integers(0, 41, size=(1, n, D)).astype(np.int32)
    lo = rng.integers(0, D - B + 1, size=(1, n)).astype(np.int16)
    L = oracle.path_banded(cv, lo, B, p1, p2, 1, 0)[0]
    acc = 0
    for j in range(n):
        bands = [(int(lo[0, i]), int(lo[0, i]) + B) for i in range(j + 1)]
        want = _brute_banded(cv[0, :j + 1], bands, p1, p2)
        a, b = bands[-1]
        np.testing.assert_array_equal(L[j, a:b] + acc, want[a:b])
        assert (L[j, :a] == oracle.ABSENT).all() and (L[j, b:] == oracle.ABSENT).all()
        acc += int(L[j, a:b].min())


def test_banded_right_view_search_hand_case():
    """d'(x') looks only at the cells (x'+d, d) inside the band of x'+d; with
    none it is invalid."""
    W, D, B = 6, 6, 2
    lo = np.array([[0, 0, 2, 2, 4, 4]], np.int16)
    S = np.full((1, W, D), oracle.ABSENT, np.int32)
    for x in range(W):
        S[0, x, lo[0, x]:lo[0, x] + B] = 50
    S[0, 3, 2] = 7          # x'=1, d=2
    S[0, 2, 2] = 9          # x'=0, d=2
    S[0, 4, 4] = 3          # x'=0, d=4: better than d=2
    ds, dp = oracle.wta_banded(S, lo, B)
    np.testing.assert_array_equal(ds, [[0, 0, 2, 2, 4, 4]])
    # x'=0: cells (0,0)=50 (1,1)=50 (2,2)=9 (3,3)=50 (4,4)=3 -> 4
    # x'=1: (1,0)=50 (3,2)=7 (4,3)=absent, (5,4)=50 -> 2
    # x'=5: (5,0) outside the band [4,6) of x=5 -> invalid
    assert dp[0, 0] == 4 and dp[0, 1] == 2 and dp[0, 5] == -1


def test_banded_right_view_search_none_inside():
    """Cells above a pixel's band never count: here no band holds a cell of the
    diagonal of x' = 0, so d'(0) is invalid."""
    lo = np.array([[1, 0, 0]], np.int16)
    S = np.full((1, 3, 3), oracle.ABSENT, np.int32)
    S[0, 0, 1] = 5
    S[0, 1, 0] = 5
    S[0, 2, 0] = 5
    _, dp = oracle.wta_banded(S, lo, 1)
    # x'=0: (0,0) below the band {1} of x=0, (1,1) and (2,2) above the bands {0}
    assert dp[0, 0] == -1
    assert dp[0, 1] == 0 and dp[0, 2] == 0


def test_banded_step_into_a_shifted_band_hand_case():
    """A neighbour disparity that lies in the previous pixel's band but below
    the current one still enters Eq. 2 with P1: the best chain into label 1
    of the second pixel comes from label 0 of the first (cost P1), a label
    the second pixel's band [1, 3) does not hold."""
    p1, p2 = 3, 20
    cv = np.array([[[0, 50, 50], [9, 4, 50]]], np.int32)
    lo = np.array([[0, 1]], np.int16)
    L = oracle.path_banded(cv, lo, 2, p1, p2, 1, 0)[0]
    # first pixel: band [0, 2), L = C
    assert L[0, 0] == 0 and L[0, 1] == 50 and L[0, 2] == oracle.ABSENT
    # second pixel, m = 0: d = 1: 4 + min(50, 0 + P1, 0 + P2) = 7;
    # d = 2: 50 + min(absent, 50 + P1, 0 + P2) = 70
    assert L[1, 0] == oracle.ABSENT and L[1, 1] == 4 + p1 and L[1, 2] == 50 + p2
    # the same by brute force over the two labelings of each final label
    want = _brute_banded(cv[0], [(0, 2), (1, 3)], p1, p2)
    assert want[1] == L[1, 1] and want[2] == L[1, 2]
