"""Seeded input generators: determinism, shapes and value ranges."""
import numpy as np
import pytest

from paper_2504_05148_gb300 import scenes


def test_tiny_is_deterministic_and_shaped():
    a, b = scenes.tiny(1000), scenes.tiny(1000)
    for f in ("left", "right", "lidar", "truth"):
        np.testing.assert_array_equal(getattr(a, f), getattr(b, f))
    assert a.left.shape == (128, 256) and a.left.dtype == np.uint8 and a.D == 64
    assert a.lidar.dtype == np.float32
    assert not np.array_equal(scenes.tiny(1001).left, a.left)
    # LiDAR on 16 rows, every 4th column (2 % outliers may land on 0 = no return)
    rows = np.flatnonzero((a.lidar > 0).any(axis=1))
    assert len(rows) == 16
    assert ((a.lidar > 0)[:, 1::4] == 0).all()
    assert 4.0 <= a.truth.min() and a.truth.max() <= 60.0


def test_kitti_density_and_beams():
    s = scenes.kitti(2000)
    assert s.left.shape == (375, 1242) and s.D == 128
    dens = (s.lidar > 0).mean()
    assert 0.04 < dens < 0.06                  # about 5 %
    rows = np.flatnonzero((s.lidar > 0).any(axis=1))
    assert len(rows) == 64 and rows.min() >= int(0.4 * 375) - 1
    s16 = scenes.kitti(2000, beams=16)
    assert len(np.flatnonzero((s16.lidar > 0).any(axis=1))) == 16
    assert s.truth.max() <= 127


@pytest.mark.parametrize("W,H,D", [(1, 1, 1), (5, 3, 4), (9, 7, 16), (33, 17, 37), (70, 9, 64)])
def test_random_small_shapes(W, H, D):
    s = scenes.random_small(7, W, H, D)
    assert s.left.shape == (H, W) and s.right.shape == (H, W) and s.lidar.shape == (H, W)
    assert s.D == D


def test_named_workloads():
    assert scenes.by_name("indoor").left.shape == (480, 640)
    s = scenes.by_name("lowlight")
    assert s.left.shape == (720, 1280) and s.D == 192 and s.left.max() <= 40


def test_poisson_schedule_rate_and_determinism():
    from paper_2504_05148_gb300 import serving
    a = serving.poisson_schedule(25.0, 200.0, 3)
    b = serving.poisson_schedule(25.0, 200.0, 3)
    np.testing.assert_array_equal(a, b)
    assert abs(len(a) / 200.0 - 25.0) < 1.5                  # mean rate (5000 arrivals)
    gaps = np.diff(a)
    assert (gaps > 0).all()
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1         # exponential: coefficient of variation 1
    assert a.max() < 200.0


def test_mixed_batch_shapes():
    from paper_2504_05148_gb300 import scenes as sc
    s = sc.mixed(4000, 64, 32, 16)
    assert s.shape == (32, 64) and s.D == 16
    assert (s.lidar >= 0).all() and np.isfinite(s.lidar).all()
    assert sc.MIXED_SHAPES == ((640, 480, 64), (1242, 375, 128), (1280, 720, 192), (1920, 1080, 256))
