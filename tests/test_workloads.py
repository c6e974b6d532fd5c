"""The synthetic input recipes: shapes, value ranges, exit sets and seeds of
the named workloads (CPU only)."""
import numpy as np

from paper_1306_4743_gb300 import workloads as W


def test_point_source_const():
    p = W.point_source_const(65)
    assert p.F.shape == (65, 65, 65) and p.F.dtype == np.float32
    assert np.all(p.F == 1.0) and abs(p.h - 1.0 / 64) < 1e-15
    z, y, x = np.nonzero(p.mask)
    assert list(zip(x, y, z)) == [(32, 32, 32)] and p.q[32, 32, 32] == 0.0


def test_oscillatory_speed_and_source():
    p = W.oscillatory(33)
    assert p.F.min() >= 0.5 - 1e-6 and p.F.max() <= 1.5 + 1e-6
    z, y, x = np.nonzero(p.mask)
    assert list(zip(x, y, z)) == [(16, 16, 16)]
    # F = 1 + 0.5 sin(4 pi x) sin(4 pi y) sin(4 pi z) at a sample node
    h = p.h
    i, j, k = 3, 5, 7
    want = 1 + 0.5 * np.sin(4 * np.pi * i * h) * np.sin(4 * np.pi * j * h) * np.sin(4 * np.pi * k * h)
    assert abs(float(p.F[k, j, i]) - want) < 1e-6


def test_barrier_blocks():
    p = W.barrier_blocks(65)
    vals = np.unique(p.F)
    assert set(vals.tolist()) == {np.float32(0.01), np.float32(1.0)}
    # blocks of 1/16 of the cube, each slow with probability 0.3 (seeded)
    slow_share = float(np.mean(p.F == np.float32(0.01)))
    assert 0.15 < slow_share < 0.45
    assert int(p.mask.sum()) == 8 and np.all(p.F[p.mask == 1] == 1.0)
    q = W.barrier_blocks(65)
    assert np.array_equal(p.F, q.F) and np.array_equal(p.mask, q.mask)


def test_gaussian_bumps_range_and_seed():
    a = W.gaussian_bumps((33, 65, 17), 4001)
    b = W.gaussian_bumps((33, 65, 17), 4001)
    c = W.gaussian_bumps((33, 65, 17), 4002)
    assert a.F.shape == (17, 65, 33)
    assert a.F.min() >= 0.2 - 1e-7 and a.F.max() <= 2.0 + 1e-7
    assert int(a.mask.sum()) == 1
    assert abs(a.h - 1.0 / 64) < 1e-15  # 1 / (longest edge - 1)
    assert np.array_equal(a.F, b.F) and not np.array_equal(a.F, c.F)


def test_batch_dims():
    d = W.batch_dims(256)
    assert len(d) == 256
    assert all(e in (33, 65, 129) for t in d for e in t)
    assert d == W.batch_dims(256)
    # the three edges all occur on each axis
    for ax in range(3):
        assert {t[ax] for t in d} == {33, 65, 129}


def test_serving_requests():
    r = W.serving_requests(n=500, rate=100.0, seed=5)
    t = np.array([a for a, _, _ in r])
    e = np.array([b for _, b, _ in r])
    assert np.all(np.diff(t) > 0)
    assert 0.007 < float(np.mean(np.diff(t))) < 0.013  # mean gap 1 / rate
    assert e.min() >= 33 and e.max() <= 385
    # log-uniform: about half the edges below the geometric mean sqrt(33 * 385)
    assert 0.4 < float(np.mean(e < np.sqrt(33 * 385))) < 0.6
    assert [s for _, _, s in r[:3]] == [5000, 5001, 5002]
