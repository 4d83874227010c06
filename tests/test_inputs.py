"""Checks of the seeded input generators (CPU)."""
import numpy as np
import pytest

from paper_1805_10167_gb300 import inputs


def _splitmix64_int(x):
    """SplitMix64 output function on Python integers (Vigna 2015)."""
    m = (1 << 64) - 1
    z = (x + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def test_splitmix64_matches_integer_definition():
    xs = np.array([0, 1, 2, 1234, 2 ** 63 + 5, 2 ** 64 - 1], dtype=np.uint64)
    got = inputs.splitmix64(xs)
    for x, g in zip(xs.tolist(), got.tolist()):
        assert g == _splitmix64_int(int(x))
    # first output of a SplitMix64 stream seeded with 0
    assert _splitmix64_int(0) == 0xE220A8397B1DCDAF


def test_uniform_range_and_moments():
    u = inputs.uniform_pm1(1 << 20, 1234)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert abs(u.mean()) < 5e-3 and abs(u.var() - 1 / 3) < 5e-3


@pytest.mark.parametrize("maker", [inputs.unit_square_mesh, lambda: inputs.annulus_mesh(32, 2),
                                   lambda: inputs.random_square_mesh(3, 40)])
def test_meshes_ccw_and_conforming(maker):
    xy, tri = maker()
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    cross = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    assert np.all(cross > 0)
    cnt = {}
    for t in tri:
        for s in range(3):
            e = tuple(sorted((int(t[s]), int(t[(s + 1) % 3]))))
            cnt[e] = cnt.get(e, 0) + 1
    assert max(cnt.values()) <= 2
    # Euler characteristic of a disk (1) or an annulus (0)
    V, E, F = xy.shape[0], len(cnt), tri.shape[0]
    assert V - E + F in (0, 1)


def test_annulus_sizes():
    xy, tri = inputs.annulus_mesh(32, 2)
    assert xy.shape[0] == 96 and tri.shape[0] == 128
    r = np.hypot(xy[:, 0], xy[:, 1])
    assert r.min() == pytest.approx(0.55) and r.max() == pytest.approx(1.0)


@pytest.mark.parametrize("T", [2, 3, 17, 64])
def test_random_mesh_face_count_and_area(T):
    xy, tri = inputs.random_square_mesh(1000 + T, T)
    assert tri.shape[0] == T
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    area = 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))
    assert area.sum() == pytest.approx(1.0, rel=1e-12)


def test_grf_statistics():
    """Empirical mean ~ 0, variance ~ sigma^2 and correlation at distance l
    ~ exp(-1/2) for the random-Fourier-feature field."""
    rng = np.random.default_rng(0)
    p = rng.uniform(0, 50, size=(20000, 2))
    g_all = []
    for seed in range(8):
        g_all.append(np.log(inputs.grf_coefficient(p, seed=seed)))
    g = np.concatenate(g_all)
    assert abs(g.mean()) < 0.05
    assert abs(g.var() - 1.0) < 0.1
    q = p + np.array([0.1, 0.0])
    c = []
    for seed in range(8):
        a = np.log(inputs.grf_coefficient(p, seed=seed))
        b = np.log(inputs.grf_coefficient(q, seed=seed))
        c.append(np.mean(a * b))
    assert abs(np.mean(c) - np.exp(-0.5)) < 0.08


def test_element_centroids_count():
    xy, tri = inputs.annulus_mesh(32, 2)
    c = inputs.element_centroids(xy, tri, 3)
    assert c.shape == (128 * 64, 2)
    r = np.hypot(c[:, 0], c[:, 1])
    assert r.min() > 0.5 and r.max() < 1.0
