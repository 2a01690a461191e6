"""The seeded input generators (paper_2210_02698_gb300/workloads.py) follow
the recipe they state: grid order, seeding, the four source kinds of the
uneven batch, the taper reading, the inclusion and 3D inputs."""
import math

import numpy as np

from paper_2210_02698_gb300 import workloads as W


def test_grid_order_and_centroids():
    g = W.Grid(5)
    x, z = g.centroids()
    i = 3 * 5 + 2                                  # b = 3, a = 2
    assert np.allclose((x[i], z[i]), (2.5 / 5, 3.5 / 5), rtol=1e-15)
    g3 = W.Grid3D(4, 0.52)
    x, y, z = g3.centroids()
    i = (3 * 4 + 1) * 4 + 2                        # c = 3, b = 1, a = 2
    assert np.allclose((x[i], y[i], z[i]), (2.5 * 0.13, 1.5 * 0.13, 3.5 * 0.13), rtol=1e-15)


def test_complex_normal_sources_are_seeded_per_column():
    s = W.complex_normal_sources(100, 3, 2000)
    assert s.flags["F_CONTIGUOUS"] and s.dtype == np.complex128
    for k in range(3):
        rng = np.random.default_rng(2000 + k)
        re, im = rng.standard_normal(100), rng.standard_normal(100)
        assert np.array_equal(s[:, k], re + 1j * im)


def test_taper_reading():
    r = np.array([0.0, 0.3, 0.35, 0.4, 0.5])
    t = W.taper(r, 0.3, 0.1)
    assert np.allclose(t, [1.0, 1.0, 0.5, 0.0, 0.0], atol=1e-15)
    rr = np.linspace(0.3, 0.4, 101)
    assert np.all(np.diff(W.taper(rr, 0.3, 0.1)) <= 0)


def test_mixed_sources_recipe():
    g = W.Grid(64)
    h = g.h
    w = 2 * math.pi * 8
    s = W.mixed_sources(g, w, 64, 2000)
    x, z = g.centroids()
    for k in range(16):                            # point sources: 1/h^2 in one cell
        nz = np.flatnonzero(s[:, k])
        assert len(nz) == 1 and s[nz[0], k] == 1.0 / h ** 2
    for k in range(16, 32):                        # line segments: 1/h near a segment in [0.1, 0.9]^2
        v = s[:, k]
        assert set(np.unique(v).tolist()) <= {0.0, 1.0 / h} and np.count_nonzero(v) >= 1
        on = np.flatnonzero(v)
        assert np.all((x[on] > 0.1 - h) & (x[on] < 0.9 + h) & (z[on] > 0.1 - h) & (z[on] < 0.9 + h))
    for k in range(32, 48):                        # Gaussian bumps: one complex amplitude, peak in [0.2, 0.8]^2
        v = s[:, k]
        c = np.array([x[np.argmax(np.abs(v))], z[np.argmax(np.abs(v))]])
        assert np.all((c > 0.2 - h) & (c < 0.8 + h))
        big = np.abs(v) > 1e-200
        phase = v[big] / np.abs(v[big])
        assert np.allclose(phase, phase[0])           # one complex amplitude
    for k in range(48, 64):                        # wavepackets: tapered Gaussian envelope at the centre
        v = s[:, k]
        r = np.hypot(x - 0.5, z - 0.5)
        assert np.all(v[r >= 0.4] == 0) and np.max(np.abs(v)) <= 1.0
        env = np.exp(-r ** 2 / (2 * 0.15 ** 2)) * W.taper(r, 0.3, 0.1)
        assert np.allclose(np.abs(v), env, atol=1e-15)


def test_point_and_gaussian_sources():
    g = W.Grid(16)
    p = W.point_source(g, 8, 8)
    assert np.flatnonzero(p[:, 0]).tolist() == [8 * 16 + 8] and p[8 * 16 + 8, 0] == 256.0
    gs = W.gaussian_center_source(g)
    x, z = g.centroids()
    assert np.allclose(gs[:, 0], np.exp(-((x - 0.5) ** 2 + (z - 0.5) ** 2) / (2 * 0.05 ** 2)))


def test_circle_segments_are_chords():
    cen, lw = W.circle_segments((0.4, 0.6), 0.2, 90)
    assert np.allclose(np.hypot(cen[:, 0] - 0.4, cen[:, 1] - 0.6), 0.2 * math.cos(math.pi / 90))
    assert np.allclose(lw, 2 * 0.2 * math.sin(math.pi / 90))


def test_media_3d():
    assert W.GRADIENT_3D.n(0.1, 0.26, 0.3) == 1.25 / (0.885 - 0.26)
    assert np.all(W.HOMOGENEOUS_3D.n(np.zeros(4), np.zeros(4), np.zeros(4)) == 1.0)
