"""Pins of the oracle's inclusion operators (oracle/inclusion.py, Sec. 3.2:
Eq. sie, Eq. s2s, Eq. m_v2s, Eq. m_s2v, Eq. m_v2v_inclu).

* The diagonal of K^{s2s} as read equals minus the segment integral of the
  local kernel (i/4) H0(w n |t|) (adaptive quadrature), with the
  O((kw)^2 log) error of the small-argument form; the literal printed forms
  do not.
* The reference solution - the exact series for a point source scattered by
  a circle on which the total field vanishes (Graf's addition theorem) -
  does vanish on the circle.
* Homogeneous medium, circle: the discrete surface solve converges to the
  series (point source), also for a volume source superposed cell by cell
  through the full composition K^{s2v} (K^{s2s})^{-1} K^{v2s} I.
* K^{s2v} is the transpose of K^{v2s} scaled by the segment lengths
  (reciprocity of g; exact for the homogeneous medium, to the table error
  for the gradient medium).
"""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import inclusion, kernel, tables
from paper_2210_02698_gb300 import workloads as W
from tests._common import load_tables

K4 = 2 * math.pi * 4
C, A = (0.5, 0.5), 0.2
ONE = (lambda x, z: np.ones_like(x))


@pytest.fixture(scope="module")
def homog():
    return tables.build_tables(W.HOMOGENEOUS, 16)


def test_s2s_diagonal_is_the_segment_integral():
    k = 40.0
    errs = []
    for kw in (0.05, 0.2):
        w = kw / k
        re = 2 * integrate.quad(lambda t: special.hankel1(0, k * t).real, 0, w / 2, limit=200)[0]
        im = 2 * integrate.quad(lambda t: special.hankel1(0, k * t).imag, 0, w / 2, limit=200)[0]
        exact = -0.25j * (re + 1j * im)
        errs.append(abs(inclusion.s2s_self(np.array([w]), k, 1.0)[0] - exact) / abs(exact))
    assert errs[0] < 1e-4 and errs[1] < 2e-3 and errs[1] / errs[0] > 8   # ~ (kw)^2 log


def test_exact_circle_series_vanishes_on_the_circle():
    th = np.linspace(0, 2 * np.pi, 13)[:-1]
    pts = np.stack([C[0] + A * np.cos(th), C[1] + A * np.sin(th)], axis=1)
    r0 = (0.12, 0.2)
    uinc = 0.25j * special.hankel1(0, K4 * np.hypot(pts[:, 0] - r0[0], pts[:, 1] - r0[1]))
    usca = inclusion.circle_exact_scattered(K4, C, A, r0, pts)
    assert np.abs(uinc + usca).max() < 1e-13 * np.abs(uinc).max()


def _point_source_error(tab, ns, diag=None):
    r0 = np.array([[0.12, 0.2]])
    obs = np.array([[0.85, 0.8], [0.5, 0.9], [0.15, 0.6], [0.8, 0.25]])
    cur = inclusion.arc(C, A, ns)
    K = inclusion.K_s2s(tab, K4, cur, ONE)
    if diag is not None:
        idx = np.arange(cur.Ns)
        K[idx, idx] = diag(cur.w, K4, np.ones(cur.Ns))
    P = np.linalg.solve(K, inclusion.green(tab, K4, cur.c, r0)[:, 0])
    usca = inclusion.K_s2v(tab, K4, cur, obs) @ P
    ex = inclusion.circle_exact_scattered(K4, C, A, r0[0], obs)
    return np.abs(usca - ex).max() / np.abs(ex).max()


def test_circle_scattering_converges_to_the_series(homog):
    e128, e512 = _point_source_error(homog, 128), _point_source_error(homog, 512)
    assert e512 < 2e-3 and e128 / e512 > 2.5
    # the diagonal as printed (no leading i) misses by >10%
    printed = (lambda w, om, n: -(w / 4) * (1 + 1j * (2 / math.pi) * (np.log(inclusion.GAMMA * om * n * w / 4) - 1)))
    assert _point_source_error(homog, 256, printed) > 0.05


def test_volume_source_composition_matches_superposed_series(homog):
    """U - K^{v2v} I = K^{s2v} (K^{s2s})^{-1} K^{v2s} I against the sum over
    source cells of I_j times the exact scattered field of a point source at
    cell j (the kernel between distinct points is exactly (i/4) H0 here)."""
    N = 32
    w = W.small_workload(W.HOMOGENEOUS, N, N / 8, 1)
    op = kernel.Operator(N, homog, K4, w.n_cells())
    x, z = w.grid.centroids()
    rc = np.hypot(x - C[0], z - C[1])
    s = np.exp(-((x - 0.2) ** 2 + (z - 0.22) ** 2) / (2 * 0.04 ** 2)) * (rc > A + 0.05)
    cur = inclusion.arc(C, A, 512)
    U, _ = inclusion.total_field(op, cur, ONE, s[:, None], v2v=np.zeros((w.grid.Nv, 1), complex))
    obs = np.nonzero((rc > A + 0.1) & (np.abs(x - 0.8) < 0.1))[0][:12]
    I = s * op.h ** 2
    src = np.nonzero(np.abs(I) > 1e-8 * np.abs(I).max())[0]
    ex = np.zeros(len(obs), dtype=complex)
    pts = np.stack([x[obs], z[obs]], axis=1)
    for j in src:
        ex += I[j] * inclusion.circle_exact_scattered(K4, C, A, (x[j], z[j]), pts)
    assert np.abs(U[obs, 0] - ex).max() < 3e-3 * np.abs(ex).max()


@pytest.mark.parametrize("medium,tol", [(W.HOMOGENEOUS, 1e-11), (W.GRADIENT, 1e-8)])
def test_s2v_is_the_scaled_transpose_of_v2s(medium, tol):
    tab = load_tables(medium)
    cur = inclusion.polyline([(0.1, 0.1), (0.1, 0.9), (0.9, 0.9), (0.9, 0.1)], 40)   # open square, side 0.8
    cells = np.random.default_rng(3).uniform(0.02, 0.98, size=(50, 2))
    Kv2s = inclusion.K_v2s(tab, K4, cur, cells)
    Ks2v = inclusion.K_s2v(tab, K4, cur, cells)
    assert np.abs(Ks2v - Kv2s.T * cur.w[None, :]).max() <= tol * np.abs(Ks2v).max()
