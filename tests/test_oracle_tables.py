"""Pins of oracle.tables: the HB ingredients of the two workload media.

Each check is independent of the hyperbolic-plane reduction used inside
oracle.tables: Cartesian finite differences of Eq. eikonal / Eq. equVs, the
paper's own Taylor recursions (Eq. recursiveT, Eq. recursiveB, Eq. C0),
reciprocity, the homogeneous limit, an adaptive quadrature, and the exact
Green's function of the medium.
"""
import math

import numpy as np
import pytest

from oracle import taylor, tables
from paper_2210_02698_gb300 import workloads as W

C0, G = 1.0, 0.5
PTS = [((0.3, 0.4), (0.7, 0.65)), ((0.1, 0.9), (0.8, 0.2)), ((0.5, 0.5), (0.52, 0.47))]


def _n(z):
    return 1.0 / (C0 + G * z)


def _tau(x, z, x0, z0):
    return tables.tau_gradient(x, z, x0, z0, C0, G)


def _grad(f, x, z, e):
    return ((f(x + e, z) - f(x - e, z)) / (2 * e), (f(x, z + e) - f(x, z - e)) / (2 * e))


def _lap(f, x, z, e):
    return (f(x + e, z) + f(x - e, z) + f(x, z + e) + f(x, z - e) - 4 * f(x, z)) / e**2


@pytest.mark.parametrize("r,r0", PTS)
def test_eikonal_fd_residual(r, r0):
    (x, z), (x0, z0) = r, r0
    gx, gz = _grad(lambda a, b: _tau(a, b, x0, z0), x, z, 1e-5)
    assert abs(math.hypot(gx, gz) - _n(z)) < 5e-8     # FD truncation ~ e^2 tau'''


@pytest.mark.parametrize("r,r0", PTS)
def test_transport_v0_fd_residual(r, r0):
    (x, z), (x0, z0) = r, r0
    t = lambda a, b: _tau(a, b, x0, z0)
    v0 = lambda a, b: tables.v0_gradient(t(a, b), G)
    e = 1e-4
    tx, tz = _grad(t, x, z, e)
    vx, vz = _grad(v0, x, z, e)
    n2 = _n(z) ** 2
    dv_dtau = (tx * vx + tz * vz) / n2          # derivative along the ray
    lap_t2 = _lap(lambda a, b: t(a, b) ** 2, x, z, e)
    T = t(x, z)
    res = 4 * T * n2 * dv_dtau + v0(x, z) * (lap_t2 - 4 * n2)
    assert abs(res) < 1e-6 * (4 * n2 * v0(x, z))


@pytest.mark.parametrize("r,r0", PTS[:2])
def test_transport_v1_fd_residual(r, r0):
    (x, z), (x0, z0) = r, r0
    t = lambda a, b: _tau(a, b, x0, z0)
    v0 = lambda a, b: tables.v0_gradient(t(a, b), G)
    v1 = lambda a, b: tables.v1_gradient(t(a, b), G)[0]
    e = 2e-3
    tx, tz = _grad(t, x, z, 1e-4)
    wx, wz = _grad(v1, x, z, 1e-4)
    n2 = _n(z) ** 2
    dv1 = (tx * wx + tz * wz) / n2
    lap_t2 = _lap(lambda a, b: t(a, b) ** 2, x, z, 1e-4)
    lap_v0 = _lap(v0, x, z, e)
    res = 4 * t(x, z) * n2 * dv1 + v1(x, z) * lap_t2 - lap_v0
    assert abs(res) < 1e-4 * abs(lap_v0)


def test_taylor_recursions_match_at_their_orders():
    x0, z0 = 0.4, 0.3
    S = taylor.n2_series_gradient(C0 + G * z0, G, 8)
    T, B, C = taylor.recursions(S)
    errs = []
    for d in (0.04, 0.02, 0.01):
        dx, dz = d * math.cos(0.7), d * math.sin(0.7)
        t = _tau(x0 + dx, z0 + dz, x0, z0)
        errs.append((abs(taylor.series_value(T, dx, dz) - t * t),
                     abs(taylor.series_value(B, dx, dz) - tables.v0_gradient(t, G)),
                     abs(taylor.series_value(C, dx, dz) - tables.v1_gradient(t, G)[0])))
    errs = np.array(errs)
    # truncation orders P_T = 6, P_B = 4, P_C = 2: errors O(d^7), O(d^5), O(d^3)
    for col, order in ((1, 5), (2, 3)):
        rate = np.log2(errs[:-1, col] / errs[1:, col])
        assert np.all(rate > order - 0.5), (col, rate)
    assert errs[0, 0] < 1e-12 and errs[-1, 0] < 1e-16
    # Eq. C0: v1 at the source
    assert abs(C[0][0] - tables.v1_gradient(np.array([0.0]), G)[0]) < 1e-15


def test_reciprocity():
    rng = np.random.default_rng(4)
    p = rng.uniform(0, 1, (50, 4))
    a = tables.ingredient_functions(W.GRADIENT)(p[:, 0], p[:, 1], p[:, 2], p[:, 3])
    b = tables.ingredient_functions(W.GRADIENT)(p[:, 2], p[:, 3], p[:, 0], p[:, 1])
    for u, v in zip(a, b):
        assert np.max(np.abs(u - v)) < 1e-14


def test_homogeneous_limit():
    tau = np.array([0.01, 0.3, 1.2])
    assert np.max(np.abs(tables.v0_gradient(tau, 1e-7) - tables.B0_2D)) < 1e-13
    assert np.max(np.abs(tables.v1_gradient(tau, 1e-7))) < 1e-13
    d = tables.tau_gradient(0.7, 0.2, 0.1, 0.6, 1.0, 1e-9)
    assert abs(d - math.hypot(0.6, 0.4)) < 1e-9


def test_v1_quadrature_against_adaptive():
    from scipy import integrate
    for T in (0.003, 0.4, 1.3):
        val = integrate.quad(lambda t: math.sqrt(math.sinh(G * t) / t) * tables._Q_gradient(np.array(t), G),
                             0, T, epsabs=0, epsrel=1e-13)[0]
        ref = val / (4 * math.sqrt(T * math.sinh(G * T)))
        assert abs(tables.v1_gradient(np.array([T]), G)[0] - ref) < 1e-15


def test_ansatz_converges_to_exact_green():
    pytest.importorskip("mpmath")
    from oracle import hankel
    T = 0.7
    e1, e0 = [], []
    for om in (20.0, 40.0, 80.0):
        ge = tables.exact_green_gradient(T, om, G)
        f0 = hankel.f0(om, T)
        g0 = tables.v0_gradient(T, G) * f0
        g1 = g0 + tables.v1_gradient(np.array([T]), G)[0] * hankel.f1(om, T)
        e1.append(abs(g1 - ge) / abs(ge))
        e0.append(abs(g0 - ge) / abs(ge))
    # N = 1 error O(omega^-2) relative, N = 0 error O(omega^-1) (Sec. 5.2)
    assert 3.5 < e1[0] / e1[1] < 4.5 and 3.5 < e1[1] / e1[2] < 4.5
    assert 1.8 < e0[0] / e0[1] < 2.2
    assert e1[-1] < 1e-7


def test_tables_layout_and_diagonal():
    tab = tables.build_tables(W.HOMOGENEOUS, 4)
    xn = tab["nodes"]
    i, j = 1 * 4 + 2, 3 * 4 + 0          # node (i1=2, i2=1) observes source (j1=0, j2=3)
    assert abs(tab["tau2"][i, j] - ((xn[2] - xn[0]) ** 2 + (xn[1] - xn[3]) ** 2)) < 1e-15
    assert np.all(np.diag(tab["tau2"]) == 0) and np.all(tab["v1"] == 0)
    assert np.allclose(tab["v0"], 1 / (2 * math.sqrt(math.pi)))
