"""Pins of the oracle's sweeping table builder (oracle/sweep.py, sweep.c;
Sec. 2.3: factored eikonal Eq. faceik and transport Eq. equVs by
Lax-Friedrichs WENO sweeping, Taylor initialisation Eq. expansionT /
expansionV0 / expansionV1, local cubic interpolation to the nodes).

* Constant-gradient medium, whose tau, v0, v1 are exact in oracle.tables:
  the mesh errors over the unit square fall at least at the orders the
  paper states for tau, v0, v1 (fifth, third, first in h0), for an interior
  source and a corner source; tables at h0 = 1/64 match the exact tables.
* Homogeneous medium: the sweeps keep the exact solution tau = n0 |r - r0|,
  v0 = B0, v1 = 0.
* Lens: the series n^2 = sum S_k about a source has an O(rho^5) remainder;
  the stored lens tables are reciprocal (tau^2, v0, v1 symmetric in
  observation and source node), invariant under the lens's symmetries
  (x -> 1 - x, z -> 1 - z, x <-> z: the medium and the node set are), v0
  stays positive (no caustic), and the eikonal and v0 solves converged.
* Independently of the mesh, ray tracing (oracle/rays.py: Hamilton's
  equations in tau and the ray-tube form of the v0 transport equation)
  reproduces the gradient medium's closed forms, and then the stored lens
  tables' tau^2 and v0 on sampled node pairs.
"""
import math

import numpy as np
import pytest

from oracle import chebyshev, rays, sweep, tables
from paper_2210_02698_gb300 import workloads as W
from tests._common import load_tables, table_path

B0 = 1.0 / (2.0 * math.sqrt(math.pi))


def _errors(medium, x0, z0, h0):
    t2, v0, v1, X, Z, info = sweep.fields(medium, x0, z0, h0)
    et2, ev0, ev1 = tables.ingredient_functions(medium)(X, Z, x0, z0)
    ins = (X >= 0) & (X <= 1) & (Z >= 0) & (Z <= 1)
    return (np.abs(np.sqrt(t2) - np.sqrt(et2))[ins].max(), np.abs(v0 - ev0)[ins].max(),
            np.abs(v1 - ev1)[ins].max(), info)


@pytest.mark.parametrize("src", ["interior", "corner"])
def test_gradient_medium_convergence_orders(src):
    xn = chebyshev.nodes(16)
    x0, z0 = (0.3141, 0.4472) if src == "interior" else (xn[0], xn[15])
    e1 = _errors(W.GRADIENT, x0, z0, 1 / 32)
    e2 = _errors(W.GRADIENT, x0, z0, 1 / 64)
    for info in (e1[3], e2[3]):
        assert np.all(info[3:] < 1e-12)                  # every solve converged
    # orders >= 4.5, 3, 1 over one halving (the paper: 5, 3, 1)
    assert e1[0] / e2[0] > 2 ** 4.5 and e2[0] < 2e-9
    assert e1[1] / e2[1] > 2 ** 3 and e2[1] < 5e-8
    assert e1[2] / e2[2] > 2 ** 1 and e2[2] < 2e-5


def test_gradient_tables_match_exact():
    src = np.array([0, 37, 120, 255])
    t = sweep.build_tables(W.GRADIENT, 16, h0=1 / 64, sources=src)
    ex = tables.build_tables(W.GRADIENT, 16)
    assert np.abs(t["tau2"] - ex["tau2"][:, src]).max() < 5e-8
    assert np.abs(t["v0"] - ex["v0"][:, src]).max() < 5e-7
    assert np.abs(t["v1"] - ex["v1"][:, src]).max() < 1e-4
    assert np.all(t["info"][:, 3:] < 1e-12)


def test_homogeneous_medium_is_a_fixed_point():
    med = W.Medium("homogeneous", n0=1.3)
    x0, z0 = 0.4, 0.7
    t2, v0, v1, X, Z, info = sweep.fields(med, x0, z0, 1 / 32)
    ins = np.isfinite(v0)
    assert np.abs(t2 - 1.3 ** 2 * ((X - x0) ** 2 + (Z - z0) ** 2)).max() < 1e-12
    assert np.abs(v0[ins] - B0).max() < 1e-12
    assert np.abs(v1[ins]).max() < 1e-11        # Lap v0 of a constant: rounding / h0^2


def test_lens_n2_series_remainder():
    med = W.LENS
    x0, z0 = 0.31, 0.62
    S = sweep.n2_series(med, x0, z0, 4)
    rng = np.random.default_rng(3)
    th = rng.uniform(0, 2 * np.pi, 16)
    errs = []
    for rho in (0.04, 0.02):
        X, Z = rho * np.cos(th), rho * np.sin(th)
        approx = sum(np.sum([c * X ** (k - m) * Z ** m for m, c in enumerate(S[k])], axis=0) for k in range(5))
        exact = med.n(x0 + X, z0 + Z) ** 2
        errs.append(np.abs(approx - exact).max())
    assert errs[0] / errs[1] > 2 ** 4.7                   # remainder O(rho^5)


def _lens():
    return load_tables(W.LENS), np.load(table_path(W.LENS))["sweep_info"]


def _node_maps(n_I=16):
    i1, i2 = np.meshgrid(np.arange(n_I), np.arange(n_I))
    i1, i2 = i1.reshape(-1), i2.reshape(-1)          # node k = i2 n_I + i1
    flip_x = i2 * n_I + (n_I - 1 - i1)
    flip_z = (n_I - 1 - i2) * n_I + i1
    swap = i1 * n_I + i2
    return flip_x, flip_z, swap


def test_lens_tables_reciprocity_symmetry_positivity():
    t, info = _lens()
    assert np.all(info[:, 3] < 1e-11) and np.all(info[:, 4] < 1e-11)   # eikonal, v0 converged
    v1max = np.abs(t["v1"]).max()
    assert np.all(info[:, 5] < 1e-3 * v1max)                            # v1: last update small
    idx = np.arange(256)
    assert np.all(t["tau2"][idx, idx] == 0.0) and np.all(t["v0"][idx, idx] == B0)
    assert t["v0"].min() > 0.2 and t["v0"].max() < 0.5                 # no caustic
    t2max = t["tau2"].max()
    # reciprocity holds to the discretisation error (measured at h0 = 1/256:
    # 3e-10 of max tau^2, 9e-8, 1.5e-3 of max |v1|)
    assert np.abs(t["tau2"] - t["tau2"].T).max() < 1e-8 * t2max
    assert np.abs(t["v0"] - t["v0"].T).max() < 1e-6
    assert np.abs(t["v1"] - t["v1"].T).max() < 1e-2 * v1max
    # the mirror and diagonal symmetries map the mesh onto itself: to
    # rounding for tau^2 and v0, to the v1 cycle residual for v1
    for m in _node_maps():
        assert np.abs(t["tau2"][np.ix_(m, m)] - t["tau2"]).max() < 1e-12 * t2max
        assert np.abs(t["v0"][np.ix_(m, m)] - t["v0"]).max() < 1e-10
        assert np.abs(t["v1"][np.ix_(m, m)] - t["v1"]).max() < 1e-3 * v1max
    # tau^2 grows with distance as n^2 |r - r0|^2 between the lens's bounds 1 and 1.1
    xn = chebyshev.nodes(16)
    px, pz = np.tile(xn, 16), np.repeat(xn, 16)
    d2 = (px[:, None] - px[None, :]) ** 2 + (pz[:, None] - pz[None, :]) ** 2
    off = d2 > 0
    ratio = t["tau2"][off] / d2[off]
    assert ratio.min() > 1.0 - 1e-9 and ratio.max() < 1.1 ** 2


def _sample_pairs(seed, nsrc=8, nobs=8):
    rng = np.random.default_rng(seed)
    out = []
    for j in rng.choice(256, nsrc, replace=False):
        out.append((int(j), rng.choice(np.setdiff1d(np.arange(256), [j]), nobs, replace=False)))
    return out


def test_ray_tracing_reproduces_gradient_closed_forms():
    xn = chebyshev.nodes(16)
    px, pz = np.tile(xn, 16), np.repeat(xn, 16)
    med = W.GRADIENT
    for j, obs in _sample_pairs(5, nsrc=4, nobs=6):
        T, v0, res = rays.tau_v0(med, px[j], pz[j], px[obs], pz[obs])
        et = tables.tau_gradient(px[obs], pz[obs], px[j], pz[j], med.c0, med.g)
        assert res.max() < 1e-12
        assert np.abs(T - et).max() < 1e-12
        assert np.abs(v0 - tables.v0_gradient(et, med.g)).max() < 1e-9


def test_lens_tables_match_ray_tracing():
    """The sweeping builder's lens tables against rays (measured: tau^2 to
    3.7e-10, v0 to 5.3e-8 on these pairs)."""
    t, _ = _lens()
    xn = chebyshev.nodes(16)
    px, pz = np.tile(xn, 16), np.repeat(xn, 16)
    for j, obs in _sample_pairs(11):
        T, v0, res = rays.tau_v0(W.LENS, px[j], pz[j], px[obs], pz[obs])
        assert res.max() < 1e-12
        assert np.abs(T * T - t["tau2"][obs, j]).max() < 2e-9
        assert np.abs(v0 - t["v0"][obs, j]).max() < 3e-7


def test_stored_lens_tables_are_the_builders_output():
    """Provenance of the stored lens tables: one column regenerated by the
    committed builder at the stored mesh (h0 = 1/256) reproduces them (to
    rounding: the builder is compiled without contracted multiply-adds, but
    libm's exp, pow and cos may differ between platforms)."""
    t, _ = _lens()
    j = 137
    r = sweep.build_tables(W.LENS, 16, h0=1 / 256, sources=[j])
    assert np.abs(r["tau2"][:, 0] - t["tau2"][:, j]).max() < 1e-12 * t["tau2"].max()
    assert np.abs(r["v0"][:, 0] - t["v0"][:, j]).max() < 1e-10
    assert np.abs(r["v1"][:, 0] - t["v1"][:, j]).max() < 1e-8


def test_ray_v1_reproduces_gradient_closed_form():
    """v1 by the ray form of Eq. equVs (s = 0) with Lap v0 from ray-traced v0
    against the gradient medium's v1 (the oracle's quadrature of the same
    equation in closed-form coefficients)."""
    xn = chebyshev.nodes(16)
    px, pz = np.tile(xn, 16), np.repeat(xn, 16)
    med = W.GRADIENT
    for j, obs in _sample_pairs(5, nsrc=3, nobs=5):
        v1 = rays.v1_along_ray(med, px[j], pz[j], px[obs], pz[obs])
        et = tables.tau_gradient(px[obs], pz[obs], px[j], pz[j], med.c0, med.g)
        assert np.abs(v1 - tables.v1_gradient(et, med.g)).max() < 1e-6


def test_lens_v1_matches_ray_transport():
    """The lens tables' v1 (first-order accurate by construction: two
    differences of v0) against the ray form of the transport equation
    (measured: within 6.2e-5 on 64 pairs, |v1| up to 0.19)."""
    t, _ = _lens()
    xn = chebyshev.nodes(16)
    px, pz = np.tile(xn, 16), np.repeat(xn, 16)
    for j, obs in _sample_pairs(11, nsrc=4, nobs=6):
        v1 = rays.v1_along_ray(W.LENS, px[j], pz[j], px[obs], pz[obs])
        assert np.abs(v1 - t["v1"][obs, j]).max() < 2e-4


def test_lens_rays_do_not_cross():
    """No caustic in the lens (the method assumes a single-valued tau): over
    fans of 360 rays from corner, centre and interior sources, the ray-tube
    width J (positive orientation of the fan) stays far from zero wherever
    the rays are inside the unit square (measured: J >= 0.61 tau)."""
    th = np.linspace(0, 2 * np.pi, 361)[:-1]
    dth = 1e-4
    for x0, z0 in [(0.0024, 0.0024), (0.5, 0.5), (0.2, 0.7)]:
        for T in np.linspace(0.05, 1.6, 8):
            TT = np.full_like(th, T)
            y = rays.trace(W.LENS, x0, z0, th, TT, 200)
            yp = rays.trace(W.LENS, x0, z0, th + dth, TT, 200)
            ym = rays.trace(W.LENS, x0, z0, th - dth, TT, 200)
            jx, jz = (yp[0] - ym[0]) / (2 * dth), (yp[1] - ym[1]) / (2 * dth)
            width = -(jx * y[3] - jz * y[2]) / np.hypot(y[2], y[3])
            ins = (y[0] >= 0) & (y[0] <= 1) & (y[1] >= 0) & (y[1] <= 1)
            if ins.any():
                assert (width[ins] / T).min() > 0.3


@pytest.mark.parametrize("medium", [W.GRADIENT, W.LENS])
def test_wavefront_order_is_bit_identical(medium):
    """Sweeping anti-diagonal by anti-diagonal (the order a parallel sweep
    takes) gives bit for bit the fields of the row-by-row Gauss-Seidel
    sweeps: an update reads only its own row and column, and along both the
    two orders visit the points in the same upwind order, so every update
    sees the same new and old values (whatever the convergence state)."""
    x0, z0 = 0.3141, 0.4472
    rows = sweep.fields(medium, x0, z0, 1 / 32)
    wave = sweep.fields(medium, x0, z0, 1 / 32, wavefront=True)
    for q in range(3):
        assert np.array_equal(rows[q], wave[q], equal_nan=True), q
    assert np.array_equal(rows[5], wave[5])


def test_sweep_visit_orders():
    """The four sweep directions visit every mesh point once: row by row
    (the default) or anti-diagonal by anti-diagonal, each direction starting
    from its own corner."""
    M = 7
    for o in range(4):
        fi = o in (1, 2)                       # i runs from M-1 down
        fj = o in (2, 3)                       # j runs from M-1 down
        rows = sweep.visit_order(o, M)
        wave = sweep.visit_order(o, M, wavefront=True)
        for order in (rows, wave):
            assert sorted(order.tolist()) == list(range(M * M))
        i, j = rows % M, rows // M
        ii, jj = (M - 1 - i if fi else i), (M - 1 - j if fj else j)
        assert np.array_equal(jj * M + ii, np.arange(M * M))
        i, j = wave % M, wave // M
        d = (M - 1 - i if fi else i) + (M - 1 - j if fj else j)
        assert np.all(np.diff(d) >= 0) and d[0] == 0 and d[-1] == 2 * M - 2
