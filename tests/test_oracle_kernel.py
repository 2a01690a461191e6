"""Pins of oracle.hankel, oracle.kernel and oracle.dense."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import dense, hankel, kernel, tables
from paper_2210_02698_gb300 import workloads as W


def test_hankel_against_mpmath():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    for x in (0.05, 0.52, 3.3, 17.0, 229.0, 1800.0):
        for q in (0, 1):
            ref = complex(mp.hankel1(q, x))
            got = special.hankel1(q, x)
            assert abs(got - ref) <= 2e-15 * abs(ref) + 1e-300, (q, x)


def test_wronskian_and_f1_limit():
    x = np.array([0.3, 2.0, 40.0, 700.0])
    J0, J1, Y0, Y1 = special.j0(x), special.j1(x), special.y0(x), special.y1(x)
    assert np.max(np.abs((J1 * Y0 - J0 * Y1) * np.pi * x / 2 - 1)) < 1e-12
    om = 50.0
    # f1(tau -> 0+) = -2 / (sqrt(pi) omega^2)
    assert abs(hankel.f1(om, 1e-9) + 2 / (math.sqrt(math.pi) * om**2)) < 1e-12 / om**2


def test_homogeneous_ansatz_is_free_space_green():
    tau = np.array([0.01, 0.2, 0.9])
    om = 30.0
    g = tables.B0_2D * hankel.f0(om, tau)
    assert np.max(np.abs(g - 0.25j * special.hankel1(0, om * tau))) < 1e-15


def test_self_term_lemma_against_brute_force_cell_integral():
    # integrate H0(omega n0 |r|) over the square cell directly (polar, 8 triangles
    # by symmetry, radial integral numerically - no use of A&S 9.1.30)
    for n0, om, h in ((1.0, 50.0, 1 / 64), (0.8, 200.0, 1 / 256), (1.0, 16 * math.pi, 1 / 64)):
        k = om * n0

        def radial(th, part):
            R = h / (2 * math.cos(th))
            f = (lambda r: special.hankel1(0, k * r).real * r) if part == 0 else \
                (lambda r: special.hankel1(0, k * r).imag * r)
            return integrate.quad(f, 0, R, epsabs=0, epsrel=1e-12, limit=200)[0]

        Ire = 8 * integrate.quad(lambda t: radial(t, 0), 0, math.pi / 4, epsrel=1e-11)[0]
        Iim = 8 * integrate.quad(lambda t: radial(t, 1), 0, math.pi / 4, epsrel=1e-11)[0]
        brute = 0.25j * (Ire + 1j * Iim) / h**2
        assert abs(kernel.self_term(n0, om, h) - brute) < 1e-9 * abs(brute)


def test_self_term_small_cell_closed_form():
    """As k h -> 0 (k = n0 w), H0(x) = 1 + (2i/pi)(ln(x/2) + gamma_E) + O(x^2 ln x)
    (A&S 9.1.12-13) averaged over the square cell of side h, where the mean of
    ln r is ln(h/2) + (ln 2)/2 + pi/4 - 3/2, gives
    K_ii -> (i/4)(1 + (2i/pi)(ln(k h/4) + gamma_E + (ln 2)/2 + pi/4 - 3/2)),
    a check of the self term independent of the lemma's theta integral."""
    gamma = 0.5772156649015329
    errs = []
    for kh in (1e-2, 1e-3):
        n0, h = 0.8, 1 / 64
        om = kh / (n0 * h)
        closed = 0.25j * (1 + (2j / math.pi) * (math.log(kh / 4) + gamma + 0.5 * math.log(2) + math.pi / 4 - 1.5))
        errs.append(abs(kernel.self_term(n0, om, h) - closed) / abs(closed))
    assert errs[0] < 1e-5 and errs[1] < 1e-7 and errs[0] / errs[1] > 50   # O((k h)^2)


def test_homogeneous_entries_exact():
    w = W.WORKLOADS["homog64"]
    tab = tables.build_tables(W.HOMOGENEOUS, 16)
    op = kernel.Operator(w.N, tab, w.omega, w.n_cells())
    rows = np.array([0, 77, 2050, 4095])
    cols = np.arange(0, 4096, 37)
    K = op.block(rows, cols)
    d = np.hypot(op.px[rows][:, None] - op.px[cols][None, :], op.pz[rows][:, None] - op.pz[cols][None, :])
    off = rows[:, None] != cols[None, :]
    exact = 0.25j * special.hankel1(0, w.omega * np.where(off, d, 1.0))
    assert np.max(np.abs(K - exact)[off]) < 1e-13


def _small_op(N=16, medium=W.GRADIENT, wl=2):
    w = W.small_workload(medium, N, wl, 2)
    tab = tables.build_tables(medium, 8)
    return kernel.Operator(w.N, tab, w.omega, w.n_cells())


def test_dense_apply_equals_full_matrix_and_adjoint_identity():
    op = _small_op()
    K = op.block(np.arange(op.Nv), np.arange(op.Nv))
    s = W.complex_normal_sources(op.Nv, 3, 11)
    U = dense.apply(op, s, chunk=100)
    assert np.max(np.abs(U - K @ (s * op.h**2))) < 1e-13 * np.max(np.abs(U))
    u = W.complex_normal_sources(op.Nv, 3, 21)
    S = dense.adjoint(op, u, chunk=70)
    assert np.max(np.abs(S - op.h**2 * K.conj().T @ u)) < 1e-13 * np.max(np.abs(S))
    lhs = np.vdot(u, U)
    rhs = np.vdot(S, s)
    assert abs(lhs - rhs) < 1e-13 * np.linalg.norm(U) * np.linalg.norm(u)


def test_gradient_entries_close_to_uninterpolated():
    # Chebyshev interpolation with n_I = 16 of the exact ingredients
    op = _small_op(N=32, wl=4)
    op16 = kernel.Operator(op.N, tables.build_tables(W.GRADIENT, 16), op.omega, op.n_cells)
    rows = np.array([3, 500, 1000])
    cols = np.arange(0, op.Nv, 5)
    K = op16.block(rows, cols)
    f = tables.ingredient_functions(W.GRADIENT)
    t2, v0, v1 = f(op.px[rows][:, None], op.pz[rows][:, None], op.px[cols][None, :], op.pz[cols][None, :])
    off = rows[:, None] != cols[None, :]
    t = np.sqrt(np.where(off, t2, 1.0))
    ex = v0 * hankel.f0(op.omega, t) + v1.reshape(t.shape) * hankel.f1(op.omega, t)
    assert np.max(np.abs(K - ex)[off]) < 1e-6 * np.max(np.abs(ex))
