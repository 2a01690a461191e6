"""Pins of the oracle's 3D ingredients (oracle/hb3d.py: Sec. 2 with d = 3,
Eq. termf, Eq. equVs, Eq. initialv0; Sec. 5.1.2 3D media and exact Green's
function; Appendix A.2 3D self term)."""
import math

import numpy as np
import pytest

from oracle import chebyshev, hb3d
from paper_2210_02698_gb300 import workloads as W

GR = W.GRADIENT_3D
PAIRS = [((0.35, 0.05, 0.22), (0.1, 0.2, 0.3)), ((0.05, 0.5, 0.45), (0.4, 0.1, 0.05)),
         ((0.26, 0.26, 0.26), (0.27, 0.24, 0.3)), ((0.5, 0.5, 0.02), (0.02, 0.02, 0.5))]


def test_half_order_terms_are_elementary():
    """Eq. termf at q = -1/2 and 1/2 (scipy's half-order Hankel functions)
    equals e^{i w tau}/(2 tau) and i e^{i w tau}/w: H_{+-1/2} are elementary
    (A&S 10.1.11-12), so a wrong sign, power or phase shows here."""
    tau = np.linspace(1e-3, 3.0, 200)
    for w in (3.0, 40.0, 500.0):
        e = np.exp(1j * w * tau)
        assert np.allclose(hb3d.f_q(-0.5, w, tau), e / (2 * tau), rtol=1e-12, atol=0)
        assert np.allclose(hb3d.f_q(0.5, w, tau), 1j * e / w, rtol=1e-12, atol=0)


def test_homogeneous_ansatz_is_free_space_green():
    """v0 = n0/(2 pi) (Eq. initialv0, d = 3), v1 = 0: the ansatz is
    e^{i k R}/(4 pi R), k = n0 w, for every w."""
    med = W.Medium3D("homogeneous", n0=1.3)
    r0 = np.array([0.2, 0.3, 0.4])
    r = np.random.default_rng(1).uniform(0, 1, size=(50, 3))
    for w in (5.0, 60.0):
        R = np.linalg.norm(r - r0, axis=1)
        want = np.exp(1j * w * 1.3 * R) / (4 * math.pi * R)
        assert np.allclose(hb3d.green(med, w, r, r0), want, rtol=1e-12, atol=0)


def test_gradient_tau_is_the_printed_arccosh_form():
    """tau = (1/|G0|) arccosh(1 + n n0 |G0|^2 R^2 / 2), |G0| = 0.8 (Sec. 5.1.2),
    at distances where the arccosh form keeps its digits."""
    for r, r0 in PAIRS:
        r, r0 = np.array(r), np.array(r0)
        R = np.linalg.norm(r - r0)
        n, n0 = GR.n(*r), GR.n(*r0)
        printed = math.acosh(1 + 0.5 * n * n0 * 0.8 ** 2 * R * R) / 0.8
        assert abs(hb3d.tau(GR, r, r0) - printed) < 1e-12 * printed


def _fd(f, p, h):
    """Fourth-order central gradient and Laplacian of f at p."""
    g, lap = np.zeros(3), 0.0
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = h
        fp1, fm1, fp2, fm2 = f(p + e), f(p - e), f(p + 2 * e), f(p - 2 * e)
        g[ax] = (8 * (fp1 - fm1) - (fp2 - fm2)) / (12 * h)
        lap += (-fp2 + 16 * fp1 - 30 * f(p) + 16 * fm1 - fm2) / (12 * h * h)
    return g, lap


@pytest.mark.parametrize("pair", PAIRS)
def test_gradient_closed_forms_solve_eikonal_and_transport(pair):
    """|grad tau| = n (Eq. eikonalnormal) and Eq. equVs with d = 3:
    4 tau n^2 dv0/dtau + v0 (Lap tau^2 - 6 n^2) = 0 and
    4 tau n^2 dv1/dtau + v1 (Lap tau^2 - 2 n^2) = Lap v0, d/dtau = (grad tau / n^2) . grad."""
    r, r0 = (np.array(v) for v in pair)
    T = lambda p: float(hb3d.tau(GR, p, r0))           # noqa: E731
    V0 = lambda p: float(hb3d.v0(GR, p, r0))           # noqa: E731
    V1 = lambda p: float(hb3d.v1(GR, p, r0))           # noqa: E731
    h = min(2e-3, 0.02 * np.linalg.norm(r - r0))      # derivatives grow as 1/R near the source
    gt, _ = _fd(T, r, h)
    _, lap_t2 = _fd(lambda p: T(p) ** 2, r, h)
    g0, lap_v0 = _fd(V0, r, h)
    g1, _ = _fd(V1, r, h)
    n, tau = GR.n(*r), T(r)
    assert abs(np.linalg.norm(gt) - n) < 1e-8 * n
    d0 = gt @ g0 / n ** 2
    d1 = gt @ g1 / n ** 2
    scale = abs(V0(r)) * n ** 2
    assert abs(4 * tau * n ** 2 * d0 + V0(r) * (lap_t2 - 6 * n ** 2)) < 1e-7 * scale
    assert abs(4 * tau * n ** 2 * d1 + V1(r) * (lap_t2 - 2 * n ** 2) - lap_v0) < 1e-7 * scale
    # and the source value of Eq. initialv0 (d = 3)
    assert abs(float(hb3d.v0(GR, r0, r0)) - GR.n(*r0) / (2 * math.pi)) < 1e-15


def test_gradient_ansatz_error_orders_against_exact_green():
    """Against the exact Green's function of the medium the N = 0 error falls
    as w^-1 and the N = 1 error as w^-2 (the orders of Eq. inferror with
    d = 3 that the paper's 3D convergence test reports), and the leading
    amplitude v0 / (2 tau) equals |G| exactly."""
    r = np.array([p[0] for p in PAIRS])
    r0 = np.array([p[1] for p in PAIRS])
    e0, e1 = [], []
    for w in (20.0, 40.0, 80.0, 160.0):
        G = hb3d.exact_green(GR, w, r, r0)
        e0.append(np.max(np.abs(hb3d.green(GR, w, r, r0, N=0) - G) / np.abs(G)))
        e1.append(np.max(np.abs(hb3d.green(GR, w, r, r0, N=1) - G) / np.abs(G)))
    for a, b in zip(e0, e0[1:]):
        assert 1.9 < a / b < 2.1
    for a, b in zip(e1, e1[1:]):
        assert 3.8 < a / b < 4.2
    assert e1[-1] < 1e-6
    amp = hb3d.v0(GR, r, r0) / (2 * hb3d.tau(GR, r, r0))
    assert np.allclose(amp, np.abs(hb3d.exact_green(GR, 50.0, r, r0)), rtol=1e-13, atol=0)


def test_cube_integral_small_k_moments():
    """As k h -> 0: Re I -> (h^2 / 4 pi) (3 ln(2 + sqrt 3) - pi/2) (the
    integral of 1/r over the unit cube about its centre) and
    Im I = (1/4 pi)(k h^3 - k^3 int r^2 dV / 6 + ...), int r^2 dV = h^5 / 4."""
    C = 3 * math.log(2 + math.sqrt(3)) - math.pi / 2
    for h in (0.1, 0.01):
        for kh in (1e-2, 1e-3):
            k = kh / h
            I = hb3d.cube_integral(k, h)
            assert abs(I.real - C * h * h / (4 * math.pi)) < 2 * kh * kh * h * h
            im = (k * h ** 3 - k ** 3 * h ** 5 / 24) / (4 * math.pi)
            assert abs(I.imag - im) < 1e-3 * kh ** 5 * h * h + 1e-15 * h * h


def test_cube_integral_against_cartesian_quadrature():
    """At k h of order one: the 48-piece polar form against a tensor
    Gauss-Legendre rule on (e^{i k r} - 1)/(4 pi r) (bounded) plus the
    k = 0 part C h^2 / (4 pi)."""
    C = 3 * math.log(2 + math.sqrt(3)) - math.pi / 2
    x, wq = np.polynomial.legendre.leggauss(48)
    for k, h in ((10.0, 0.1), (30.0, 0.1), (3.0, 1.0)):
        # the octant [0, h/2]^3, 8 copies; nodes mapped from [-1, 1]
        t = (x + 1) * h / 4
        wt = wq * h / 4
        X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
        Wt = wt[:, None, None] * wt[None, :, None] * wt[None, None, :]
        R = np.sqrt(X * X + Y * Y + Z * Z)
        smooth = 8 * np.sum(Wt * (np.exp(1j * k * R) - 1) / (4 * math.pi * R))
        want = smooth + C * h * h / (4 * math.pi)
        got = hb3d.cube_integral(k, h)
        assert abs(got - want) < 1e-6 * abs(want)



def test_tables_homogeneous_interpolate_exactly():
    """tau^2 = n0^2 |r - r0|^2 has degree 2 in each coordinate, so the 3D
    tensor interpolation (n_I >= 3) reproduces it and the entries equal
    e^{i k R}/(4 pi R) off the diagonal; the diagonal is the cube integral."""
    med = W.Medium3D("homogeneous", n0=1.1)
    g = W.Grid3D(6, 0.5)
    w = 2 * math.pi * 4
    op = hb3d.Operator3(g, hb3d.build_tables3(med, 4, g.L), w, med)
    idx = np.arange(g.Nv)
    K = op.block(idx, idx)
    P = op.pts
    R = np.linalg.norm(P[:, None, :] - P[None, :, :], axis=-1)
    off = ~np.eye(g.Nv, dtype=bool)
    want = np.exp(1j * w * 1.1 * R[off]) / (4 * math.pi * R[off])
    assert np.max(np.abs(K[off] - want) / np.abs(want)) < 1e-11
    assert np.allclose(np.diag(K), hb3d.cube_integral(1.1 * w, g.h) / g.h ** 3, rtol=1e-14, atol=0)


def test_tables_gradient_interpolation_converges():
    """Interpolated tau^2 and v0 of the gradient medium at random point pairs
    of [0, 0.52]^3 converge to the closed forms as n_I grows (a transposed or
    misordered node index would stay O(1) wrong)."""
    rng = np.random.default_rng(4)
    ro, rs = rng.uniform(0, 0.52, size=(40, 3)), rng.uniform(0, 0.52, size=(40, 3))
    errs = []
    for n_I in (3, 5, 7):
        tab = hb3d.build_tables3(GR, n_I, 0.52)
        To = hb3d.tensor_basis3(tab["nodes"], *ro.T)
        Ts = hb3d.tensor_basis3(tab["nodes"], *rs.T)
        t2 = np.einsum("ai,ij,aj->a", To, tab["tau2"], Ts)
        a0 = np.einsum("ai,ij,aj->a", To, tab["v0"], Ts)
        e_t2 = np.max(np.abs(t2 - hb3d.tau(GR, ro, rs) ** 2))
        e_v0 = np.max(np.abs(a0 - hb3d.v0(GR, ro, rs)) / hb3d.v0(GR, ro, rs))
        errs.append(max(e_t2, e_v0))
    assert errs[0] / errs[1] > 10 and errs[1] / errs[2] > 10 and errs[2] < 3e-4   # spectral: ~20x per 2 nodes


def test_dense_sum_is_the_matrix_product():
    """U = K (s h^3) in column chunks equals the full matrix product."""
    g = W.Grid3D(4, 0.52)
    op = hb3d.Operator3(g, hb3d.build_tables3(GR, 5, g.L), 2 * math.pi * 3, GR)
    s = W.complex_normal_sources(g.Nv, 2, 9)
    idx = np.arange(g.Nv)
    full = op.block(idx, idx) @ (s * g.h ** 3)
    assert np.allclose(hb3d.dense_apply3(op, s, chunk=7), full, rtol=1e-13, atol=0)


def test_tensor_basis_is_cardinal_at_the_nodes():
    """T_i(r^c_j) = delta_ij with the node order of the tables (x fastest):
    catches a basis whose axis order disagrees with the node layout (the 3D
    media are symmetric under x <-> z, so interpolation alone cannot)."""
    xn = 0.52 * chebyshev.nodes(3)
    P = hb3d.node_points3(xn)
    assert np.allclose(hb3d.tensor_basis3(xn, *P.T), np.eye(len(P)), atol=1e-13)
    assert np.allclose(P[1], [xn[1], xn[0], xn[0]]) and np.allclose(P[3], [xn[0], xn[1], xn[0]])
