"""Scattering by a curve inclusion (Sec. 3.2): the surface operators
K^{s2s}, K^{v2s}, K^{s2v} and the total field at the cell centres
U = (K^{v2v} + K^{s2v} (K^{s2s})^{-1} K^{v2s}) I   (Eq. m_v2v_inclu).

Test infrastructure (see ``oracle/__init__``).  Dense and plain: every
operator is assembled entry by entry, the surface system is solved by
numpy's LU.

The curve C is cut into N_s straight segments with centres r^s_i and
lengths w_i; Eq. sie (u^inc = -u^sca on C) is enforced at the centres:
  K^{s2s} P = U^inc                                     (Eq. m_sie)
  K^{s2s}_ij = -g(r^s_i, r^s_j) w_j,  i != j            (Eq. s2s)
  K^{s2s}_ii = -(i w_i / 4) (1 + (2i/pi) (ln(gamma w n(r^s_i) w_i / 4) - 1)),
  U^inc = K^{v2s} I,  K^{v2s}_ij = g(r^s_i, r_j)        (Eq. m_v2s)
  U^sca = K^{s2v} P,  K^{s2v}_ij = g(r_i, r^s_j) w_j    (Eq. m_s2v)
with g = v0 f0 + v1 f1 (Eq. babich) and tau^2, v0, v1 Chebyshev-interpolated
at the points (Sec. 4.1), as for K^{v2v}.

Readings.  The diagonal of Eq. s2s is printed without the factor i in front
and with the -1 inside the logarithm's argument; it is read as the negative
of the segment integral of the local kernel (i/4) H0(w n |t|), whose
small-argument form H0(x) = 1 + (2i/pi)(ln(x/2) + gamma_E) + O(x^2 ln x)
integrates over |t| < w_i/2 to w_i (1 + (2i/pi)(ln(gamma w n w_i / 4) - 1)),
gamma = e^{gamma_E} (pinned against quadrature in tests/test_oracle_inclusion.py).
Eq. sie makes the total field vanish on C (a Dirichlet, "sound-soft"
condition) although the section names the inclusion sound-hard; the oracle
follows the equations.
"""
import math

import numpy as np

from . import chebyshev, hankel

GAMMA = math.exp(0.5772156649015329)   # e^{Euler's constant}


class Curve:
    """N_s segments: centres (N_s, 2) and lengths (N_s,)."""

    def __init__(self, centers, lengths):
        self.c = np.asarray(centers, dtype=np.float64)
        self.w = np.asarray(lengths, dtype=np.float64)

    @property
    def Ns(self):
        return len(self.w)


def arc(center, radius, ns, theta0=0.0, theta1=2 * math.pi):
    """The arc of the circle from theta0 to theta1 as ns equal chords
    (centres on the chords' midpoints, lengths the chord lengths)."""
    t = np.linspace(theta0, theta1, ns + 1)
    p = np.stack([center[0] + radius * np.cos(t), center[1] + radius * np.sin(t)], axis=1)
    return Curve(0.5 * (p[1:] + p[:-1]), np.hypot(*(p[1:] - p[:-1]).T))


def polyline(points, ns):
    """An open polygonal curve through ``points`` cut into ns segments of
    equal length (segments follow the corners)."""
    points = np.asarray(points, dtype=np.float64)
    seg = np.hypot(*(points[1:] - points[:-1]).T)
    total = seg.sum()
    s = np.linspace(0.0, total, ns + 1)
    cum = np.concatenate([[0.0], np.cumsum(seg)])

    def at(si):
        k = min(np.searchsorted(cum, si, side="right") - 1, len(seg) - 1)
        f = (si - cum[k]) / seg[k]
        return points[k] + f * (points[k + 1] - points[k])

    q = np.array([at(si) for si in s])
    # a segment that turns a corner is split there; its centre is the
    # arc-length midpoint, its length the arc length
    mids = np.array([at(0.5 * (s[i] + s[i + 1])) for i in range(ns)])
    return Curve(mids, np.diff(s))


def green(tab, omega, ro, rs):
    """g(ro_a, rs_b) for observation points ro (m, 2) and sources rs (n, 2)
    (distinct points), Eq. babich with the Chebyshev-interpolated
    ingredients (Eq. chebinterpblock)."""
    xn = tab["nodes"]
    To = chebyshev.tensor_basis(xn, ro[:, 0], ro[:, 1])
    Ts = chebyshev.tensor_basis(xn, rs[:, 0], rs[:, 1])
    t2 = chebyshev.interp_block(tab["tau2"], To, Ts)
    v0 = chebyshev.interp_block(tab["v0"], To, Ts)
    v1 = chebyshev.interp_block(tab["v1"], To, Ts)
    tau = np.sqrt(np.maximum(t2, 0.0))
    return v0 * hankel.f0(omega, tau) + v1 * hankel.f1(omega, tau)


def s2s_self(w, omega, n):
    """K^{s2s}_ii (the reading above)."""
    L = np.log(GAMMA * omega * n * w / 4.0)
    return -(0.25j * w) * (1.0 + (2j / math.pi) * (L - 1.0))


def K_s2s(tab, omega, curve, n_of):
    """Eq. s2s; n_of(x, z) gives n at the segment centres."""
    K = -green(tab, omega, curve.c, curve.c) * curve.w[None, :]
    idx = np.arange(curve.Ns)
    K[idx, idx] = s2s_self(curve.w, omega, n_of(curve.c[:, 0], curve.c[:, 1]))
    return K


def K_v2s(tab, omega, curve, cells):
    """Eq. m_v2s: g(r^s_i, r_j) for the cell centres ``cells`` (N_v, 2)."""
    return green(tab, omega, curve.c, cells)


def K_s2v(tab, omega, curve, points):
    """Eq. m_s2v: g(r_i, r^s_j) w_j for observation points (m, 2)."""
    return green(tab, omega, points, curve.c) * curve.w[None, :]


def total_field(op, curve, n_of, s, v2v=None):
    """U = K^{v2v} I + K^{s2v} (K^{s2s})^{-1} K^{v2s} I at the cell centres
    (Eq. m_v2v_inclu), I = s h^2; ``op`` an oracle.kernel.Operator (its K^{v2v}
    dense sum unless ``v2v`` gives it)."""
    from . import dense
    cells = np.stack([op.px, op.pz], axis=1)
    I = np.asarray(s) * op.h ** 2
    U_v = dense.apply(op, s) if v2v is None else v2v
    U_inc = K_v2s(op.tab, op.omega, curve, cells) @ I
    P = np.linalg.solve(K_s2s(op.tab, op.omega, curve, n_of), U_inc)
    return U_v + K_s2v(op.tab, op.omega, curve, cells) @ P, P


def circle_exact_scattered(k, center, radius, r0, r, mmax=None):
    """Exact field scattered by a circle (radius a) on which the total field
    vanishes, for the point source (i/4) H0(k |r - r0|) outside it, at
    points r outside it: by Graf's addition theorem
      u^sca(r) = -(i/4) sum_m [J_m(ka) / H_m(ka)] H_m(k rho) H_m(k rho0) e^{i m (phi - phi0)}."""
    from scipy import special
    r = np.atleast_2d(np.asarray(r, dtype=np.float64))
    d = r - np.asarray(center)
    d0 = np.asarray(r0) - np.asarray(center)
    rho, phi = np.hypot(d[:, 0], d[:, 1]), np.arctan2(d[:, 1], d[:, 0])
    rho0, phi0 = math.hypot(*d0), math.atan2(d0[1], d0[0])
    if mmax is None:
        mmax = int(k * max(rho.max(), rho0) + 40)
    out = np.zeros(len(rho), dtype=np.complex128)
    for m in range(-mmax, mmax + 1):
        coef = special.jv(m, k * radius) / special.hankel1(m, k * radius)
        out += coef * special.hankel1(m, k * rho) * special.hankel1(m, k * rho0) * np.exp(1j * m * (phi - phi0))
    return -0.25j * out
