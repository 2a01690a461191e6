"""Tabulated HB ingredients tau^2, v0, v1 at Chebyshev node pairs (Sec. 4.1).

Test infrastructure (see ``oracle/__init__``).

The paper tabulates f(r^c_i, r^c_j) for f = tau^2, v0, v1 with one eikonal
and transport solve per source node r^c_j (Sec. 4.1, Fig. table-compute).
Here the two media used by the workloads have exact ingredients, so the
oracle evaluates them directly instead of sweeping a grid:

* homogeneous n = n0 (Sec. 5.1.1, constant media): tau = n0 |r - r0|,
  v0 = 1/(2 sqrt(pi)), v1 = 0.
* constant velocity gradient c = c0 + g z, n = 1/c (Sec. 5.1.1,
  constant-gradient media): the paper's closed form
  tau = (1/g) arccosh(1 + g^2 |r-r0|^2 / (2 c(r) c(r0))), evaluated in the
  algebraically equal form tau = (2/g) asinh(g |r-r0| / (2 sqrt(c c0))) which
  keeps full precision as r -> r0.
  The paper gives no closed form for v0, v1.  They are obtained from the
  transport recurrence Eq. equVs (d = 2) along the ray:
    s = -1:  4 tau n^2 dv0/dtau + v0 (Lap tau^2 - 4 n^2) = 0,
    s =  0:  4 tau n^2 dv1/dtau + v1  Lap tau^2          = Lap v0,
  with v0(r0) = 1/(2 sqrt(pi)) (Eq. initialv0) and v1 bounded at r0.
  In this medium the travel-time metric n^2 |dr|^2 is the hyperbolic plane
  of curvature -g^2 (tau is g^-1 times the Poincare half-plane distance of
  the closed form above), so along every ray Lap tau / n^2 = g coth(g tau)
  and Lap tau^2 = n^2 (2 + 2 g tau coth(g tau)); both transport equations
  become ODEs in tau alone.  The s = -1 equation integrates to
    v0 = (1/(2 sqrt(pi))) sqrt(g tau / sinh(g tau)),
  and, with v0 = F(tau) so that Lap v0 = n^2 (F'' + g coth(g tau) F'),
  the s = 0 equation is  4 tau v1' + (2 + 2 g tau coth g tau) v1 = Q(tau),
  Q = F'' + g coth(g tau) F', solved with the integrating factor
  mu = sqrt(tau sinh(g tau)):
    v1(T) = 1 / (4 sqrt(T sinh gT)) * int_0^T sqrt(sinh(g t)/t) Q(t) dt.
  The integral is taken with 64-point Gauss-Legendre (numpy's nodes).
  Pins (tests/test_oracle_tables.py): Cartesian finite-difference residuals
  of Eq. eikonal and Eq. equVs, the paper's Taylor recursions (Eq. recursiveT,
  Eq. recursiveB, Eq. C0), reciprocity, the g -> 0 limit, and the exact
  Green's function of this medium (see ``exact_green_gradient``).

Diagonal (i == j) entries: tau^2 = 0, v0 = B0 = 1/(2 sqrt(pi)) and v1 = C0,
the value of v1 at the source (Eq. C0).
"""
import math

import numpy as np

from . import chebyshev

B0_2D = 1.0 / (2.0 * math.sqrt(math.pi))     # Eq. initialv0, d = 2


# ------------------------------------------------------------ gradient ----
def tau_gradient(x, z, x0, z0, c0, g):
    """Closed-form travel time of the constant-gradient medium (Sec. 5.1.1)."""
    c = c0 + g * np.asarray(z, dtype=np.float64)
    cs = c0 + g * np.asarray(z0, dtype=np.float64)
    d = np.hypot(np.asarray(x, dtype=np.float64) - x0, np.asarray(z, dtype=np.float64) - z0)
    if g == 0.0:
        return d / c
    return (2.0 / g) * np.arcsinh(g * d / (2.0 * np.sqrt(c * cs)))


def _phi(u):
    """phi(u) = 1/(2u) - coth(u)/2 and phi'(u); series below u = 0.2."""
    u = np.asarray(u, dtype=np.float64)
    small = u < 0.2
    us = np.where(small, u, 0.2)
    ul = np.where(small, 1.0, u)
    u2 = us * us
    ph_s = us * (-1 / 6 + u2 * (1 / 90 + u2 * (-1 / 945 + u2 * (1 / 9450 - u2 / 93555))))
    dph_s = -1 / 6 + u2 * (1 / 30 + u2 * (-1 / 189 + u2 * (1 / 1350 - u2 / 10395)))
    ph_l = 0.5 / ul - 0.5 / np.tanh(ul)
    dph_l = -0.5 / ul**2 + 0.5 / np.sinh(ul) ** 2
    return np.where(small, ph_s, ph_l), np.where(small, dph_s, dph_l)


def v0_gradient(tau, g):
    """Solution of Eq. equVs (s = -1) along the ray: B0 sqrt(g tau / sinh g tau)."""
    tau = np.asarray(tau, dtype=np.float64)
    if g == 0.0:
        return np.full(tau.shape, B0_2D)
    u = g * tau
    ratio = np.where(u > 0, u / np.sinh(np.where(u > 0, u, 1.0)), 1.0)
    return B0_2D * np.sqrt(ratio)


def _Q_gradient(t, g):
    """Q = F'' + g coth(g t) F' with F = v0_gradient, F'/F = g phi(g t)."""
    u = g * t
    ph, dph = _phi(u)
    F = v0_gradient(t, g)
    return g * g * F * (ph * ph + dph + ph / np.tanh(u))


def v1_gradient(tau, g, nq: int = 64):
    """Bounded solution of Eq. equVs (s = 0, d = 2) along the ray."""
    tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
    if g == 0.0:
        return np.zeros(tau.shape)
    out = np.empty(tau.shape)
    xg, wg = np.polynomial.legendre.leggauss(nq)
    # limit at the source: 4 v1(0) = Q(0) = -g^2 B0 / 3  (from the ODE at tau = 0)
    v1_0 = -g * g * B0_2D / 12.0
    for idx, T in np.ndenumerate(tau):
        if T <= 0.0:
            out[idx] = v1_0
            continue
        t = 0.5 * T * (xg + 1.0)
        w = 0.5 * T * wg
        integrand = np.sqrt(np.sinh(g * t) / t) * _Q_gradient(t, g)
        out[idx] = np.sum(w * integrand) / (4.0 * math.sqrt(T * math.sinh(g * T)))
    return out


def exact_green_gradient(tau, omega, g, dps: int = 30):
    """Exact outgoing Green's function of [Lap + omega^2 n^2] u = -delta in
    the constant-gradient medium: with the hyperbolic-plane reading above,
    G = (1/2pi) Q_{-1/2 - i kappa}(cosh(g tau)), kappa = sqrt(omega^2/g^2 - 1/4).
    Needs mpmath (CPU tests only).  Used to pin the truncated ansatz Eq. babich."""
    import mpmath as mp

    mp.mp.dps = dps
    kap = mp.sqrt(mp.mpf(omega) ** 2 / mp.mpf(g) ** 2 - mp.mpf(1) / 4)
    nu = -mp.mpf(1) / 2 - 1j * kap
    return complex(mp.legenq(nu, 0, mp.cosh(mp.mpf(g) * mp.mpf(tau)), type=3) / (2 * mp.pi))


# ---------------------------------------------------------- tabulation ----
def ingredient_functions(medium):
    """Return f(x, z, x0, z0) -> (tau2, v0, v1) for observation (x, z) and
    source (x0, z0), broadcasting; exact functions of the two media."""
    if medium.kind == "homogeneous":
        n0 = medium.n0

        def f(x, z, x0, z0):
            d2 = (np.asarray(x) - x0) ** 2 + (np.asarray(z) - z0) ** 2
            t2 = n0 * n0 * d2
            return t2, np.full(np.shape(t2), B0_2D), np.zeros(np.shape(t2))
        return f
    if medium.kind == "gradient":
        c0, g = medium.c0, medium.g

        def f(x, z, x0, z0):
            t = tau_gradient(x, z, x0, z0, c0, g)
            return t * t, v0_gradient(t, g), v1_gradient(t, g).reshape(np.shape(t))
        return f
    raise NotImplementedError(
        f"no exact ingredients for medium kind {medium.kind!r}: use oracle.sweep.build_tables")


def build_tables(medium, n_I: int):
    """F^c tables (Sec. 4.1): dict with 'nodes' (n_I,), 'tau2', 'v0', 'v1'
    each (N_I, N_I) float64, row = observation node i, column = source node j,
    node index i = i2*n_I + i1."""
    xn = chebyshev.nodes(n_I)
    NI = n_I * n_I
    px = np.tile(xn, n_I)
    pz = np.repeat(xn, n_I)
    f = ingredient_functions(medium)
    X, Z = px[:, None], pz[:, None]
    X0, Z0 = px[None, :], pz[None, :]
    t2, v0, v1 = f(np.broadcast_to(X, (NI, NI)), np.broadcast_to(Z, (NI, NI)),
                   np.broadcast_to(X0, (NI, NI)), np.broadcast_to(Z0, (NI, NI)))
    t2 = np.array(t2, dtype=np.float64)
    v0 = np.array(v0, dtype=np.float64)
    v1 = np.array(v1, dtype=np.float64)
    idx = np.arange(NI)
    t2[idx, idx] = 0.0
    v0[idx, idx] = B0_2D
    if medium.kind == "gradient":
        v1[idx, idx] = v1_gradient(np.array([0.0]), medium.g)[0]
    else:
        v1[idx, idx] = 0.0
    return {"nodes": xn, "tau2": t2, "v0": v0, "v1": v1, "n_I": n_I}
