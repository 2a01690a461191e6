"""Lagrangian cross-check of the HB ingredients tau, v0 and v1 (Sec. 2): rays
of the eikonal equation and the ray-tube form of the transport equations.

Test infrastructure (see ``oracle/__init__``); independent of ``sweep``
(no mesh, no Taylor boxes), used to pin the sweeping builder's lens tables.

Rays of |grad tau| = n in the travel-time parameter: dx/dtau = p / n^2,
dp/dtau = grad n / n, |p| = n, from the source r0 with initial direction
theta (classical RK4, vectorised over rays).  A target r is reached by
Newton's method on (theta, T) for x(T; theta) = r.

Amplitude: along a ray, Eq. equVs with s = -1 (d = 2) reads
d ln v0 / dtau = -Lap tau / (2 n^2) + 1 / (2 tau), while the geometrical
spreading J = |dx/dtheta| at fixed tau (ray-tube width per unit angle)
obeys d ln (n J) / dtau = Lap tau / n^2 (flux conservation of the tube).
Hence v0 = (1 / (2 sqrt(pi))) sqrt(tau / (n J)), the constant fixed by
Eq. initialv0 (near the source tau ~ n0 rho and J ~ rho).  In the
constant-gradient medium n J = sinh(g tau) / g and this is the oracle's
closed form v0 = B0 sqrt(g tau / sinh g tau).  v1 follows from the s = 0
equation along the same ray (``v1_along_ray``).
"""
import math

import numpy as np

B0_2D = 1.0 / (2.0 * math.sqrt(math.pi))


def _n_grad(medium, x, z):
    """n and grad n of the medium at arrays (x, z)."""
    if medium.kind == "gradient":
        c = medium.c0 + medium.g * z
        n = 1.0 / c
        return n, np.zeros_like(x), -medium.g * n * n
    if medium.kind == "lens":
        a, w = medium.amp, medium.w
        dx, dz = x - medium.center[0], z - medium.center[1]
        e = a * np.exp(-(dx * dx + dz * dz) / (w * w))
        return 1.0 + e, -2.0 * dx / (w * w) * e, -2.0 * dz / (w * w) * e
    if medium.kind == "homogeneous":
        return np.full_like(x, medium.n0), np.zeros_like(x), np.zeros_like(x)
    raise NotImplementedError(medium.kind)


def trace(medium, x0, z0, theta, T, nsteps=400):
    """Ray positions and momenta at tau = T (arrays over rays)."""
    theta = np.asarray(theta, dtype=np.float64)
    T = np.broadcast_to(np.asarray(T, dtype=np.float64), theta.shape)
    n0, _, _ = _n_grad(medium, np.full(theta.shape, float(x0)), np.full(theta.shape, float(z0)))
    y = np.stack([np.full(theta.shape, float(x0)), np.full(theta.shape, float(z0)),
                  n0 * np.cos(theta), n0 * np.sin(theta)])
    h = T / nsteps

    def f(y):
        n, nx, nz = _n_grad(medium, y[0], y[1])
        n2 = n * n
        return np.stack([y[2] / n2, y[3] / n2, nx / n, nz / n])

    for _ in range(nsteps):
        k1 = f(y)
        k2 = f(y + 0.5 * h * k1)
        k3 = f(y + 0.5 * h * k2)
        k4 = f(y + h * k3)
        y = y + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return y


def tau_v0(medium, x0, z0, x, z, nsteps=400, dtheta=1e-5, iters=30, tol=1e-13):
    """tau and v0 at targets (x, z) (arrays) from the source (x0, z0), by
    shooting; returns (tau, v0, residual |x(T; theta) - r|)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    n0, _, _ = _n_grad(medium, np.array([float(x0)]), np.array([float(z0)]))
    th = np.arctan2(z - z0, x - x0)
    T = n0[0] * np.hypot(x - x0, z - z0)
    for _ in range(iters):
        y = trace(medium, x0, z0, th, T, nsteps)
        yp = trace(medium, x0, z0, th + dtheta, T, nsteps)
        ym = trace(medium, x0, z0, th - dtheta, T, nsteps)
        n, _, _ = _n_grad(medium, y[0], y[1])
        rx, rz = y[0] - x, y[1] - z
        # Jacobian of (x, z) in (theta, T)
        a11, a21 = (yp[0] - ym[0]) / (2 * dtheta), (yp[1] - ym[1]) / (2 * dtheta)
        a12, a22 = y[2] / (n * n), y[3] / (n * n)
        det = a11 * a22 - a12 * a21
        dth = (a22 * rx - a12 * rz) / det
        dT = (-a21 * rx + a11 * rz) / det
        th = th - dth
        T = T - dT
        if np.max(np.hypot(rx, rz)) < tol:
            break
    y = trace(medium, x0, z0, th, T, nsteps)
    yp = trace(medium, x0, z0, th + dtheta, T, nsteps)
    ym = trace(medium, x0, z0, th - dtheta, T, nsteps)
    n, _, _ = _n_grad(medium, y[0], y[1])
    J = np.hypot(yp[0] - ym[0], yp[1] - ym[1]) / (2 * dtheta)
    v0 = B0_2D * np.sqrt(T / (n * J))
    return T, v0, np.hypot(y[0] - x, y[1] - z)


def v1_along_ray(medium, x0, z0, x, z, nq=24, delta=1e-2, nsteps=400):
    """v1 at targets (x, z) from the source (x0, z0) by the ray form of
    Eq. equVs with s = 0 (d = 2): with Lap tau^2 = 2 n^2 + 2 tau Lap tau and
    d ln(n J)/dtau = Lap tau / n^2 the integrating factor is mu = sqrt(tau n J):
        v1(T) = (1 / mu(T)) int_0^T mu(t) Lap v0(x(t)) / (4 t n(x(t))^2) dt,
    the bounded solution.  Gauss-Legendre in t (nq nodes); Lap v0 by the
    fourth-order 9-point cross stencil of spacing delta on v0 from tau_v0."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    z = np.atleast_1d(np.asarray(z, dtype=np.float64))
    m = len(x)
    # the ray to each target: initial angle and travel time
    n0, _, _ = _n_grad(medium, np.array([float(x0)]), np.array([float(z0)]))
    th = np.arctan2(z - z0, x - x0)
    T = n0[0] * np.hypot(x - x0, z - z0)
    dth = 1e-5
    for _ in range(30):
        y = trace(medium, x0, z0, th, T, nsteps)
        yp = trace(medium, x0, z0, th + dth, T, nsteps)
        ym = trace(medium, x0, z0, th - dth, T, nsteps)
        n, _, _ = _n_grad(medium, y[0], y[1])
        rx, rz = y[0] - x, y[1] - z
        a11, a21 = (yp[0] - ym[0]) / (2 * dth), (yp[1] - ym[1]) / (2 * dth)
        a12, a22 = y[2] / (n * n), y[3] / (n * n)
        det = a11 * a22 - a12 * a21
        th = th - (a22 * rx - a12 * rz) / det
        T = T - (-a21 * rx + a11 * rz) / det
        if np.max(np.hypot(rx, rz)) < 1e-13:
            break
    xg, wg = np.polynomial.legendre.leggauss(nq)
    t = 0.5 * T[:, None] * (xg[None, :] + 1.0)           # m x nq
    w = 0.5 * T[:, None] * wg[None, :]
    thq = np.repeat(th[:, None], nq, axis=1)
    tf, thf = t.reshape(-1), thq.reshape(-1)
    yq = trace(medium, x0, z0, thf, tf, nsteps)
    yqp = trace(medium, x0, z0, thf + dth, tf, nsteps)
    yqm = trace(medium, x0, z0, thf - dth, tf, nsteps)
    nq_, _, _ = _n_grad(medium, yq[0], yq[1])
    Jq = np.hypot(yqp[0] - yqm[0], yqp[1] - yqm[1]) / (2 * dth)
    # Lap v0 at the quadrature points: v0 at the point and at +-delta,
    # +-2 delta along each axis
    px, pz = yq[0], yq[1]
    offs = [(0, 0), (1, 0), (-1, 0), (2, 0), (-2, 0), (0, 1), (0, -1), (0, 2), (0, -2)]
    sx = np.concatenate([px + a * delta for a, _ in offs])
    sz = np.concatenate([pz + b * delta for _, b in offs])
    _, v0s, _ = tau_v0(medium, x0, z0, sx, sz, nsteps, dtheta=1e-4)
    k = len(px)
    v = [v0s[i * k:(i + 1) * k] for i in range(len(offs))]
    lap = ((-v[3] + 16 * v[1] - 30 * v[0] + 16 * v[2] - v[4]) +
           (-v[7] + 16 * v[5] - 30 * v[0] + 16 * v[6] - v[8])) / (12.0 * delta * delta)
    mu = np.sqrt(tf * nq_ * Jq)
    integrand = (mu * lap / (4.0 * tf * nq_ * nq_)).reshape(m, nq)
    nT, _, _ = _n_grad(medium, x, z)
    yT = trace(medium, x0, z0, th, T, nsteps)
    yTp = trace(medium, x0, z0, th + dth, T, nsteps)
    yTm = trace(medium, x0, z0, th - dth, T, nsteps)
    JT = np.hypot(yTp[0] - yTm[0], yTp[1] - yTm[1]) / (2 * dth)
    return np.sum(w * integrand, axis=1) / np.sqrt(T * nT * JT)
