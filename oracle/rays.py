"""Lagrangian cross-check of the HB ingredients tau and v0 (Sec. 2): rays of
the eikonal equation and the ray-tube form of the transport equation.

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
closed form v0 = B0 sqrt(g tau / sinh g tau).
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
