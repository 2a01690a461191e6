"""3D ingredients of the HB integrator: the ansatz with d = 3 (Sec. 2,
Eq. hb, Eq. termf, Eq. babich), the paper's 3D media (Sec. 5.1.2), exact
ingredients and the exact Green's function of the 3D constant-gradient
medium, and the 3D self term (Appendix A.2).  Groundwork for a 3D path; no
GPU code uses it yet.

Test infrastructure (see ``oracle/__init__``).

Ansatz.  With d = 3 the terms are f_q, q = s - 1/2 (Eq. hb), evaluated
literally from Eq. termf with scipy's half-order Hankel functions; they are
elementary: f_{-1/2} = e^{i w tau} / (2 tau) and f_{1/2} = i e^{i w tau} / w
(pinned in tests/test_oracle_3d.py).  Eq. initialv0 gives v0 = n0 / (2 pi)
at the source, so the leading term near the source is n0 e^{i w tau} /
(4 pi tau) (Eq. babich1).

Constant-gradient medium n = a / (c - y) (velocity linear in y, gradient
-1/a).  Its travel-time metric n^2 |dr|^2 = a^2 |dr|^2 / (c - y)^2 is the
hyperbolic upper half-space scaled by a, so tau = a d with
cosh d = 1 + R^2 / (2 P), R = |r - r0|, P = (c - y)(c - y0) (the closed
form the paper prints, with |G0| = 1/a), computed as d = 2 asinh(R / (2 sqrt P))
to keep digits at small R.  Readings (the paper calls v0, v1 of this medium
unknown and solves for them numerically):
  * ray tubes of hyperbolic space have area (a sinh d)^2 per unit solid angle
    in the travel-time metric, and Eq. equVs with s = -1, d = 3 reads
    d ln v0 / d tau = -Lap tau / (2 n^2) + 1 / tau along a ray, which with
    the tube's flux balance d ln(n A) / d tau = Lap tau / n^2 integrates to
    v0 = sqrt(n n0) / (2 pi) * d / sinh d   (Eq. initialv0 fixes the constant);
  * the exact Green's function (Sec. 5.1.2, Holford)
    G = sqrt(|y - c| |y0 - c|) / (2 pi R R') exp(2 i sqrt(a^2 w^2 - 1/4) artanh(R / R')),
    R' the distance to the image of r0 in the plane y = c, has
    2 artanh(R / R') = d and amplitude v0 / (2 tau) exactly; its phase
    sqrt(a^2 w^2 - 1/4) d = w tau - d / (8 a w) + O(w^-3), and matching the
    1/w term of the N = 1 ansatz gives v1 = -v0 / (16 a^2).
Both are pinned by finite-difference residuals of Eq. eikonalnormal and
Eq. equVs (s = -1 and s = 0, d = 3) and by the error orders w^-1 (N = 0)
and w^-2 (N = 1) against G.

3D self term (Appendix A.2): the cell-centred entry is the integral of the
leading term n0 e^{i w tau} / (4 pi tau), tau = n0 |r - r_i|, over the cube of
side h around r_i, divided by h^3 (the 3D counterpart of the 2D reading
K_ii = (cell integral of g) / h^2, since U = K (s h^d)).  Written out: the
radial integral of e^{i k r} r in closed form, k = n0 w, times the angular
integral over the 48 congruent pieces of the cube, by adaptive quadrature.

Tables and entries (Sec. 4.1 in 3D): tau^2, v0, v1 at all pairs of the n_I^3
tensor Chebyshev nodes of the box (row = observation node, node index
i = (i3 n_I + i2) n_I + i1, x fastest), interpolated at cell centres by
T^o F^c T^s with T_i(r) = l_{i1}(x) l_{i2}(y) l_{i3}(z) (Eq. chebinterpblock);
the dense sum U = K I, I = s h^3, on N^3 cells (Eq. m_v2v with d = 3).
"""
import math

import numpy as np
from scipy import integrate, special

from . import chebyshev


# ------------------------------------------------------------- f_q, d = 3 ----
def f_q(q, omega, tau):
    """Eq. termf: i (sqrt(pi)/2) e^{i q pi} (2 tau / omega)^q H^(1)_q(omega tau)."""
    tau = np.asarray(tau, dtype=np.float64)
    return (1j * math.sqrt(math.pi) / 2.0 * np.exp(1j * q * math.pi) * (2.0 * tau / omega) ** q
            * special.hankel1(q, omega * tau))


def kernel(omega, tau, vs):
    """Eq. babich with d = 3: sum_s v_s f_{s - 1/2}(omega, tau), vs = (v0, v1, ...)."""
    return sum(v * f_q(s - 0.5, omega, tau) for s, v in enumerate(vs))


# -------------------------------------------- constant-gradient medium ----
def _P(medium, y, y0):
    return (medium.c - np.asarray(y)) * (medium.c - np.asarray(y0))


def hyperbolic_distance(medium, r, r0):
    """d with cosh d = 1 + R^2 / (2 (c - y)(c - y0)); r, r0 arrays (..., 3)."""
    r, r0 = np.asarray(r, dtype=np.float64), np.asarray(r0, dtype=np.float64)
    R = np.linalg.norm(r - r0, axis=-1)
    return 2.0 * np.arcsinh(R / (2.0 * np.sqrt(_P(medium, r[..., 1], r0[..., 1]))))


def tau(medium, r, r0):
    """Travel time: n0 |r - r0| (homogeneous) or a d (gradient)."""
    r, r0 = np.asarray(r, dtype=np.float64), np.asarray(r0, dtype=np.float64)
    if medium.kind == "homogeneous":
        return medium.n0 * np.linalg.norm(r - r0, axis=-1)
    if medium.kind == "gradient":
        return medium.a * hyperbolic_distance(medium, r, r0)
    raise NotImplementedError(medium.kind)


def v0(medium, r, r0):
    """n0 / (2 pi) (homogeneous); sqrt(n n0) / (2 pi) d / sinh d (gradient)."""
    r, r0 = np.asarray(r, dtype=np.float64), np.asarray(r0, dtype=np.float64)
    if medium.kind == "homogeneous":
        return np.full(np.broadcast(r[..., 0], r0[..., 0]).shape, medium.n0 / (2.0 * math.pi))
    if medium.kind == "gradient":
        d = hyperbolic_distance(medium, r, r0)
        n = medium.n(r[..., 0], r[..., 1], r[..., 2])
        n0 = medium.n(r0[..., 0], r0[..., 1], r0[..., 2])
        ratio = np.where(d > 0, d / np.sinh(np.where(d > 0, d, 1.0)), 1.0)
        return np.sqrt(n * n0) / (2.0 * math.pi) * ratio
    raise NotImplementedError(medium.kind)


def v1(medium, r, r0):
    """0 (homogeneous: Lap v0 = 0); -v0 / (16 a^2) (gradient)."""
    if medium.kind == "homogeneous":
        return 0.0 * v0(medium, r, r0)
    if medium.kind == "gradient":
        return -v0(medium, r, r0) / (16.0 * medium.a ** 2)
    raise NotImplementedError(medium.kind)


def exact_green(medium, omega, r, r0):
    """The exact Green's function of Sec. 5.1.2 (gradient medium), or
    e^{i w n0 R} / (4 pi R) (homogeneous)."""
    r, r0 = np.asarray(r, dtype=np.float64), np.asarray(r0, dtype=np.float64)
    R = np.linalg.norm(r - r0, axis=-1)
    if medium.kind == "homogeneous":
        return np.exp(1j * omega * medium.n0 * R) / (4.0 * math.pi * R)
    if medium.kind == "gradient":
        img = r0.copy()
        img[..., 1] = 2.0 * medium.c - r0[..., 1]
        Rp = np.linalg.norm(r - img, axis=-1)
        amp = np.sqrt(np.abs(r[..., 1] - medium.c) * np.abs(r0[..., 1] - medium.c)) / (2.0 * math.pi * R * Rp)
        return amp * np.exp(2j * math.sqrt(medium.a ** 2 * omega ** 2 - 0.25) * np.arctanh(R / Rp))
    raise NotImplementedError(medium.kind)


def green(medium, omega, r, r0, N=1):
    """The truncated ansatz g = sum_{s <= N} v_s f_{s - 1/2} with the exact
    ingredients of the medium (no tables)."""
    vs = [v0(medium, r, r0), v1(medium, r, r0)][:N + 1]
    return kernel(omega, tau(medium, r, r0), vs)


# ----------------------------------------------------------- self term ----
def _radial(k, R):
    """int_0^R e^{i k r} r dr = (e^{i k R}(1 - i k R) - 1) / k^2; its series
    sum_{n >= 2} (1 - n)/n! (i k R)^n / k^2 where k R is small."""
    x = k * R
    if x < 1e-2:
        out, term = 0.0j, 1.0 + 0j
        for n in range(1, 12):
            term *= 1j * x / n                       # (i x)^n / n!
            if n >= 2:
                out += (1 - n) * term
        return out * R * R / (x * x) if x > 0 else 0.5 * R * R
    return (np.exp(1j * x) * (1.0 - 1j * x) - 1.0) / (k * k)


def cube_integral(k, h):
    """I = int over the cube of side h centred at 0 of e^{i k r} / (4 pi r) dV:
    I = (1/4pi) int_{S2} int_0^{r1(khat)} e^{i k r} r dr dOmega, over 48
    congruent pieces: the face z = h/2 with 0 <= y <= x <= h/2, where
    dOmega = (h/2) dx dy / rho^3 and r1 = rho = |(x, y, h/2)|."""
    b = h / 2.0

    def f(y, x, part):
        rho = math.sqrt(x * x + y * y + b * b)
        v = _radial(k, rho) * b / rho ** 3
        return v.real if part == 0 else v.imag

    opts = dict(epsabs=0.0, epsrel=1e-12)
    re = integrate.dblquad(lambda y, x: f(y, x, 0), 0.0, b, 0.0, lambda x: x, **opts)[0]
    im = integrate.dblquad(lambda y, x: f(y, x, 1), 0.0, b, 0.0, lambda x: x, **opts)[0]
    return 48.0 / (4.0 * math.pi) * (re + 1j * im)


def self_term(n0, omega, h):
    """K_ii = (1/h^3) int_cube n0 e^{i w tau} / (4 pi tau) dV, tau = n0 r."""
    return cube_integral(n0 * omega, h) / h ** 3


# ------------------------------------------------ tables and entries ----
def tensor_basis3(xn, px, py, pz):
    """T_i(r) = l_{i1}(x) l_{i2}(y) l_{i3}(z), i = (i3 n_I + i2) n_I + i1;
    shape (len(p), n_I^3)."""
    Lx, Ly, Lz = (chebyshev.lagrange(xn, p) for p in (px, py, pz))
    n = len(xn)
    return (Lz[:, :, None, None] * Ly[:, None, :, None] * Lx[:, None, None, :]).reshape(len(Lx), n ** 3)


def node_points3(xn):
    """The n_I^3 tensor nodes (x fastest), shape (n_I^3, 3)."""
    Z, Y, X = np.meshgrid(xn, xn, xn, indexing="ij")
    return np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], axis=1)


def build_tables3(medium, n_I, L):
    """tau^2, v0, v1 at all node pairs of the box [0, L]^3 from the exact
    ingredients (the diagonal: tau^2 = 0, v0 = n0 / (2 pi), v1 its limit)."""
    xn = L * chebyshev.nodes(n_I)
    P = node_points3(xn)
    r, r0 = P[:, None, :], P[None, :, :]
    return {"nodes": xn, "n_I": n_I, "L": L, "tau2": tau(medium, r, r0) ** 2,
            "v0": v0(medium, r, r0), "v1": v1(medium, r, r0)}


class Operator3:
    """K on the N^3 cell centres of a Grid3D: interpolated ingredients off the
    diagonal (Eq. chebinterpblock, Eq. babich with d = 3, N = 1), the 3D self
    term on it."""

    def __init__(self, grid, tab, omega, medium):
        self.grid, self.tab, self.omega, self.medium = grid, tab, omega, medium
        self.h, self.Nv = grid.h, grid.Nv
        x, y, z = grid.centroids()
        self.pts = np.stack([x, y, z], axis=1)
        self.n_cells = medium.n(x, y, z)
        self._self = {}

    def self_term(self, i):
        n0 = float(self.n_cells[i])
        if n0 not in self._self:
            self._self[n0] = self_term(n0, self.omega, self.h)
        return self._self[n0]

    def block(self, rows, cols):
        rows, cols = np.asarray(rows), np.asarray(cols)
        xn = self.tab["nodes"]
        To = tensor_basis3(xn, *self.pts[rows].T)
        Ts = tensor_basis3(xn, *self.pts[cols].T)
        t2, a0, a1 = (chebyshev.interp_block(self.tab[q], To, Ts) for q in ("tau2", "v0", "v1"))
        diag = rows[:, None] == cols[None, :]
        t = np.where(diag, 1.0, np.sqrt(np.maximum(t2, 0.0)))
        K = kernel(self.omega, t, (a0, a1))
        for a, b in zip(*np.nonzero(diag)):
            K[a, b] = self.self_term(rows[a])
        return K


def dense_apply3(op, s, rows=None, chunk=512):
    """U_i = sum_j K_ij I_j, I = s h^3 (Eq. m_v2v, d = 3)."""
    s = np.asarray(s, dtype=np.complex128)
    s = s[:, None] if s.ndim == 1 else s
    rows = np.arange(op.Nv) if rows is None else np.asarray(rows)
    I = s * op.h ** 3
    U = np.zeros((len(rows), s.shape[1]), dtype=np.complex128)
    for c0 in range(0, op.Nv, chunk):
        cols = np.arange(c0, min(op.Nv, c0 + chunk))
        U += op.block(rows, cols) @ I[cols]
    return U
