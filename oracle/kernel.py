"""Matrix entries of the discretised HB integrator K^{v2v} (Sec. 3.1).

Test infrastructure (see ``oracle/__init__``).

Off-diagonal entries (Eq. m_v2v, Eq. babich with N = 1, d = 2):
  K_ij = g(r_i, r_j) = v0 f0(omega, tau) + v1 f1(omega, tau),
with tau^2, v0, v1 Chebyshev-interpolated from the tables by the blocked
Eq. chebinterpblock, and tau = sqrt(max(tau^2, 0)) (tau^2 is interpolated,
Sec. 4.1; negative interpolated values near the diagonal are clamped).

Diagonal entries (Appendix A): the cell integral of g is approximated by
(i/4) I(r_i) with the lemma Eq. HankelIntegral2dlemma,
  I = (n0 omega)^-2 [ 8 int_0^{pi/4} R(theta) H1(R(theta)) dtheta + 4 i ],
  R(theta) = h n0 omega / (2 cos theta),  n0 = n(r_i).
Because U = K I with I_j = s_j h^2 (Eq. m_v2v), the diagonal matrix entry is
that integral divided by the cell area: K_ii = (i/4) I(r_i) / h^2.
The theta integral is scipy.integrate.quad (adaptive Gauss-Kronrod).
"""
import math

import numpy as np
from scipy import integrate, special

from . import chebyshev, hankel


class Operator:
    """Everything the entries need: grid, tables, omega, n at the cells."""

    def __init__(self, N, tables, omega, n_cells):
        self.N = N
        self.h = 1.0 / N
        self.Nv = N * N
        self.omega = float(omega)
        self.tab = tables
        self.xn = tables["nodes"]
        a = (np.arange(N) + 0.5) * self.h
        self.px = np.tile(a, N)
        self.pz = np.repeat(a, N)
        self.n_cells = np.asarray(n_cells, dtype=np.float64)
        self._self = {}

    def basis(self, idx):
        return chebyshev.tensor_basis(self.xn, self.px[idx], self.pz[idx])

    def self_term(self, i):
        n0 = float(self.n_cells[i])
        if n0 not in self._self:
            self._self[n0] = self_term(n0, self.omega, self.h)
        return self._self[n0]

    def block(self, rows, cols):
        """K[rows, cols] (natural indices), complex128, diagonal included."""
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        To = self.basis(rows)
        Ts = self.basis(cols)
        t2 = chebyshev.interp_block(self.tab["tau2"], To, Ts)
        v0 = chebyshev.interp_block(self.tab["v0"], To, Ts)
        v1 = chebyshev.interp_block(self.tab["v1"], To, Ts)
        tau = np.sqrt(np.maximum(t2, 0.0))
        diag = rows[:, None] == cols[None, :]
        tau_safe = np.where(diag, 1.0, tau)
        K = v0 * hankel.f0(self.omega, tau_safe) + v1 * hankel.f1(self.omega, tau_safe)
        ii, jj = np.nonzero(diag)
        for a, b in zip(ii, jj):
            K[a, b] = self.self_term(rows[a])
        return K


def self_term(n0, omega, h):
    """K_ii = (i/4) I / h^2 with I from Eq. HankelIntegral2dlemma."""
    k = h * n0 * omega / 2.0

    def re(th):
        R = k / math.cos(th)
        return R * special.hankel1(1, R).real

    def im(th):
        R = k / math.cos(th)
        return R * special.hankel1(1, R).imag

    opts = dict(epsabs=0.0, epsrel=2e-14, limit=200)
    Ire = integrate.quad(re, 0.0, math.pi / 4, **opts)[0]
    Iim = integrate.quad(im, 0.0, math.pi / 4, **opts)[0]
    I = (8.0 * (Ire + 1j * Iim) + 4.0j) / (n0 * omega) ** 2
    return 0.25j * I / h**2
