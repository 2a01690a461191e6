"""Chebyshev low-rank interpolation of the HB ingredients (Sec. 4.1).

Test infrastructure (see ``oracle/__init__``).

Eq. chebinterp: f(r, r0) ~ sum_i sum_j T_i(r) f(r^c_i, r^c_j) T_j(r0), with the
2D tensor interpolants T_i(r) = l_{i1}(x) l_{i2}(z) and l_k the 1D Lagrange
polynomial on the n_I Chebyshev nodes of [0,1].  Eq. chebinterpblock writes a
whole m x n block as T^o F^c T^s.

Readings (the paper does not fix them): first-kind nodes
x_k = 1/2 - 1/2 cos((2k-1) pi / (2 n_I)), k = 1..n_I (ascending); the 2D node
index is i = i2 * n_I + i1 (x index fastest).
"""
import numpy as np


def nodes(n_I: int) -> np.ndarray:
    """First-kind Chebyshev nodes on [0,1], ascending."""
    k = np.arange(1, n_I + 1, dtype=np.float64)
    return 0.5 - 0.5 * np.cos((2 * k - 1) * np.pi / (2 * n_I))


def lagrange(xn: np.ndarray, x) -> np.ndarray:
    """l_k(x) = prod_{m != k} (x - x_m) / (x_k - x_m), the product form of
    Sec. 4.1.  Returns shape (len(x), n_I)."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(xn)
    L = np.ones((len(x), n))
    for k in range(n):
        for m in range(n):
            if m != k:
                L[:, k] *= (x - xn[m]) / (xn[k] - xn[m])
    return L


def tensor_basis(xn: np.ndarray, px, pz) -> np.ndarray:
    """T_i(r) = l_{i1}(x) l_{i2}(z), i = i2*n_I + i1.  Shape (len(p), n_I^2)."""
    Lx = lagrange(xn, px)
    Lz = lagrange(xn, pz)
    n = len(xn)
    return (Lz[:, :, None] * Lx[:, None, :]).reshape(len(Lx), n * n)


def interp_block(Fc: np.ndarray, To: np.ndarray, Ts: np.ndarray) -> np.ndarray:
    """Eq. chebinterpblock: F = T^o F^c T^s with T^o_{ij} = T_j(r_i) (rows =
    observation points) and T^s_{ij} = T_i(r_j) (columns = source points).
    ``To`` is (m, N_I); ``Ts`` is given as (n, N_I) and transposed here."""
    return To @ Fc @ Ts.T
