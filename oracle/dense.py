"""Dense HB sums (Sec. 3.1, Eq. m_v2v) and their adjoint.

Test infrastructure (see ``oracle/__init__``).

apply:   U_i = sum_j K_ij I_j,  I_j = s_j h^2        (u = A s, A = h^2 K)
adjoint: S_j = h^2 sum_i conj(K_ij) U_i              (s = A^H u)
Rows (or columns for the adjoint) may be a subset; the sum is always over
all N_v cells, taken in column chunks of the full operator.
"""
import numpy as np


def apply(op, s, rows=None, chunk=1024):
    s = np.asarray(s, dtype=np.complex128)
    if s.ndim == 1:
        s = s[:, None]
    rows = np.arange(op.Nv) if rows is None else np.asarray(rows)
    I = s * op.h**2
    U = np.zeros((len(rows), s.shape[1]), dtype=np.complex128)
    for c0 in range(0, op.Nv, chunk):
        cols = np.arange(c0, min(op.Nv, c0 + chunk))
        U += op.block(rows, cols) @ I[cols]
    return U


def adjoint(op, u, cols=None, chunk=1024):
    u = np.asarray(u, dtype=np.complex128)
    if u.ndim == 1:
        u = u[:, None]
    cols = np.arange(op.Nv) if cols is None else np.asarray(cols)
    S = np.zeros((len(cols), u.shape[1]), dtype=np.complex128)
    for r0 in range(0, op.Nv, chunk):
        rows = np.arange(r0, min(op.Nv, r0 + chunk))
        S += op.block(rows, cols).conj().T @ u[rows]
    return S * op.h**2
