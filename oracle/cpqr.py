"""Interpolative decomposition by column-pivoted QR (Sec. 4.2.1, Eq. ID).

Test infrastructure (see ``oracle/__init__``).

K(tau, nu) ~ K(tau, nu_bar) V_{tau,nu}: the skeleton columns nu_bar are the
first r pivots of a rank-revealing (column-pivoted Householder) QR with a
relative tolerance, and V = [I | R11^-1 R12] Pi^T.

Readings (the paper says only "rank-revealing QR with a relative tolerance"):
* step k pivots on the trailing column of largest 2-norm, the norms
  recomputed from the current trailing matrix (no downdating); columns whose
  norm comes within TIE |R_00| of the largest (within a factor 1 - TIE at
  step 0) count as tied, and the lowest current position among them wins.
  Blocks of a regular grid hold columns that are mirror images of one
  another, whose norms agree in exact arithmetic and differ only by rounding;
  with the window, two implementations that round differently still pick the
  same pivot (a difference in the last bits of a norm changes nothing unless
  it straddles the window's edge);
* the rank is the first k >= 1 with |R_kk| <= eps |R_00| (k = min(m, n) if
  none); an all-zero matrix gets rank 1;
* the skeleton list is in pivot order.
"""
import numpy as np
from scipy.linalg import solve_triangular


TIE = 1e-12   # tie window, relative to |R_00|


def pivot(norms, k, r00):
    """Position (within the trailing columns) of the step-k pivot and the
    largest trailing norm: the lowest position whose norm is at least the
    largest minus TIE |R_00| (at step 0, r00 unknown: the largest times
    1 - TIE)."""
    top = float(np.max(norms))
    thr = top * (1.0 - TIE) if k == 0 else top - TIE * r00
    return int(np.nonzero(norms >= thr)[0][0]), top


def cpqr_id(A, eps):
    """Return (skel, V, R_diag): A[:, skel] @ V ~ A, V is r x n."""
    A = np.array(A, dtype=np.complex128, copy=True)
    m, n = A.shape
    perm = np.arange(n)
    kmax = min(m, n)
    rdiag = []
    r = kmax
    for k in range(kmax):
        norms = np.sqrt(np.sum(np.abs(A[k:, k:]) ** 2, axis=0))
        q, top = pivot(norms, k, r00 if k else 0.0)
        p = k + q
        if k == 0:
            r00 = norms[q]
            if top == 0.0:
                r = 1
                rdiag.append(0.0)
                break
        elif top <= eps * r00:
            r = k
            break
        if p != k:
            A[:, [k, p]] = A[:, [p, k]]
            perm[[k, p]] = perm[[p, k]]
        # Householder reflector H = I - 2 v v^H / (v^H v) mapping x to -e^{i arg x0}|x| e1
        x = A[k:, k].copy()
        alpha = norms[p - k]
        phase = x[0] / abs(x[0]) if x[0] != 0 else 1.0
        v = x.copy()
        v[0] += phase * alpha
        vv = np.vdot(v, v).real
        if vv > 0.0:
            A[k:, k:] -= np.outer(v, (2.0 / vv) * (v.conj() @ A[k:, k:]))
        rdiag.append(abs(A[k, k]))
    R11 = np.triu(A[:r, :r])
    R12 = A[:r, r:]
    if r > 0 and n > r and rdiag[0] > 0.0:
        T = solve_triangular(R11, R12, lower=False)
    else:
        T = np.zeros((r, n - r), dtype=np.complex128)
    Vp = np.concatenate([np.eye(r, dtype=np.complex128), T], axis=1)
    V = np.empty((r, n), dtype=np.complex128)
    V[:, perm] = Vp
    return perm[:r].copy(), V, np.array(rdiag)
