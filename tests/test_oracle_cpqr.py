"""Pins of oracle.cpqr (Eq. ID) against its definition and LAPACK's geqp3."""
import numpy as np
import scipy.linalg as sl

from oracle import cpqr
from paper_2210_02698_gb300 import workloads as W


def test_reconstruction_rank_and_identity_columns():
    A = W.random_id_matrices(4, 90, 40, 30, 0.55, seed=5)
    for b in range(4):
        M = A[b].T
        eps = 1e-6
        sk, V, rd = cpqr.cpqr_id(M, eps)
        r = len(sk)
        assert V.shape == (r, 40)
        assert np.max(np.abs(V[:, sk] - np.eye(r))) < 1e-12
        err = np.linalg.norm(M - M[:, sk] @ V, 2)
        assert err < 50 * eps * np.linalg.norm(M, 2)
        # the truncation rule: |R_rr| <= eps |R_00| < |R_(r-1)(r-1)|
        assert rd[-1] > eps * rd[0]
        s = np.linalg.svd(M, compute_uv=False)
        assert s[r] < 100 * eps * s[0]


def test_pivots_match_lapack_geqp3():
    A = W.random_id_matrices(3, 60, 25, 25, 0.7, seed=9)
    for b in range(3):
        M = A[b].T
        sk, V, rd = cpqr.cpqr_id(M, 0.0)
        _, R, P = sl.qr(M, pivoting=True, mode="economic")
        assert list(sk) == list(P[:len(sk)])
        assert np.allclose(rd, np.abs(np.diag(R))[:len(rd)], rtol=1e-10)


def test_ties_and_degenerate_cases():
    rng = np.random.default_rng(3)
    a = rng.standard_normal(10) + 1j * rng.standard_normal(10)
    M = np.stack([a, a, 0.5 * a], axis=1)
    sk, V, _ = cpqr.cpqr_id(M, 1e-12)
    assert list(sk) == [0]                       # exact tie -> lowest index
    assert np.allclose(M[:, sk] @ V, M)
    Z = np.zeros((5, 4), dtype=complex)
    sk, V, _ = cpqr.cpqr_id(Z, 1e-6)
    assert len(sk) == 1 and np.allclose(Z[:, sk] @ V, 0)
    one = rng.standard_normal((1, 6)) + 0j
    sk, V, _ = cpqr.cpqr_id(one, 1e-6)
    assert len(sk) == 1 and np.allclose(one[:, sk] @ V, one)


def test_tie_window_picks_the_lowest_position():
    """Columns whose norms agree to within TIE |R_00| are tied and the lowest
    position wins; a gap larger than the window is a real difference.  The
    window is measured against |R_00|, not against the current largest norm
    (step 1 below: a relative gap of 5e-12 against the column's own norm, but
    half the window against |R_00| = 10)."""
    T = cpqr.TIE
    rng = np.random.default_rng(17)
    a = rng.standard_normal(6) + 1j * rng.standard_normal(6)
    a /= np.linalg.norm(a)
    # step 0: the first column is smaller by half the window -> still chosen
    M = np.stack([a * (1 - 0.5 * T), a, 0.1 * a[::-1]], axis=1)
    assert cpqr.cpqr_id(M, 0.0)[0][0] == 0
    # ... smaller by three windows -> the larger second column wins
    M = np.stack([a * (1 - 3 * T), a, 0.1 * a[::-1]], axis=1)
    assert cpqr.cpqr_id(M, 0.0)[0][0] == 1
    # step 1: after the big first column, y (position 1) trails x (position 2)
    # by 0.5 TIE |R_00| in absolute terms -> y; by 2 TIE |R_00| -> x
    e0 = np.zeros(5, dtype=complex)
    e0[0] = 10.0
    x = np.zeros(5, dtype=complex)
    x[1:] = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    x /= np.linalg.norm(x)
    y = np.zeros(5, dtype=complex)
    y[1:] = np.roll(x[1:], 1) * np.exp(0.3j)                 # same norm, other direction
    for gap, want in ((0.5, 1), (2.0, 2)):
        M = np.stack([e0, y * (1 - gap * T * 10.0), x], axis=1)
        sk = cpqr.cpqr_id(M, 0.0)[0]
        assert sk[0] == 0 and sk[1] == want, (gap, sk)
    # the pivot helper itself
    norms = np.array([1.0, 1.0 - 0.4 * T, 1.0 + 0.4 * T, 0.5])
    assert cpqr.pivot(norms, 0, 0.0) == (0, 1.0 + 0.4 * T)
    assert cpqr.pivot(norms[1:], 1, 1.0)[0] == 0
