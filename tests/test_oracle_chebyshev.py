"""Pins of oracle.chebyshev (Sec. 4.1, Eq. chebinterp, Eq. chebinterpblock)."""
import numpy as np

from oracle import chebyshev


def test_nodes_are_shifted_chebyshev_zeros():
    for n in (3, 7, 16):
        x = chebyshev.nodes(n)
        assert np.all(np.diff(x) > 0) and x[0] > 0 and x[-1] < 1
        # zeros of T_n(2x - 1) = cos(n arccos(2x - 1))
        assert np.max(np.abs(np.cos(n * np.arccos(2 * x - 1)))) < 1e-13


def test_lagrange_cardinal_and_partition_of_unity():
    x = chebyshev.nodes(16)
    L = chebyshev.lagrange(x, x)
    assert np.max(np.abs(L - np.eye(16))) < 1e-14
    t = np.linspace(0, 1, 101)
    assert np.max(np.abs(chebyshev.lagrange(x, t).sum(axis=1) - 1)) < 1e-12


def test_lagrange_reproduces_polynomials_below_order():
    x = chebyshev.nodes(12)
    rng = np.random.default_rng(1)
    c = rng.standard_normal(12)          # degree 11 < n_I
    t = np.linspace(0, 1, 57)
    interp = chebyshev.lagrange(x, t) @ np.polyval(c, x)
    assert np.max(np.abs(interp - np.polyval(c, t))) < 1e-10


def test_block_form_equals_double_sum_of_eq_chebinterp():
    # brute-force double sum sum_i sum_j T_i(r) F_ij T_j(r0) on a tiny case
    n = 3
    xn = chebyshev.nodes(n)
    rng = np.random.default_rng(2)
    Fc = rng.standard_normal((n * n, n * n))
    obs = rng.uniform(0, 1, (4, 2))
    src = rng.uniform(0, 1, (5, 2))
    To = chebyshev.tensor_basis(xn, obs[:, 0], obs[:, 1])
    Ts = chebyshev.tensor_basis(xn, src[:, 0], src[:, 1])
    blk = chebyshev.interp_block(Fc, To, Ts)

    def l1(k, t):
        return np.prod([(t - xn[m]) / (xn[k] - xn[m]) for m in range(n) if m != k])

    for a in range(4):
        for b in range(5):
            s = 0.0
            for i1 in range(n):
                for i2 in range(n):
                    for j1 in range(n):
                        for j2 in range(n):
                            Ti = l1(i1, obs[a, 0]) * l1(i2, obs[a, 1])
                            Tj = l1(j1, src[b, 0]) * l1(j2, src[b, 1])
                            s += Ti * Fc[i2 * n + i1, j2 * n + j1] * Tj
            assert abs(s - blk[a, b]) < 1e-12


def test_squared_distance_is_reproduced_exactly():
    # |r - r0|^2 has degree 2 per coordinate, so n_I >= 3 interpolates it exactly
    n = 16
    xn = chebyshev.nodes(n)
    px, pz = np.tile(xn, n), np.repeat(xn, n)
    Fc = (px[:, None] - px[None, :]) ** 2 + (pz[:, None] - pz[None, :]) ** 2
    rng = np.random.default_rng(3)
    obs = rng.uniform(0, 1, (20, 2))
    src = rng.uniform(0, 1, (30, 2))
    blk = chebyshev.interp_block(Fc, chebyshev.tensor_basis(xn, obs[:, 0], obs[:, 1]),
                                 chebyshev.tensor_basis(xn, src[:, 0], src[:, 1]))
    exact = ((obs[:, None, :] - src[None, :, :]) ** 2).sum(-1)
    assert np.max(np.abs(blk - exact)) < 1e-12
