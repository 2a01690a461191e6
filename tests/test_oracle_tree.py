"""Pins of oracle.tree (Sec. 4.2 cluster tree, Eq. proxyv2v) and of the
oracle HODBF (Sec. 4.2.1) against the dense sum on a tiny grid."""
import math

import numpy as np
import pytest

from oracle import butterfly, dense, kernel, tables, tree
from paper_2210_02698_gb300 import workloads as W


@pytest.mark.parametrize("N,leaf", [(16, 16), (32, 64), (24, 20)])
def test_cluster_tree_structure(N, leaf):
    perm, bounds = tree.cluster_tree(N, leaf)
    Nv = N * N
    assert sorted(perm) == list(range(Nv))
    Lv = len(bounds) - 1
    assert Lv == tree.num_levels(Nv, leaf)
    assert np.all(np.diff(bounds[-1]) <= leaf) and np.all(np.diff(bounds[-1]) >= 1)
    for l in range(Lv):
        assert len(bounds[l]) == (1 << l) + 1
        # children partition the parent
        assert np.all(bounds[l + 1][::2] == bounds[l])
    if N & (N - 1) == 0:
        # power-of-two grids: every node is an axis-aligned rectangle of cells
        for l in range(Lv + 1):
            for k in range(1 << l):
                P = perm[bounds[l][k]:bounds[l][k + 1]]
                a, b = P % N, P // N
                assert (a.max() - a.min() + 1) * (b.max() - b.min() + 1) == len(P)
    # leaves are in natural order
    for k in range(1 << Lv):
        P = perm[bounds[Lv][k]:bounds[Lv][k + 1]]
        assert np.all(np.diff(P) > 0)


def test_proxy_rows_brute_force():
    N = 32
    perm, bounds = tree.cluster_tree(N, 16)
    rng = np.random.default_rng(8)
    t0, t1 = bounds[2][1], bounds[2][2]
    for nseed, chi in ((3, 20.0), (10, 2.0), (40, 20.0)):
        seeds = rng.choice(np.arange(bounds[2][2], bounds[2][3]), size=nseed, replace=False)
        got = tree.proxy_rows(t0, t1, seeds, chi, 10.0, perm, N)
        size = t1 - t0
        m = min(size, math.ceil(chi * nseed))
        want = set()
        if m >= size:
            want = set(range(t0, t1))
        else:
            for k in range(m):
                want.add(t0 + (k * size) // m)
            for p in range(t0, t1):
                for s in seeds:
                    da = perm[p] % N - perm[s] % N
                    db = perm[p] // N - perm[s] // N
                    if da * da + db * db <= 100:
                        want.add(p)
        assert list(got) == sorted(want)


@pytest.mark.slow
def test_oracle_hodbf_matches_dense_at_tolerance():
    w = W.small_workload(W.GRADIENT, 16, 2, 2)
    op = kernel.Operator(w.N, tables.build_tables(W.GRADIENT, 8), w.omega, w.n_cells())
    s = W.complex_normal_sources(op.Nv, 2, 3)
    U = dense.apply(op, s)
    for eps, tol in ((1e-4, 1e-3), (1e-8, 1e-6)):
        H = butterfly.HODBF(op, 16, eps, 20.0, 10.0)
        err = np.linalg.norm(H.apply(s) - U) / np.linalg.norm(U)
        assert err < tol, (eps, err)
