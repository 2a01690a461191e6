"""The K^{s2v} butterfly prototype (oracle/curve_butterfly.py, Sec. 4.2
K^{s2v} item) against the dense K^{s2v} of oracle/inclusion.py."""
import numpy as np
import pytest

from oracle import curve_butterfly as cb, inclusion
from paper_2210_02698_gb300 import workloads as W
from tests._common import oracle_op


def test_segment_tree_partitions_the_segments():
    cen, _ = W.circle_segments((0.5, 0.5), 0.3, 100)
    perm, bounds = cb.segment_tree(cen, 8)
    assert sorted(perm.tolist()) == list(range(100))
    for l in range(1, len(bounds)):
        b = bounds[l]
        assert b[0] == 0 and b[-1] == 100 and np.all(np.diff(b) >= 0)
        assert set(b[::2].tolist()) <= set(b.tolist()) and np.array_equal(b[::2], bounds[l - 1])
    leaves = bounds[-1]
    assert np.max(np.diff(leaves)) <= 8
    # siblings split the longer side: on a circle, a leaf is an arc of neighbouring segments
    for i in range(len(leaves) - 1):
        seg = np.sort(perm[leaves[i]:leaves[i + 1]])
        gaps = np.diff(np.concatenate([seg, [seg[0] + 100]]))
        assert np.count_nonzero(gaps > 1) <= 1


@pytest.mark.parametrize("eps", [1e-6, 1e-10])
def test_s2v_butterfly_matches_dense(eps):
    w = W.small_workload(W.GRADIENT, 32, 4, 3)
    op = oracle_op(w)
    cen, lw = W.circle_segments((0.5, 0.5), 0.25, 256)
    cur = inclusion.Curve(cen, lw)
    bf = cb.S2VButterfly(op, cur, leaf_v=16, leaf_s=4, eps=eps)
    assert bf.L == 6
    p = W.complex_normal_sources(len(lw), 3, 17)
    cells = np.stack([op.px, op.pz], axis=1)
    want = inclusion.K_s2v(op.tab, op.omega, cur, cells) @ p
    err = np.linalg.norm(bf.apply(p) - want) / np.linalg.norm(want)
    assert err < 30 * eps
    # compressed below the dense block, ranks bounded
    assert bf.factor_entries() < w.grid.Nv * len(lw)
    print("eps", eps, "rel err", err, "entries", bf.factor_entries(), "dense", w.grid.Nv * len(lw),
          "max rank by level", bf.max_rank_by_level())
