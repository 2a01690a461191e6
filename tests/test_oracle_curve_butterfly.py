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


@pytest.mark.parametrize("eps", [1e-6])
def test_compressed_operators_match_dense(eps):
    """K^{s2v}, K^{v2s} (single butterflies, L = min(L_v, L_s)) and K^{s2s}
    (HODBF) against the dense operators, on random vectors."""
    w = W.small_workload(W.GRADIENT, 32, 4, 3)
    op = oracle_op(w)
    cen, lw = W.circle_segments((0.5, 0.5), 0.25, 256)
    cur = inclusion.Curve(cen, lw)
    ci = cb.CompressedInclusion(op, cur, W.GRADIENT.n, leaf_v=16, leaf_s=4, eps=eps)
    assert ci.s2v.L == 6 and ci.Ls == 6
    cells = np.stack([op.px, op.pz], axis=1)
    rng = np.random.default_rng(8)
    p = rng.standard_normal(len(lw)) + 1j * rng.standard_normal(len(lw))
    x = rng.standard_normal(w.grid.Nv) + 1j * rng.standard_normal(w.grid.Nv)
    Sp, Vp = ci.S.perm, ci.V.perm

    def run(bf, vec, perm_in, perm_out, n_out):
        y = np.zeros(n_out, dtype=complex)
        bf.apply(vec[perm_in], y)
        out = np.empty_like(y)
        out[perm_out] = y
        return out

    errs = {
        "s2v": (run(ci.s2v, p, Sp, Vp, w.grid.Nv), inclusion.K_s2v(op.tab, op.omega, cur, cells) @ p),
        "v2s": (run(ci.v2s, x, Vp, Sp, len(lw)), inclusion.K_v2s(op.tab, op.omega, cur, cells) @ x),
    }
    y = ci.s2s_apply(p[Sp])
    s2s = np.empty_like(y)
    s2s[Sp] = y
    errs["s2s"] = (s2s, inclusion.K_s2s(op.tab, op.omega, cur, W.GRADIENT.n) @ p)
    for name, (got, want) in errs.items():
        assert np.linalg.norm(got - want) / np.linalg.norm(want) < 30 * eps, name
    # compressed below the dense block; ranks peak inside the butterfly
    assert ci.s2v.entries() < w.grid.Nv * len(lw)
    ranks = ci.s2v.max_rank_by_level()
    assert 0 < np.argmax(ranks) < ci.s2v.L
    print("eps", eps, {k: float(np.linalg.norm(a - b) / np.linalg.norm(b)) for k, (a, b) in errs.items()},
          "s2v entries", ci.s2v.entries(), "of", w.grid.Nv * len(lw), "ranks", ranks)


def test_compressed_total_field_matches_dense():
    """U = K^{v2v} I + K^{s2v} (K^{s2s})^{-1} K^{v2s} I with the compressed
    operators and a GMRES solve against the dense LU path (Eq. m_v2v_inclu)."""
    from oracle import dense
    w = W.small_workload(W.GRADIENT, 32, 4, 2)
    op = oracle_op(w)
    cen, lw = W.circle_segments((0.5, 0.5), 0.25, 128)
    cur = inclusion.Curve(cen, lw)
    s = W.complex_normal_sources(w.grid.Nv, 2, 23)
    v2v = dense.apply(op, s)
    want, _ = inclusion.total_field(op, cur, W.GRADIENT.n, s, v2v=v2v)
    ci = cb.CompressedInclusion(op, cur, W.GRADIENT.n, leaf_v=16, leaf_s=4, eps=1e-8)
    got = ci.total_field(s, v2v)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-6
    assert np.linalg.norm(v2v - want) / np.linalg.norm(want) > 1e-2      # the inclusion matters
