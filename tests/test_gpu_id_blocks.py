"""The interpolative decompositions of a real build (Sec. 4.2.1, Eq. ID on
the sampled blocks of Eq. proxy) against the oracle, block by block.

hb_record_id_blocks makes hb_build keep copies of some of the sampled blocks
it hands to its ID: the proxy rows and column set, the samples as the ID
received them, the rank and the pivot order it chose.  For each kept block:
  * the samples equal the oracle's entries K(rows, cols) to 1e-11 of the
    block's largest entry (the entry evaluation of Eq. chebinterp + Eq. hb);
  * the oracle's CPQR (oracle/cpqr.py) on exactly those samples picks the
    same rank and the same skeleton list, in the same order, bit for bit.
"""
import numpy as np
import pytest

from tests._common import gpu_op, load_tables, oracle_op
from paper_2210_02698_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_02698_gb300 import build
    build.build()


def _check_blocks(w, per_level, min_levels):
    from oracle import cpqr
    from paper_2210_02698_gb300 import binding
    og = oracle_op(w)
    gp = gpu_op(w, precision=binding.HB_FP64)
    gp.record_id_blocks(per_level)
    gp.build()
    recs = gp.recorded_id_blocks()
    gp.close()
    assert len({r["level"] for r in recs}) >= min_levels
    bad = []
    for q, r in enumerate(recs):
        A = r["A"]
        want = og.block(r["rows"], r["cols"])
        scale = float(np.max(np.abs(want)))
        assert float(np.max(np.abs(A - want))) <= 1e-11 * scale, f"block {q} (level {r['level']}) entries"
        skel0, _, _ = cpqr.cpqr_id(A, w.eps)
        got = r["pivots"][:r["rank"]]
        if r["rank"] != len(skel0) or not np.array_equal(got, skel0):
            bad.append((q, r["level"], A.shape, r["rank"], len(skel0)))
    assert not bad, f"ID differs from the oracle on {len(bad)} of {len(recs)} blocks: {bad[:8]}"
    return len(recs)


def test_id_blocks_of_the_256_gradient_build():
    """The benchmark workload (256^2, w = 64 pi, eps = 1e-6): 8 blocks of
    every butterfly level."""
    w = W.WORKLOADS["grad256"]
    assert _check_blocks(w, 8, 9) >= 70


def test_every_id_block_of_a_32_grid():
    """All blocks of a whole build (32^2 gradient medium, leaf 16: 6 levels)."""
    w = W.small_workload(W.GRADIENT, 32, 4, 1, leaf=16)
    assert _check_blocks(w, 1 << 20, 5) > 100


def test_id_blocks_of_the_lens_medium():
    """The Gaussian lens (tables from the sweeping builder), 64^2."""
    w = W.small_workload(W.LENS, 64, 8, 1)
    assert _check_blocks(w, 24, 5) >= 60
