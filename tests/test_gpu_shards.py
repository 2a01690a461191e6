"""Row shards of the apply (Sec. 4.2: each off-diagonal butterfly of the
HODBF writes only its own rows), checked on one GPU by running every rank's
share in turn: hb_apply_shard for each of P = 2, 4, 8 ranks writes exactly
its own cells, and together they give hb_apply's result bit for bit (the
same tasks in the same order); the ranks' hb_apply_shard_adjoint shares add
up to hb_apply_adjoint's result (FP64: to 1e-13; mixed precision: each
share is rounded to split-BF16 on its own, so the sum is held to the mixed
path's bar, rel-L2 1e-4 against the FP64 adjoint).  One and two m-tiles of
right-hand sides.  The collectives around them run on CPU ranks
in tests/test_dist_gloo.py."""
import numpy as np
import pytest

from paper_2210_02698_gb300 import workloads as W
from tests._common import gpu_op, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_02698_gb300 import build
    build.build()


@pytest.mark.parametrize("N,leaf,nrhs", [(64, 64, 3), (48, 32, 20), (40, 64, 2)])
def test_shards_reassemble_the_apply(N, leaf, nrhs):
    import torch
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.GRADIENT, N, N / 8, nrhs, leaf=leaf)
    s_dev = to_dev(W.complex_normal_sources(w.grid.Nv, nrhs, 55))
    u_dev = to_dev(W.complex_normal_sources(w.grid.Nv, nrhs, 56))
    op = gpu_op(w, precision=binding.HB_FP64)
    op.build()
    perm = torch.from_numpy(op.tree_perm()).cuda()
    ref64 = torch.empty_like(s_dev)
    op.apply_adjoint(u_dev, ref64, nrhs)
    for prec in (binding.HB_FP64, binding.HB_MIXED_BF16X3):
        op.set_precision(prec)
        full = torch.empty_like(s_dev)
        op.apply(s_dev, full, nrhs)
        fullA = torch.empty_like(s_dev)
        op.apply_adjoint(u_dev, fullA, nrhs)
        torch.cuda.synchronize()
        for P in (2, 4, 8):
            got = torch.full_like(s_dev, float("nan"))
            accA = torch.zeros_like(s_dev)
            covered = 0
            for r in range(P):
                lo, hi = op.shard_rows(P, r)
                mine = perm[lo:hi]
                covered += hi - lo
                op.apply_shard(s_dev, got, nrhs, P, r)
                # the adjoint share sees only this rank's cells of u
                u_mine = torch.zeros_like(u_dev)
                u_mine[:, mine] = u_dev[:, mine]
                share = torch.full_like(s_dev, float("nan"))
                op.apply_shard_adjoint(u_mine, share, nrhs, P, r)
                torch.cuda.synchronize()
                assert torch.isfinite(torch.view_as_real(share)).all()
                accA += share
            assert covered == w.grid.Nv
            # every cell written by exactly its owner, equal to the whole apply
            assert torch.equal(got, full), (prec, P)
            if prec == binding.HB_FP64:
                rel = float((accA - fullA).abs().max() / fullA.abs().max())
                assert rel < 1e-13, (P, rel)
            else:
                rel = float(torch.linalg.norm(accA - ref64) / torch.linalg.norm(ref64))
                assert rel < 1e-4, (P, rel)
    op.close()


def test_shard_arguments():
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.GRADIENT, 32, 4, 1, leaf=64)
    op = gpu_op(w)
    op.build()
    assert op.shard_rows(1, 0) == (0, w.grid.Nv)
    for P, r in ((3, 0), (2, 2), (64, 0)):   # not a power of two; rank out of range; more ranks than leaves
        with pytest.raises(binding.HBError) as e:
            op.shard_rows(P, r)
        assert e.value.status == binding.HB_ERR_ARG
    op.close()
