"""The Gaussian-lens medium n = 1 + 0.1 exp(-|r - (0.5,0.5)|^2 / 0.3^2)
(Sec. 5.1.1 smooth media), whose tables come from the oracle's sweeping
builder: the GPU butterfly apply and its adjoint against the dense oracle
on the same tables, with the uneven source mix of the 1024^2 workload
(point sources, line segments, complex Gaussian bumps, Gaussian
wavepackets), on a small grid in full and at 1024^2 on sampled rows in the
configuration the benchmark times (Sec. 4.2 HODBF, Sec. 4.2.1 butterflies).
"""
import numpy as np
import pytest

from paper_2210_02698_gb300 import workloads as W
from tests._common import from_dev, gpu_op, oracle_dense_rows, oracle_op, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _apply(op, s, adjoint=False):
    import torch
    out = torch.empty((s.shape[1], s.shape[0]), dtype=torch.complex128, device="cuda")
    (op.apply_adjoint if adjoint else op.apply)(to_dev(s), out, s.shape[1])
    torch.cuda.synchronize()
    return from_dev(out)


def _col_rel(got, want):
    return float(np.max(np.linalg.norm(got - want, axis=0) / np.linalg.norm(want, axis=0)))


def test_lens_small_grid_vs_dense_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from oracle import dense
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.LENS, 64, 8, 8)
    s = W.mixed_sources(w.grid, w.omega, 8, 31)
    og, gp = oracle_op(w), gpu_op(w, precision=binding.HB_FP64)
    gp.build()
    want, wantA = dense.apply(og, s), dense.adjoint(og, s)
    assert rel_l2(_apply(gp, s), want) < 1e-5 and _col_rel(_apply(gp, s), want) < 1e-5
    assert rel_l2(_apply(gp, s, True), wantA) < 1e-5
    gp.set_precision(binding.HB_MIXED_BF16X3)
    got = _apply(gp, s)
    assert rel_l2(got, want) < 1e-4 and _col_rel(got, want) < 1e-4
    assert _col_rel(_apply(gp, s, True), wantA) < 1e-4
    gp.close()


@pytest.mark.slow
def test_lens1024_fullsize_sampled_rows():
    """1024^2 cells, w = 2 pi 128, 64 mixed right-hand sides (two passes of
    32 in the mixed apply); 24 seeded rows against the dense oracle."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from oracle import dense
    from paper_2210_02698_gb300 import binding
    w = W.WORKLOADS["lens1024"]
    s = W.workload_sources(w)
    rows = W.sample_rows(w.grid.Nv, 24, 4242)
    want = oracle_dense_rows(w, s, rows)
    gp = gpu_op(w, precision=binding.HB_MIXED_BF16X3)
    gp.build()
    s_dev = to_dev(s)
    u = torch.empty_like(s_dev)
    rows_t = torch.from_numpy(rows).cuda()
    gp.apply(s_dev, u, s.shape[1])
    got = u[:, rows_t].cpu().numpy().T
    print("lens1024 mixed rel-L2", rel_l2(got, want), "worst column", _col_rel(got, want))
    assert rel_l2(got, want) < 1e-4
    gp.set_precision(binding.HB_FP64)
    gp.apply(s_dev, u, s.shape[1])
    got64 = u[:, rows_t].cpu().numpy().T
    assert rel_l2(got64, want) < 1e-5
    gp.close()
