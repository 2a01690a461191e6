"""GPU parity of entry evaluation and the matrix-free dense apply / adjoint
(Eq. m_v2v, Eq. chebinterpblock, Eq. babich, Appendix A) against the oracle.
Bar: FP64 relative L2 <= 1e-12."""
import numpy as np
import pytest

from tests._common import from_dev, gpu_op, oracle_op, rel_l2, to_dev
from paper_2210_02698_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_02698_gb300 import build
    build.build()


def _entries(op, rows, cols):
    import torch
    out = torch.empty((len(cols), len(rows)), dtype=torch.complex128, device="cuda")
    op.entries(rows, cols, out)
    return out.cpu().numpy().T


@pytest.mark.parametrize("name", ["homog64", "grad256"])
def test_entries_match_oracle(name):
    w = W.WORKLOADS[name]
    og, gp = oracle_op(w), gpu_op(w)
    rng = np.random.default_rng(5)
    rows = rng.choice(w.grid.Nv, 37, replace=False)
    cols = np.concatenate([rows[:5], rng.choice(w.grid.Nv, 90, replace=False)])   # includes diagonals
    got = _entries(gp, rows, cols)
    want = og.block(rows, cols)
    err = np.abs(got - want)
    assert np.max(err / (np.abs(want) + 1e-3 * np.max(np.abs(want)))) < 1e-11
    assert rel_l2(got, want) < TOL


def test_self_terms_match_lemma():
    from oracle import kernel
    w = W.WORKLOADS["grad256"]
    gp = gpu_op(w)
    idx = np.array([0, 1000, 40000, 65535])
    got = np.diag(_entries(gp, idx, idx))
    n = w.n_cells()[idx]
    want = np.array([kernel.self_term(v, w.omega, w.grid.h) for v in n])
    assert np.max(np.abs(got - want) / np.abs(want)) < 1e-11


def test_dense_apply_full_homogeneous_64():
    from oracle import dense
    w = W.WORKLOADS["homog64"]
    og, gp = oracle_op(w), gpu_op(w)
    s = W.workload_sources(w)
    want = dense.apply(og, s)
    import torch
    u = torch.empty((1, w.grid.Nv), dtype=torch.complex128, device="cuda")
    gp.apply_dense(to_dev(s), u, 1)
    torch.cuda.synchronize()
    assert rel_l2(from_dev(u), want) < TOL


@pytest.mark.parametrize("N,nrhs", [(40, 3), (72, 5)])
def test_dense_apply_and_adjoint_ragged(N, nrhs):
    """Grids that are not multiples of the 64-cell tile, several RHS chunks."""
    import torch
    from oracle import dense
    w = W.small_workload(W.GRADIENT, N, N / 8, nrhs)
    og, gp = oracle_op(w), gpu_op(w)
    s = W.complex_normal_sources(w.grid.Nv, nrhs, 31)
    u = torch.empty((nrhs, w.grid.Nv), dtype=torch.complex128, device="cuda")
    gp.apply_dense(to_dev(s), u, nrhs)
    assert rel_l2(from_dev(u), dense.apply(og, s)) < TOL
    a = torch.empty_like(u)
    gp.apply_dense_adjoint(to_dev(s), a, nrhs)
    assert rel_l2(from_dev(a), dense.adjoint(og, s)) < TOL


def test_dense_apply_grad256_sampled_rows():
    """Full-size 256^2 workload with 16 RHS: sampled rows against the oracle."""
    import torch
    from oracle import dense
    w = W.WORKLOADS["grad256"]
    og, gp = oracle_op(w), gpu_op(w)
    s = W.workload_sources(w)
    u = torch.empty((w.nrhs, w.grid.Nv), dtype=torch.complex128, device="cuda")
    gp.apply_dense(to_dev(s), u, w.nrhs)
    rows = W.sample_rows(w.grid.Nv, 24, 77)
    want = dense.apply(og, s, rows=rows, chunk=8192)
    assert rel_l2(from_dev(u)[rows], want) < TOL
