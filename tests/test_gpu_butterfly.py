"""GPU HODBF / butterfly construction and apply (Sec. 4.2, Eq. butterfly_mat)
against the oracle.  Bars: tree order and proxy rows bit-exact; FP64
butterfly at eps = 1e-6 within rel-L2 1e-5 of the dense oracle; mixed
precision within 1e-4; adjoint identity to rounding."""
import numpy as np
import pytest

from tests._common import from_dev, gpu_op, oracle_op, rel_l2, to_dev
from paper_2210_02698_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_02698_gb300 import build
    build.build()


def _apply(op, s, adjoint=False):
    import torch
    nrhs = s.shape[1]
    out = torch.empty((nrhs, s.shape[0]), dtype=torch.complex128, device="cuda")
    (op.apply_adjoint if adjoint else op.apply)(to_dev(s), out, nrhs)
    torch.cuda.synchronize()
    return from_dev(out)


@pytest.mark.parametrize("N,leaf", [(32, 64), (24, 20), (64, 64)])
def test_tree_and_proxy_rows_match_oracle(N, leaf):
    from oracle import tree
    w = W.small_workload(W.GRADIENT, N, N / 8, 1, leaf=leaf)
    gp = gpu_op(w)
    perm, bounds = tree.cluster_tree(N, leaf)
    assert np.array_equal(gp.tree_perm(), perm)
    rng = np.random.default_rng(N)
    for lvl in range(1, len(bounds)):
        k = rng.integers(0, (1 << lvl) - 1)
        t0, t1 = int(bounds[lvl][k]), int(bounds[lvl][k + 1])
        s0, s1 = int(bounds[lvl][k + 1]), int(bounds[lvl][k + 2])
        seeds = rng.choice(np.arange(s0, s1), size=min(s1 - s0, 7), replace=False)
        want = tree.proxy_rows(t0, t1, seeds, w.chi, 10.0, perm, N)
        assert np.array_equal(gp.proxy_rows(t0, t1, seeds), want)


# 24 RHS: one pass of two m-tiles; 40 RHS: passes of 32 (two m-tiles) + 8 (one); 17: FP64 passes 16 + 1;
# 8 x 8: a single leaf (no butterfly at all); 9 x 9: two leaves of 41 and 40 cells
@pytest.mark.parametrize("N,leaf,nrhs", [(32, 64, 3), (48, 32, 2), (64, 64, 4), (48, 64, 24), (32, 32, 40),
                                         (40, 64, 17), (8, 64, 2), (9, 64, 3)])
def test_butterfly_fp64_and_mixed_vs_dense_oracle(N, leaf, nrhs):
    from oracle import dense
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.GRADIENT, N, N / 8, nrhs, leaf=leaf)
    og, gp = oracle_op(w), gpu_op(w, precision=binding.HB_FP64)
    gp.build()
    s = W.complex_normal_sources(w.grid.Nv, nrhs, 41)
    want = dense.apply(og, s)
    got = _apply(gp, s)
    assert rel_l2(got, want) < 1e-5
    gp.set_precision(binding.HB_MIXED_BF16X3)
    assert rel_l2(_apply(gp, s), want) < 1e-4
    # adjoint against the dense oracle adjoint, both precisions
    gp.set_precision(binding.HB_FP64)
    wantA = dense.adjoint(og, s)
    assert rel_l2(_apply(gp, s, adjoint=True), wantA) < 1e-5
    gp.set_precision(binding.HB_MIXED_BF16X3)
    assert rel_l2(_apply(gp, s, adjoint=True), wantA) < 1e-4


def test_fp64_adjoint_is_exact_adjoint_of_compressed_operator():
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.GRADIENT, 64, 8, 2)
    gp = gpu_op(w, precision=binding.HB_FP64)
    gp.build()
    x = W.complex_normal_sources(w.grid.Nv, 2, 1)
    y = W.complex_normal_sources(w.grid.Nv, 2, 2)
    Ax = _apply(gp, x)
    AHy = _apply(gp, y, adjoint=True)
    lhs = np.vdot(y, Ax)
    rhs = np.vdot(AHy, x)
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(Ax) * np.linalg.norm(y)


def test_tight_tolerance_reproduces_dense():
    from oracle import dense
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.GRADIENT, 32, 4, 1, eps=1e-13)
    og, gp = oracle_op(w), gpu_op(w, precision=binding.HB_FP64)
    gp.build()
    s = W.complex_normal_sources(w.grid.Nv, 1, 9)
    assert rel_l2(_apply(gp, s), dense.apply(og, s)) < 1e-11


def test_grad256_fullsize_sampled_rows():
    """The 256^2, 16-RHS workload in the configuration the benchmark times:
    128 seeded rows of the forward apply and 64 seeded columns of the
    adjoint against the dense oracle, FP64 (1e-5) and mixed (1e-4), each
    right-hand side on its own as well as all together."""
    from oracle import dense
    from paper_2210_02698_gb300 import binding
    w = W.WORKLOADS["grad256"]
    og, gp = oracle_op(w), gpu_op(w, precision=binding.HB_FP64, autotune=1)
    gp.build()
    s = W.workload_sources(w)
    rows = W.sample_rows(w.grid.Nv, 128, 99)
    cols = W.sample_rows(w.grid.Nv, 64, 98)
    want = dense.apply(og, s, rows=rows, chunk=8192)
    wantA = dense.adjoint(og, s, cols=cols, chunk=8192)

    def worst_col(a, b):
        return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))
    for prec, tol in ((binding.HB_FP64, 1e-5), (binding.HB_MIXED_BF16X3, 1e-4)):
        gp.set_precision(prec)
        got, gotA = _apply(gp, s)[rows], _apply(gp, s, True)[cols]
        assert rel_l2(got, want) < tol and worst_col(got, want) < tol
        assert rel_l2(gotA, wantA) < tol and worst_col(gotA, wantA) < tol
    gp.close()


def test_autograd_gradient_matches_finite_differences():
    """Source-inversion loss ||P u(s) - d||^2 with the hand-written adjoint as
    backward; the loss is quadratic in s so central differences are exact up
    to rounding (Sec. 3.1 operator, adjoint apply)."""
    import torch
    from paper_2210_02698_gb300 import binding
    from paper_2210_02698_gb300.autograd import hb_apply
    w = W.small_workload(W.GRADIENT, 64, 8, 1)
    for prec, tol in ((binding.HB_FP64, 1e-8), (binding.HB_MIXED_BF16X3, 1e-4)):
        gp = gpu_op(w, precision=prec)
        gp.build()
        rng = np.random.default_rng(12)
        P = torch.from_numpy(np.sort(rng.choice(w.grid.Nv, 64, replace=False))).cuda()
        s_ref = torch.from_numpy(W.complex_normal_sources(w.grid.Nv, 1, 3).T.copy()).cuda()
        with torch.no_grad():
            d = hb_apply(s_ref, gp)[:, P]
        s0 = torch.from_numpy(W.complex_normal_sources(w.grid.Nv, 1, 4).T.copy()).cuda()
        s = s0.clone().requires_grad_(True)

        def loss(x):
            r = hb_apply(x, gp)[:, P] - d
            return (r.abs() ** 2).sum()

        L = loss(s)
        L.backward()
        g = s.grad.detach()
        for k in range(8):
            dl = torch.from_numpy(W.complex_normal_sources(w.grid.Nv, 1, 100 + k).T.copy()).cuda()
            # the loss is quadratic in s: central differences are exact for
            # any step, so a step of the size of s0 keeps the difference of
            # the two losses far above their rounding
            t = float(s0.norm() / dl.norm())
            with torch.no_grad():
                fd = (loss(s0 + t * dl) - loss(s0 - t * dl)) / (2 * t)
            pred = torch.real(torch.vdot(g.reshape(-1), dl.reshape(-1)))
            assert abs(float(fd - pred)) <= tol * abs(float(pred)) + tol * float(g.norm() * dl.norm())


def test_maximum_rhs_on_a_small_grid():
    """1024 right-hand sides (the documented maximum; 32 mixed passes, 64 FP64
    passes) on a 16 x 16 grid with two tree levels; 1025 is refused."""
    import torch
    from oracle import dense
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.GRADIENT, 16, 2, 1024)
    og, gp = oracle_op(w), gpu_op(w, precision=binding.HB_FP64)
    gp.build()
    s = W.complex_normal_sources(w.grid.Nv, 1024, 77)
    want = dense.apply(og, s)
    assert rel_l2(_apply(gp, s), want) < 1e-5
    gp.set_precision(binding.HB_MIXED_BF16X3)
    got = _apply(gp, s)
    assert rel_l2(got, want) < 1e-4
    assert np.max(np.linalg.norm(got - want, axis=0) / np.linalg.norm(want, axis=0)) < 1e-4
    wantA = dense.adjoint(og, s)
    assert rel_l2(_apply(gp, s, adjoint=True), wantA) < 1e-4
    s1 = torch.zeros((1025, w.grid.Nv), dtype=torch.complex128, device="cuda")
    with pytest.raises(binding.HBError) as e:
        gp.apply(s1, torch.empty_like(s1), 1025)
    assert e.value.status == binding.HB_ERR_ARG
    gp.close()
