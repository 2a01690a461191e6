"""Frequency reuse (Sec. 4.1: tau^2, v0 and v1 do not depend on omega, so
one table set serves every frequency): hb_set_omega moves a built handle to
another omega.  Rebuilt there, it gives the same factors and the same
applies - FP64 and mixed, forward and adjoint, bit for bit - as a handle
created at that omega from the same tables, matches the dense oracle at the
new omega, and re-assembles a curve set on it; applies on the unbuilt
handle and a bad omega are refused."""
import numpy as np
import pytest

from paper_2210_02698_gb300 import workloads as W
from tests._common import from_dev, gpu_op, oracle_op, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_02698_gb300 import build
    build.build()


def _applies(op, s_dev, nrhs):
    import torch
    from paper_2210_02698_gb300 import binding
    out = []
    for prec in (binding.HB_FP64, binding.HB_MIXED_BF16X3):
        op.set_precision(prec)
        u, a = torch.empty_like(s_dev), torch.empty_like(s_dev)
        op.apply(s_dev, u, nrhs)
        op.apply_adjoint(s_dev, a, nrhs)
        torch.cuda.synchronize()
        out += [from_dev(u), from_dev(a)]
    return out


@pytest.mark.parametrize("N,leaf,nrhs", [(48, 32, 3), (40, 64, 17)])
def test_set_omega_equals_a_fresh_handle(N, leaf, nrhs):
    from oracle import dense
    from paper_2210_02698_gb300 import binding
    w1 = W.small_workload(W.GRADIENT, N, N / 8, nrhs, leaf=leaf)
    w2 = W.small_workload(W.GRADIENT, N, N / 12, nrhs, leaf=leaf)   # another frequency, same tables
    s = W.complex_normal_sources(w1.grid.Nv, nrhs, 61)
    s_dev = to_dev(s)
    op = gpu_op(w1)
    op.build()
    before = _applies(op, s_dev, nrhs)
    op.set_omega(w2.omega)
    with pytest.raises(binding.HBError) as e:   # unbuilt until hb_build
        op.apply(s_dev, s_dev.clone(), nrhs)
    assert e.value.status == binding.HB_ERR_STATE
    op.build()
    moved = _applies(op, s_dev, nrhs)
    fresh = gpu_op(w2)
    fresh.build()
    want = _applies(fresh, s_dev, nrhs)
    for got, ref in zip(moved, want):
        assert np.array_equal(got, ref)
    assert op.info()["max_rank"] == fresh.info()["max_rank"]
    assert op.info()["factor_entries"] == fresh.info()["factor_entries"]
    # the new frequency changed the operator, and the oracle agrees at it
    assert rel_l2(moved[0], before[0]) > 1e-2
    og = oracle_op(w2)
    assert rel_l2(moved[0], dense.apply(og, s)) < 1e-5
    assert rel_l2(moved[1], dense.adjoint(og, s)) < 1e-5
    assert rel_l2(moved[2], dense.apply(og, s)) < 1e-4
    # back to the first frequency: the first results again
    op.set_omega(w1.omega)
    op.build()
    for got, ref in zip(_applies(op, s_dev, nrhs), before):
        assert np.array_equal(got, ref)
    op.close()
    fresh.close()


def test_set_omega_reassembles_the_curve():
    import torch
    from paper_2210_02698_gb300 import binding
    w1 = W.small_workload(W.GRADIENT, 32, 4, 2)
    w2 = W.small_workload(W.GRADIENT, 32, 3, 2)
    cen, lw = W.circle_segments((0.5, 0.5), 0.2, 96)
    nseg = W.GRADIENT.n(cen[:, 0], cen[:, 1])
    s_dev = to_dev(W.complex_normal_sources(w1.grid.Nv, 2, 62))
    op = gpu_op(w1, precision=binding.HB_FP64)
    op.set_curve(cen, lw, nseg)
    op.set_omega(w2.omega)
    fresh = gpu_op(w2, precision=binding.HB_FP64)
    fresh.set_curve(cen, lw, nseg)
    got, want = torch.empty_like(s_dev), torch.empty_like(s_dev)
    op.apply_inclusion(s_dev, got, 2, v2v_dense=True)
    fresh.apply_inclusion(s_dev, want, 2, v2v_dense=True)
    torch.cuda.synchronize()
    assert torch.equal(got, want)
    with pytest.raises(binding.HBError) as e:
        op.set_omega(-1.0)
    assert e.value.status == binding.HB_ERR_ARG
    op.close()
    fresh.close()
