"""hb_apply / hb_apply_adjoint captured in a CUDA graph (after one eager call
has set up the scratch and the launch plans) replay bit-identically to eager
calls, for new inputs written into the captured buffers, in both
precisions."""
import pytest

from paper_2210_02698_gb300 import workloads as W
from tests._common import gpu_op, to_dev


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_apply_in_cuda_graph_replays_eager_results(precision):
    import torch
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.GRADIENT, 64, 8, 3)
    R = w.nrhs
    op = gpu_op(w, precision=binding.HB_FP64 if precision == "fp64" else binding.HB_MIXED_BF16X3)
    op.build()
    st = torch.cuda.Stream()
    s_dev = to_dev(W.complex_normal_sources(w.grid.Nv, R, 41))
    u_dev = torch.empty_like(s_dev)
    a_dev = torch.empty_like(s_dev)
    with torch.cuda.stream(st):
        op.apply(s_dev, u_dev, R, st)            # eager: scratch and plans are set up here
        op.apply_adjoint(s_dev, a_dev, R, st)
    st.synchronize()

    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        op.apply(s_dev, u_dev, R, st)
        op.apply_adjoint(s_dev, a_dev, R, st)
    for seed in (42, 43):
        s_new = to_dev(W.complex_normal_sources(w.grid.Nv, R, seed))
        s_dev.copy_(s_new)
        g.replay()
        torch.cuda.synchronize()
        u_eager, a_eager = torch.empty_like(s_dev), torch.empty_like(s_dev)
        op.apply(s_new, u_eager, R)
        op.apply_adjoint(s_new, a_eager, R)
        torch.cuda.synchronize()
        assert torch.equal(u_dev, u_eager)
        assert torch.equal(a_dev, a_eager)
    op.close()
