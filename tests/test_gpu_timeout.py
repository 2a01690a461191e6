"""Failure detection of the mixed apply without a GPU fault.  With the wait
self-test on, the first warp of every step launch (of the dataflow launch:
after its stream) also waits - through the same bounded wait as the data
waits - on an mbarrier that nothing completes;
with a short budget the wait runs out, the mapped error word is set and the
next apply reports HB_ERR_TIMEOUT.  The apply itself completes, and the CUDA
context stays usable: the same handle, self-test off, matches the oracle."""
import pytest

from paper_2210_02698_gb300 import workloads as W
from tests._common import gpu_op, oracle_op, rel_l2, to_dev, from_dev


@pytest.mark.gpu
@pytest.mark.parametrize("shape", [0, 2, 4, 5, 6])   # per depth; dataflow; cones; fused level pairs; grid barriers
def test_wait_that_runs_out_is_reported_and_context_survives(shape):
    import torch
    from paper_2210_02698_gb300 import binding
    from oracle import dense
    w = W.small_workload(W.GRADIENT, 48, 8, 2)
    s = W.workload_sources(w)
    want = dense.apply(oracle_op(w), s)
    s_dev = to_dev(s)
    u_dev = torch.empty_like(s_dev)

    # about 0.5 ms of SM cycles per wait: the data waits finish long before
    op = gpu_op(w, precision=binding.HB_MIXED_BF16X3, barrier_cycles=1 << 20, autotune=shape)
    op.build()
    op.set_wait_selftest(True)
    op.apply(s_dev, u_dev, s.shape[1])
    torch.cuda.synchronize()
    assert rel_l2(from_dev(u_dev), want) < 1e-4      # the data path is untouched
    with pytest.raises(binding.HBError) as e:
        op.apply(s_dev, u_dev, s.shape[1])
    assert e.value.status == binding.HB_ERR_TIMEOUT
    torch.cuda.synchronize()                          # no sticky CUDA error

    op.set_wait_selftest(False)
    op.apply(s_dev, u_dev, s.shape[1])                # the error word was cleared when reported
    op.apply_adjoint(s_dev, u_dev, s.shape[1])
    op.apply(s_dev, u_dev, s.shape[1])
    torch.cuda.synchronize()
    assert rel_l2(from_dev(u_dev), want) < 1e-4
    op.close()
