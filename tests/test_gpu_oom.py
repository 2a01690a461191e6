"""Out-of-memory handling without exhausting the GPU (host-side fault
injection): the library's device allocation cap (hb_device_alloc_cap) makes
an allocation fail as a real out-of-memory would.  A build that fails
mid-way returns HB_ERR_OOM, frees everything it had allocated (the live
device bytes return to their value before the build) and leaves the handle
unbuilt, so that a second build succeeds; an apply whose scratch cannot be
allocated returns HB_ERR_OOM and works when repeated with room."""
import pytest

from paper_2210_02698_gb300 import workloads as W
from tests._common import from_dev, gpu_op, oracle_op, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def test_failed_build_and_apply_leave_nothing_behind():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from oracle import dense
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.GRADIENT, 48, 6, 2)
    s = W.workload_sources(w)
    want = dense.apply(oracle_op(w), s)
    import gc
    gc.collect()   # operators of earlier tests are gone before the live bytes are read
    op = gpu_op(w, precision=binding.HB_MIXED_BF16X3, workspace_mb=16)
    try:
        live0 = binding.device_alloc_cap(-1)
        # room for the 16 MB build workspace and 64 KB more: a later
        # allocation of the build (its factor segments) fails
        binding.device_alloc_cap(live0 + (16 << 20) + (64 << 10))
        with pytest.raises(binding.HBError) as e:
            op.build()
        assert e.value.status == binding.HB_ERR_OOM
        assert binding.device_alloc_cap(-1) == live0
        binding.device_alloc_cap(0)
        op.build()
        live1 = binding.device_alloc_cap(-1)
        assert live1 > live0

        s_dev = to_dev(s)
        u = torch.empty_like(s_dev)
        binding.device_alloc_cap(live1 + 1)
        with pytest.raises(binding.HBError) as e:
            op.apply(s_dev, u, s.shape[1])
        assert e.value.status == binding.HB_ERR_OOM
        binding.device_alloc_cap(0)
        op.apply(s_dev, u, s.shape[1])
        torch.cuda.synchronize()
        assert rel_l2(from_dev(u), want) < 1e-4
    finally:
        binding.device_alloc_cap(0)
        op.close()
