"""Race detection without a sanitizer: every apply is a fixed schedule of
per-warp streams with no atomics, so repeated applies give bitwise-equal
outputs (FP64 and mixed butterfly, both directions, and the dense sum with
its source shares added in a fixed order)."""
import numpy as np
import pytest

from paper_2210_02698_gb300 import workloads as W
from tests._common import gpu_op, to_dev

pytestmark = pytest.mark.gpu


def test_ten_replays_are_bitwise_equal():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.GRADIENT, 64, 8, 3)
    s_dev = to_dev(W.workload_sources(w))
    op = gpu_op(w, precision=binding.HB_FP64)
    op.build()
    runs = [(binding.HB_FP64, op.apply), (binding.HB_FP64, op.apply_adjoint),
            (binding.HB_MIXED_BF16X3, op.apply), (binding.HB_MIXED_BF16X3, op.apply_adjoint),
            (binding.HB_FP64, op.apply_dense)]
    for prec, fn in runs:
        op.set_precision(prec)
        outs = []
        for _ in range(10):
            u = torch.full_like(s_dev, float("nan"))
            fn(s_dev, u, s_dev.shape[0])
            torch.cuda.synchronize()
            outs.append(u.cpu().numpy())
        for o in outs[1:]:
            assert np.array_equal(o, outs[0])
        assert np.all(np.isfinite(outs[0]))
    op.close()
