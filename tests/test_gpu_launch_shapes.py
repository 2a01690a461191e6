"""The launch shapes of the mixed apply give the same numbers.

A chain (one n-tile group of one task) accumulates its items in the same
order in every shape; only where and when chains run changes.  So the gather
plus one launch per dependency depth (the default), the persistent dataflow
launch, the cone launch of the first butterfly levels, the transfer depths
fused in pairs, every depth in one cooperative launch with grid barriers,
and whatever shape
the autotuner picks all give bitwise equal outputs (the tensor-core leaf
shapes equal one another), in both directions and at one and two m-tiles (16 and 32
right-hand sides per pass)."""
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


@pytest.mark.parametrize("N,leaf,nrhs", [(64, 64, 3), (48, 32, 24), (9, 64, 2)])
def test_shapes_are_bitwise_equal(N, leaf, nrhs):
    import torch
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.GRADIENT, N, N / 8, nrhs, leaf=leaf)
    s_dev = to_dev(W.complex_normal_sources(w.grid.Nv, nrhs, 77))
    outs, shapes = {}, {}
    for tune in (0, 2, 3, 4, 5, 6, 1):
        op = gpu_op(w, precision=binding.HB_MIXED_BF16X3, autotune=tune)
        op.build()
        u = torch.full_like(s_dev, float("nan"))
        a = torch.full_like(s_dev, float("nan"))
        op.apply(s_dev, u, nrhs)
        op.apply_adjoint(s_dev, a, nrhs)
        torch.cuda.synchronize()
        outs[tune] = (u.cpu().numpy(), a.cpu().numpy())
        mt = (nrhs + 15) // 16
        shapes[tune] = (op.launch_shape(False, mt), op.launch_shape(True, mt))
        op.close()
    # the dataflow launch computes the same chains as the per-depth launches;
    # the tuned shape equals the forced shape of the same mode (mode 2 = the
    # tensor-core leaf kernel, whose leaf sums differ in rounding)
    assert np.array_equal(outs[2][0], outs[0][0]) and np.array_equal(outs[2][1], outs[0][1])
    # the cone launch and the fused level pairs run the same chains too
    assert np.array_equal(outs[4][0], outs[0][0]) and np.array_equal(outs[4][1], outs[0][1])
    assert np.array_equal(outs[5][0], outs[0][0]) and np.array_equal(outs[5][1], outs[0][1])
    assert np.array_equal(outs[6][0], outs[0][0]) and np.array_equal(outs[6][1], outs[0][1])
    for d in (0, 1):
        ref = {0: outs[0][d], 1: outs[0][d], 3: outs[0][d], 5: outs[0][d], 7: outs[0][d],
               2: outs[3][d], 4: outs[3][d], 6: outs[3][d]}[shapes[1][d]["mode"]]
        assert np.array_equal(outs[1][d], ref), d
    assert np.all(np.isfinite(outs[0][0])) and np.all(np.isfinite(outs[0][1]))
    assert shapes[0][0]["mode"] == 0 and shapes[0][1]["mode"] == 0
    assert shapes[2][0]["mode"] == 1 and shapes[2][1]["mode"] == 1
    assert shapes[3][0]["mode"] == 2 and shapes[3][1]["mode"] == 2
    assert shapes[4][0]["mode"] == 3 and shapes[4][1]["mode"] == 3
    assert shapes[5][0]["mode"] == 5 and shapes[5][1]["mode"] == 5
    assert shapes[6][0]["mode"] == 7 and shapes[6][1]["mode"] == 7
    for sh in shapes[1]:
        assert sh["mode"] in (0, 1, 2, 3, 4, 5, 6, 7) and sh["candidates"] >= 4 and sh["tuned_ms"] > 0


def test_dataflow_replays_and_alternating_directions():
    """Many launches on one handle (the readiness words count launches):
    forward and adjoint alternate, at one and two m-tiles, and every repeat
    is bitwise equal to the first."""
    import torch
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.GRADIENT, 64, 8, 20)
    s_dev = to_dev(W.complex_normal_sources(w.grid.Nv, 20, 5))
    op = gpu_op(w, precision=binding.HB_MIXED_BF16X3, autotune=2)
    op.build()
    first = {}
    for rep in range(6):
        for adj in (False, True):
            for R in (20, 7):
                u = torch.full((R, w.grid.Nv), float("nan"), dtype=torch.complex128, device="cuda")
                (op.apply_adjoint if adj else op.apply)(s_dev[:R].contiguous(), u, R)
                torch.cuda.synchronize()
                got = u.cpu().numpy()
                key = (adj, R)
                if key in first:
                    assert np.array_equal(got, first[key]), (rep, key)
                else:
                    first[key] = got
    op.close()
