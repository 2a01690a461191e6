"""The leaf outputs on the 5th-generation tensor cores (csrc/leaf_tc.cu:
tcgen05.mma with accumulators in tensor memory; Sec. 4.2 HODBF, the dense
leaf blocks and the K^L / V^0^H terms of every butterfly) against the dense
oracle and the FP64 butterfly, forward and adjoint: one and two m-tiles,
leaves of 64, of 32, ragged leaves (41 and 40 cells), leaves of more than
64 cells (two tensor-core chains per leaf), odd numbers of 8-input groups
(the zero-block tail).  Bars as for the mixed apply: rel-L2 1e-4 against
the oracle, every right-hand side on its own."""
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


def _apply(op, s, adjoint=False):
    import torch
    out = torch.full((s.shape[1], s.shape[0]), float("nan"), dtype=torch.complex128, device="cuda")
    (op.apply_adjoint if adjoint else op.apply)(to_dev(s), out, s.shape[1])
    torch.cuda.synchronize()
    return from_dev(out)


def _worst_col(a, b):
    return float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))


@pytest.mark.parametrize("N,leaf,nrhs", [(32, 64, 3), (48, 32, 2), (64, 64, 4), (48, 64, 24), (9, 64, 3),
                                         (40, 100, 17), (24, 20, 5)])
def test_tensor_core_leaves_vs_dense_oracle(N, leaf, nrhs):
    from oracle import dense
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.GRADIENT, N, N / 8, nrhs, leaf=leaf)
    og = oracle_op(w)
    gp = gpu_op(w, precision=binding.HB_MIXED_BF16X3, autotune=3)
    gp.build()
    s = W.complex_normal_sources(w.grid.Nv, nrhs, 91)
    want, wantA = dense.apply(og, s), dense.adjoint(og, s)
    got, gotA = _apply(gp, s), _apply(gp, s, True)
    mt = (min(nrhs, 32) + 15) // 16
    assert gp.launch_shape(False, mt)["mode"] == 2 and gp.launch_shape(True, mt)["mode"] == 2
    assert rel_l2(got, want) < 1e-4 and _worst_col(got, want) < 1e-4
    assert rel_l2(gotA, wantA) < 1e-4 and _worst_col(gotA, wantA) < 1e-4
    # against the FP64 butterfly of the same factors: only the mixed
    # arithmetic differs
    gp.set_precision(binding.HB_FP64)
    assert rel_l2(got, _apply(gp, s)) < 1e-4 and rel_l2(gotA, _apply(gp, s, True)) < 1e-4
    gp.close()


def test_tensor_core_leaves_replay_bitwise_and_in_graphs():
    """Ten replays give bitwise-equal outputs (no atomics in the leaf kernel),
    and the apply captured in a CUDA graph replays them."""
    import torch
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.GRADIENT, 64, 8, 16)
    gp = gpu_op(w, precision=binding.HB_MIXED_BF16X3, autotune=3)
    gp.build()
    s_dev = to_dev(W.complex_normal_sources(w.grid.Nv, 16, 7))
    outs = []
    for _ in range(10):
        u = torch.full_like(s_dev, float("nan"))
        gp.apply(s_dev, u, 16)
        torch.cuda.synchronize()
        outs.append(u.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])
    st = torch.cuda.Stream()
    u = torch.full_like(s_dev, float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        gp.apply(s_dev, u, 16, st)
    g.replay()
    torch.cuda.synchronize()
    assert np.array_equal(u.cpu().numpy(), outs[0])
    gp.close()
