"""The largest configuration in full: 2048^2 cells (N_v = 4,194,304) of the
constant-gradient medium c = 1 + 0.5 z at w = 2 pi 256 (8 cells per
wavelength), eps = 1e-6, 128 complex Gaussian right-hand sides, mixed
precision (Sec. 4.2 HODBF, Sec. 4.2.1 butterflies; ~5e9 stored factor
entries, so every factor and tile offset runs past 2^31).  16 seeded rows
of the forward apply and 16 seeded columns of the adjoint against the dense
oracle, each right-hand side within 1e-4."""
import numpy as np
import pytest

from paper_2210_02698_gb300 import workloads as W
from tests._common import gpu_op, oracle_dense_rows, rel_l2

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_grad2048_128_rhs_sampled_rows_and_columns():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_02698_gb300 import binding, build
    build.build()
    w = W.WORKLOADS["grad2048"]
    s = W.workload_sources(w)
    R = s.shape[1]
    import time
    t0 = time.perf_counter()
    gp = gpu_op(w, precision=binding.HB_MIXED_BF16X3)
    gp.build()
    t_build = time.perf_counter() - t0
    assert gp.info()["factor_entries"] > (1 << 32)
    rows = W.sample_rows(w.grid.Nv, 16, 20480)
    cols = W.sample_rows(w.grid.Nv, 16, 20481)
    s_dev = torch.from_numpy(np.ascontiguousarray(s.T)).cuda()
    u = torch.empty_like(s_dev)
    gp.apply(s_dev, u, R)
    got = u[:, torch.from_numpy(rows).cuda()].cpu().numpy().T
    gp.apply_adjoint(s_dev, u, R)
    gotA = u[:, torch.from_numpy(cols).cuda()].cpu().numpy().T
    del s_dev, u
    gp.close()
    torch.cuda.empty_cache()
    t0 = time.perf_counter()
    want = oracle_dense_rows(w, s, rows)
    wantA = oracle_dense_rows(w, s, cols, adjoint=True)
    print(f"grad2048 build {t_build:.0f} s, oracle rows {time.perf_counter() - t0:.0f} s")
    col = lambda a, b: float(np.max(np.linalg.norm(a - b, axis=0) / np.linalg.norm(b, axis=0)))  # noqa: E731
    print("grad2048 mixed rel-L2 forward", rel_l2(got, want), "worst column", col(got, want),
          "adjoint", rel_l2(gotA, wantA), "worst column", col(gotA, wantA))
    assert rel_l2(got, want) < 1e-4 and col(got, want) < 1e-4
    assert rel_l2(gotA, wantA) < 1e-4 and col(gotA, wantA) < 1e-4
