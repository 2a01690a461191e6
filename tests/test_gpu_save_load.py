"""hb_save / hb_load: a reloaded operator applies bit-identically (same
factors, same plans), and the oracle's CPU butterfly apply over the saved
file (oracle/factor_file.py, the format documented with hb_save) agrees with
the GPU FP64 butterfly apply to rounding and with the dense oracle to the
compression error (Sec. 4.2, Sec. 4.2.1)."""
import numpy as np
import pytest

from paper_2210_02698_gb300 import workloads as W
from tests._common import gpu_op, oracle_op, rel_l2, to_dev, from_dev


@pytest.mark.gpu
def test_save_load_roundtrip_and_oracle_file_apply(tmp_path):
    import torch
    from paper_2210_02698_gb300 import binding
    from oracle import dense
    from oracle.factor_file import FactorFile
    w = W.small_workload(W.GRADIENT, 64, 8, 3)
    s = W.workload_sources(w)
    R = s.shape[1]
    s_dev = to_dev(s)

    op = gpu_op(w, precision=binding.HB_FP64)
    with pytest.raises(binding.HBError) as e:
        op.save(tmp_path / "early.hbf")
    assert e.value.status == binding.HB_ERR_STATE
    with pytest.raises(binding.HBError) as e:
        op.rank_profile()
    assert e.value.status == binding.HB_ERR_STATE
    op.build()
    path = tmp_path / "op.hbf"
    op.save(path)

    def run(o, adjoint=False):
        u = torch.empty_like(s_dev)
        (o.apply_adjoint if adjoint else o.apply)(s_dev, u, R)
        torch.cuda.synchronize()
        return from_dev(u)

    u64, a64 = run(op), run(op, True)
    op.set_precision(binding.HB_MIXED_BF16X3)
    umx = run(op)

    ld = binding.Operator.load(path)
    assert (ld.nx, ld.ny) == (w.N, w.N)
    assert ld.info()["factor_entries"] == op.info()["factor_entries"]
    ld.set_precision(binding.HB_FP64)
    assert np.array_equal(run(ld), u64)
    assert np.array_equal(run(ld, True), a64)
    ld.set_precision(binding.HB_MIXED_BF16X3)
    assert np.array_equal(run(ld), umx)

    F = FactorFile(path)
    # ranks by HODBF level l and butterfly level k: the library's profile
    # against the ranks the file holds
    n = F.Lv + 1
    fmx, fsum, fcnt = np.zeros((n, n), dtype=np.int64), np.zeros((n, n)), np.zeros((n, n))
    for b in F.butterflies:
        for k in range(int(b["L"]) + 1):
            r = np.asarray(b["rank"][k], dtype=np.int64)
            l = int(b["l"])
            fmx[l, k] = max(fmx[l, k], int(r.max()))
            fsum[l, k] += r.sum()
            fcnt[l, k] += len(r)
    mx, mean = op.rank_profile()
    assert np.array_equal(mx, fmx) and mx.max() == op.info()["max_rank"]
    assert np.allclose(mean, np.divide(fsum, fcnt, out=np.zeros_like(fsum), where=fcnt > 0), rtol=1e-14, atol=0)
    lmx, lmean = ld.rank_profile()
    assert np.array_equal(lmx, mx) and np.array_equal(lmean, mean)
    assert rel_l2(F.apply(s), u64) < 1e-13
    assert rel_l2(F.apply_adjoint(s), a64) < 1e-13
    assert rel_l2(F.apply(s), dense.apply(oracle_op(w), s)) < 1e-5

    # a truncated file is rejected, nothing leaks into the context
    bad = tmp_path / "bad.hbf"
    bad.write_bytes(path.read_bytes()[:100000])
    with pytest.raises(binding.HBError) as e:
        binding.Operator.load(bad)
    assert e.value.status == binding.HB_ERR_ARG
    op.close()
    ld.close()
