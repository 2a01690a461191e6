"""The compressed inclusion operators (hb_curve_compress; Sec. 4.2's
K^{v2s} / K^{s2v} items, each one butterfly between the cells' cluster
tree and the segments' K-D tree, Sec. 4.2.1) against the oracle: the total
field (Eq. m_v2v_inclu) with the butterflies in place of the dense
K^{v2s}, K^{s2v} agrees with the dense oracle (oracle/inclusion.py, pinned
against the exact circle-scattering series) and with the library's dense
path to the compression tolerance (eps = 1e-6, FP64), for interior and
boundary-hugging curves, several right-hand sides; the butterflies have the
levels of the cut trees and store fewer entries than the dense operators;
a new curve drops them."""
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


@pytest.mark.parametrize("N,ns,centre,radius,leaf_s", [(48, 256, (0.5, 0.5), 0.3, 16),
                                                        (32, 192, (0.45, 0.55), 0.4, 8)])
def test_compressed_total_field(N, ns, centre, radius, leaf_s):
    import torch
    from oracle import inclusion
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.GRADIENT, N, N / 8, 3, leaf=32)
    cen, lw = W.circle_segments(centre, radius, ns)
    nseg = W.GRADIENT.n(cen[:, 0], cen[:, 1])
    s = W.complex_normal_sources(w.grid.Nv, 3, 71)
    want, _ = inclusion.total_field(oracle_op(w), inclusion.Curve(cen, lw), W.GRADIENT.n, s)
    gp = gpu_op(w, precision=binding.HB_FP64)
    gp.set_curve(cen, lw, nseg)
    u_dense = torch.empty((3, w.grid.Nv), dtype=torch.complex128, device="cuda")
    gp.apply_inclusion(to_dev(s), u_dense, 3, v2v_dense=True)
    gp.curve_compress(leaf_s)
    u_bf = torch.empty_like(u_dense)
    gp.apply_inclusion(to_dev(s), u_bf, 3, v2v_dense=True)
    torch.cuda.synchronize()
    dense, bf = from_dev(u_dense), from_dev(u_bf)
    assert rel_l2(dense, want) < 1e-10
    assert rel_l2(bf, want) < 1e-5
    assert rel_l2(bf, dense) < 1e-5
    # the inclusion's part of the field is what the butterflies carry
    free = dense - from_dev(_free_field(gp, s, w))
    assert rel_l2(bf - from_dev(_free_field(gp, s, w)), free) < 1e-4
    Lv = gp.info()["levels"]
    for which in (0, 1):
        levels, max_rank, entries = gp.curve_info(which)
        assert 1 <= levels <= Lv and 1 <= max_rank <= ns
        assert entries < ns * w.grid.Nv
    # a new curve drops the compressed operators
    gp.set_curve(cen, lw, nseg)
    with pytest.raises(binding.HBError) as e:
        gp.curve_info(0)
    assert e.value.status == binding.HB_ERR_STATE
    gp.close()


def _free_field(gp, s, w):
    import torch
    u = torch.empty((s.shape[1], w.grid.Nv), dtype=torch.complex128, device="cuda")
    gp.apply_dense(to_dev(s), u, s.shape[1])
    torch.cuda.synchronize()
    return u


def test_compress_arguments():
    from paper_2210_02698_gb300 import binding
    w = W.small_workload(W.GRADIENT, 32, 4, 1)
    gp = gpu_op(w)
    with pytest.raises(binding.HBError) as e:
        gp.curve_compress(16)                       # no curve yet
    assert e.value.status == binding.HB_ERR_STATE
    cen, lw = W.circle_segments((0.5, 0.5), 0.2, 64)
    gp.set_curve(cen, lw, W.GRADIENT.n(cen[:, 0], cen[:, 1]))
    with pytest.raises(binding.HBError) as e:
        gp.curve_compress(0)
    assert e.value.status == binding.HB_ERR_ARG
    gp.close()
