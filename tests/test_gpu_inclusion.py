"""GPU parity of the curve-inclusion path (Sec. 3.2: Eq. s2s, Eq. m_v2s,
Eq. m_s2v, Eq. m_v2v_inclu) against the oracle (oracle/inclusion.py, itself
pinned against the exact circle-scattering series in
tests/test_oracle_inclusion.py).

Bars (FP64): operator entries as the volume entries (max relative 1e-11 with
a floor, rel-L2 1e-12); the total field with the dense K^{v2v} rel-L2 1e-10
(the LU solve of K^{s2s} amplifies rounding by its condition number); with
the compressed FP64 K^{v2v} the compression tolerance (eps = 1e-6)."""
import numpy as np
import pytest

from tests._common import from_dev, gpu_op, load_tables, oracle_op, rel_l2, to_dev
from paper_2210_02698_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_02698_gb300 import build
    build.build()


def _case(medium, N=32, ns=64, nrhs=3):
    w = W.small_workload(medium, N, N / 8, nrhs)
    cen, lw = W.circle_segments((0.5, 0.5), 0.2, ns)
    nseg = medium.n(cen[:, 0], cen[:, 1])
    return w, cen, lw, nseg


def _oracle_curve(cen, lw):
    from oracle import inclusion
    return inclusion.Curve(cen, lw)


@pytest.mark.parametrize("medium", [W.HOMOGENEOUS, W.GRADIENT])
def test_curve_operators_match_oracle(medium):
    import torch
    from oracle import inclusion
    w, cen, lw, nseg = _case(medium)
    ns, Nv = len(lw), w.grid.Nv
    gp = gpu_op(w)
    gp.set_curve(cen, lw, nseg)
    s2s = torch.empty((ns, ns), dtype=torch.complex128, device="cuda")    # column-major ns x ns
    v2s = torch.empty((Nv, ns), dtype=torch.complex128, device="cuda")    # column-major ns x Nv
    s2v = torch.empty((ns, Nv), dtype=torch.complex128, device="cuda")    # column-major Nv x ns
    gp.curve_operators(s2s, v2s, s2v)
    torch.cuda.synchronize()
    tab = load_tables(medium)
    cur = _oracle_curve(cen, lw)
    x, z = w.grid.centroids()
    cells = np.stack([x, z], axis=1)
    n_of = medium.n
    pairs = [(s2s.cpu().numpy().T, inclusion.K_s2s(tab, w.omega, cur, n_of)),
             (v2s.cpu().numpy().T, inclusion.K_v2s(tab, w.omega, cur, cells)),
             (s2v.cpu().numpy().T, inclusion.K_s2v(tab, w.omega, cur, cells))]
    for got, want in pairs:
        assert got.shape == want.shape
        err = np.abs(got - want)
        assert np.max(err / (np.abs(want) + 1e-3 * np.max(np.abs(want)))) < 1e-11
        assert rel_l2(got, want) < 1e-12
    # the diagonal of K^{s2s} is the segment self term, not a kernel value
    d = np.diag(pairs[0][0])
    assert np.allclose(d, inclusion.s2s_self(lw, w.omega, nseg), rtol=1e-13, atol=0)


@pytest.mark.parametrize("medium", [W.HOMOGENEOUS, W.GRADIENT])
def test_total_field_matches_oracle(medium):
    import torch
    from oracle import inclusion
    from paper_2210_02698_gb300 import binding
    w, cen, lw, nseg = _case(medium)
    s = W.complex_normal_sources(w.grid.Nv, w.nrhs, 41)
    want, _ = inclusion.total_field(oracle_op(w), _oracle_curve(cen, lw), medium.n, s)
    gp = gpu_op(w, precision=binding.HB_FP64)
    gp.set_curve(cen, lw, nseg)
    u = torch.empty((w.nrhs, w.grid.Nv), dtype=torch.complex128, device="cuda")
    gp.apply_inclusion(to_dev(s), u, w.nrhs, v2v_dense=True)
    torch.cuda.synchronize()
    dense = from_dev(u)
    assert rel_l2(dense, want) < 1e-10
    # the compressed K^{v2v} (FP64 factors) within the compression tolerance
    gp.build()
    u2 = torch.empty_like(u)
    gp.apply_inclusion(to_dev(s), u2, w.nrhs)
    torch.cuda.synchronize()
    assert rel_l2(from_dev(u2), want) < 1e-5
    # the inclusion changes the field: its part is not negligible
    from oracle import dense as odense
    free = odense.apply(oracle_op(w), s)
    assert rel_l2(free, want) > 1e-2


def test_curve_state_and_argument_errors():
    import torch
    from paper_2210_02698_gb300 import binding
    w, cen, lw, nseg = _case(W.GRADIENT, ns=16)
    gp = gpu_op(w)
    s = to_dev(W.complex_normal_sources(w.grid.Nv, 1, 3))
    u = torch.empty_like(s)
    with pytest.raises(binding.HBError) as e:
        gp.apply_inclusion(s, u, 1, v2v_dense=True)
    assert e.value.status == binding.HB_ERR_STATE
    bad = lw.copy()
    bad[3] = -1.0
    with pytest.raises(binding.HBError) as e:
        gp.set_curve(cen, bad, nseg)
    assert e.value.status == binding.HB_ERR_ARG
    gp.set_curve(cen, lw, nseg)
    with pytest.raises(binding.HBError) as e:          # compressed K^{v2v} before hb_build
        gp.apply_inclusion(s, u, 1)
    assert e.value.status == binding.HB_ERR_STATE
    gp.apply_inclusion(s, u, 1, v2v_dense=True)
    first = u.clone()
    # a second curve replaces the first; setting the first again reproduces it
    cen2, lw2 = W.circle_segments((0.4, 0.6), 0.15, 24)
    gp.set_curve(cen2, lw2, W.GRADIENT.n(cen2[:, 0], cen2[:, 1]))
    gp.apply_inclusion(s, u, 1, v2v_dense=True)
    assert not torch.equal(u, first)
    gp.set_curve(cen, lw, nseg)
    gp.apply_inclusion(s, u, 1, v2v_dense=True)
    torch.cuda.synchronize()
    assert torch.equal(u, first)
