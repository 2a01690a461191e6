"""The GPU table builder (hb_sweep_tables; Sec. 2.3 sweeping, Sec. 4.1
tables) against the oracle's FP64 builder (oracle/sweep.c) on the same
mesh, Taylor numbers and sources: one CTA per source updating each
anti-diagonal of a sweep in parallel computes the row-by-row Gauss-Seidel
iterates, so the tables and the iteration counts are equal bit for bit -
constant-gradient and lens media, interior, corner and edge nodes, the
lens at the mesh of the stored tables (h0 = 1/256) on sampled sources
(40 iterations per solve there).
With the Taylor numbers of hb_sweep_taylor the tables agree with the
oracle's to rounding.  Argument errors are reported without a launch."""
import numpy as np
import pytest

from oracle import chebyshev, sweep
from paper_2210_02698_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_02698_gb300 import build
    build.build()


def _case(medium, n_I, h0, src, margin=0.3):
    xn = chebyshev.nodes(n_I)
    px = np.ascontiguousarray(np.tile(xn, n_I))
    pz = np.ascontiguousarray(np.repeat(xn, n_I))
    M, lo, w0, w1, roi0, roi1 = sweep.mesh(h0, margin)
    n, _, _ = sweep.mesh_n(medium, M, lo, h0)
    tin = np.ascontiguousarray(np.stack([sweep.taylor_input(medium, px[j], pz[j]) for j in src]))
    return (M, lo, h0, w0, w1, roi0, roi1), n, px, pz, np.asarray(src, dtype=np.int32), tin


def _oracle(mesh, n, px, pz, src, tin, max_iter, tol):
    import ctypes
    M, lo, h0, w0, w1, roi0, roi1 = mesh
    NI, ns = px.size, src.size
    t2, a0, a1 = (np.empty((NI, ns)) for _ in range(3))
    info = np.empty((ns, 6))
    p = sweep._p
    r = sweep.lib().hb_oracle_sweep_tables(M, lo, h0, w0, w1, roi0, roi1, p(n), NI, p(px), p(pz), ns,
                                           src.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), p(tin), max_iter,
                                           tol, p(t2), p(a0), p(a1), p(info))
    assert r == 0
    return t2, a0, a1, info


@pytest.mark.parametrize("medium,n_I,h0,src", [
    (W.GRADIENT, 4, 1 / 32, [0, 5, 15]),
    (W.LENS, 6, 1 / 48, [0, 7, 14, 20, 35]),
])
def test_tables_equal_the_oracle_bitwise(medium, n_I, h0, src):
    from paper_2210_02698_gb300 import binding
    mesh, n, px, pz, s, tin = _case(medium, n_I, h0, src)
    want = _oracle(mesh, n, px, pz, s, tin, 400, 1e-12)
    got = binding.sweep_tables(*mesh, n, px, pz, s, tin, 400, 1e-12)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    assert np.all(got[3][:, 3:5] < 1e-12)         # the eikonal and v0 solves converged


def test_lens_at_the_stored_mesh_on_sampled_sources():
    # 40 iterations per solve (the iterates, converged or not, are what is
    # compared; the full solves take minutes at this mesh)
    from paper_2210_02698_gb300 import binding
    mesh, n, px, pz, s, tin = _case(W.LENS, 16, 1 / 256, [0, 100, 255])
    want = _oracle(mesh, n, px, pz, s, tin, 40, 1e-12)
    got = binding.sweep_tables(*mesh, n, px, pz, s, tin, 40, 1e-12)
    for g, w in zip(got, want):
        assert np.array_equal(g, w)


def test_taylor_numbers_of_the_library():
    from paper_2210_02698_gb300 import binding
    mesh, n, px, pz, s, tin = _case(W.LENS, 6, 1 / 48, [3, 21])
    s2 = np.stack([np.concatenate([np.asarray(q, dtype=np.float64) for q in sweep.n2_series(W.LENS, px[j], pz[j], 4)])
                   for j in s])
    mine = binding.sweep_taylor(s2)
    want = _oracle(mesh, n, px, pz, s, tin, 400, 1e-12)
    got = binding.sweep_tables(*mesh, n, px, pz, s, mine, 400, 1e-12)
    for g, w in zip(got[:3], want[:3]):
        assert np.max(np.abs(g - w)) <= 1e-12 * np.max(np.abs(w))


def test_arguments():
    from paper_2210_02698_gb300 import binding
    mesh, n, px, pz, s, tin = _case(W.GRADIENT, 4, 1 / 32, [0])
    M, lo, h0, w0, w1, roi0, roi1 = mesh
    for bad in ((M, lo, h0, w0, M, roi0, roi1), (M, lo, -h0, w0, w1, roi0, roi1), (M, lo, h0, w0, w1, roi0, w1)):
        with pytest.raises(binding.HBError) as e:
            binding.sweep_tables(*bad, n, px, pz, s, tin)
        assert e.value.status == binding.HB_ERR_ARG
    with pytest.raises(binding.HBError) as e:
        binding.sweep_tables(*mesh, n, px, pz, np.array([16], dtype=np.int32), tin)   # node out of range
    assert e.value.status == binding.HB_ERR_ARG
