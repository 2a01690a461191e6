"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports
every symbol include/hb.h declares, and rejects bad arguments without a GPU."""
import ctypes as C
import shutil

import numpy as np
import pytest

from tests._common import header_symbols


@pytest.fixture(scope="module")
def L():
    if shutil.which("nvcc") is None and not __import__("os").path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2210_02698_gb300 import binding, build
    build.build()
    return binding.lib()


def test_every_declared_symbol_is_exported(L):
    from paper_2210_02698_gb300 import binding
    syms = header_symbols()
    assert set(syms) == set(binding.EXPORTS)
    for s in syms:
        assert hasattr(L, s), s


def test_argument_errors_without_compute(L):
    from paper_2210_02698_gb300 import binding
    hnd = C.c_void_p()
    # null arguments -> HB_ERR_ARG, message kept per thread
    assert L.hb_create(None, None, 1.0, None, C.byref(hnd)) == binding.HB_ERR_ARG
    assert b"null" in L.hb_last_error(None)
    g = binding.Grid(4, 4, 0.0, 0.0, 0.25)
    nodes = np.linspace(0.1, 0.9, 3)
    tab = np.zeros((9, 9))
    nc = np.ones(16)
    t = binding.Tables(3, nodes.ctypes.data, nodes.ctypes.data, tab.ctypes.data, tab.ctypes.data,
                       tab.ctypes.data, nc.ctypes.data)
    o = binding.Options(1e-6, 4, 20.0, 10.0, 0, 0, 0)
    assert L.hb_create(C.byref(g), C.byref(t), -1.0, C.byref(o), C.byref(hnd)) == binding.HB_ERR_ARG
    bad = binding.Options(0.0, 4, 20.0, 10.0, 0, 0, 0)
    assert L.hb_create(C.byref(g), C.byref(t), 5.0, C.byref(bad), C.byref(hnd)) == binding.HB_ERR_ARG
    t17 = binding.Tables(17, nodes.ctypes.data, nodes.ctypes.data, tab.ctypes.data, tab.ctypes.data,
                         tab.ctypes.data, nc.ctypes.data)
    assert L.hb_create(C.byref(g), C.byref(t17), 5.0, C.byref(o), C.byref(hnd)) == binding.HB_ERR_UNSUPPORTED
    assert L.hb_apply(None, None, None, 1, None) == binding.HB_ERR_ARG
    assert L.hb_id_batch(-1, None, None, None, None, 1e-6, None, None, None) == binding.HB_ERR_ARG
    L.hb_destroy(None)


def test_no_device_is_an_error_not_a_fallback(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2210_02698_gb300 import binding
    g = binding.Grid(4, 4, 0.0, 0.0, 0.25)
    nodes = np.linspace(0.1, 0.9, 3)
    tab = np.zeros((9, 9))
    nc = np.ones(16)
    t = binding.Tables(3, nodes.ctypes.data, nodes.ctypes.data, tab.ctypes.data, tab.ctypes.data,
                       tab.ctypes.data, nc.ctypes.data)
    o = binding.Options(1e-6, 4, 20.0, 10.0, 0, 0, 0)
    hnd = C.c_void_p()
    assert L.hb_create(C.byref(g), C.byref(t), 5.0, C.byref(o), C.byref(hnd)) == binding.HB_ERR_CUDA


def test_device_alloc_cap_is_host_state(L):
    """hb_device_alloc_cap only sets a number and reports the library's live
    device bytes (none before any handle exists): no device work."""
    from paper_2210_02698_gb300 import binding
    live = binding.device_alloc_cap(-1)
    assert live >= 0
    try:
        assert binding.device_alloc_cap(1 << 20) == live
        assert binding.device_alloc_cap(-1) == live
    finally:
        binding.device_alloc_cap(0)


def test_device_buffers_are_checked_before_any_call():
    """The binding refuses buffers the library would read as device
    complex128 memory: host arrays, CPU tensors, other dtypes, strided
    views, too few elements (HB_ERR_ARG before the library is called)."""
    import torch
    from paper_2210_02698_gb300 import binding

    class FakeCuda:
        """Stands for a CUDA tensor (none exists on this host)."""
        def __init__(self, dtype="torch.complex128", contiguous=True, numel=8):
            self.is_cuda, self.dtype, self._c, self._n = True, dtype, contiguous, numel

        def data_ptr(self):
            return 4096

        def is_contiguous(self):
            return self._c

        def numel(self):
            return self._n

    assert binding._device_buf(FakeCuda(), 8, "s") == 4096
    assert binding._device_buf(1234, 8, "s") == 1234          # a raw address passes unchecked
    bad = [np.zeros(8, dtype=np.complex128), torch.zeros(8, dtype=torch.complex128),
           FakeCuda(dtype="torch.complex64"), FakeCuda(contiguous=False), FakeCuda(numel=7), None]
    for b in bad:
        with pytest.raises(binding.HBError) as e:
            binding._device_buf(b, 8, "s")
        assert e.value.status == binding.HB_ERR_ARG


def test_id_batch_buffers_checked_as_the_gpu_tests_build_them():
    """The size rules of the ID entry points accept buffers built exactly
    as the GPU tests build them (CPU tensors standing in for CUDA ones) and
    refuse a short or mistyped one."""
    import torch
    from paper_2210_02698_gb300 import binding, workloads as W

    class AsCuda:
        def __init__(self, t):
            self.t, self.is_cuda, self.dtype = t, True, t.dtype

        def data_ptr(self):
            return self.t.data_ptr()

        def is_contiguous(self):
            return self.t.is_contiguous()

        def numel(self):
            return self.t.numel()

    rng = np.random.default_rng(3)
    a = rng.standard_normal(10) + 1j * rng.standard_normal(10)
    A3 = W.random_id_matrices(3, 37, 90, 25, 0.5, seed=12)
    mats = [np.stack([a, a, 0.5 * a], axis=1), np.zeros((5, 4), dtype=complex),
            rng.standard_normal((1, 6)) + 0j] + [A3[b].T.copy() for b in range(3)]
    m = np.array([x.shape[0] for x in mats], dtype=np.int32)
    n = np.array([x.shape[1] for x in mats], dtype=np.int32)
    off = np.concatenate([[0], np.cumsum(m.astype(np.int64) * n)[:-1]]).astype(np.int64)
    A = torch.from_numpy(np.concatenate([x.T.reshape(-1) for x in mats]))
    rank = torch.zeros(len(mats), dtype=torch.int32)
    skel = torch.zeros(int(n.sum()), dtype=torch.int32)
    V = torch.zeros(int((n.astype(np.int64) ** 2).sum()), dtype=torch.complex128)
    bufs = [AsCuda(t) for t in (A, rank, skel, V)]
    binding._id_args(bufs[0], m, n, off, *bufs[1:])
    for k, bad in enumerate([A[:-1], rank.to(torch.int64), skel[:-1], V.to(torch.complex64)]):
        b = list(bufs)
        b[k] = AsCuda(bad)
        with pytest.raises(binding.HBError) as e:
            binding._id_args(b[0], m, n, off, *b[1:])
        assert e.value.status == binding.HB_ERR_ARG


def test_factor_file_reader_rejects_corrupt_files_without_a_device(L, tmp_path):
    """hb_load parses the whole header before it needs a device, so on this
    host a valid file reaches the device check (HB_ERR_CUDA; HB_OK where a
    GPU exists) while truncated files and corrupt counts are refused with
    HB_ERR_ARG - a count larger than the file is refused before anything is
    allocated for it."""
    import torch
    from paper_2210_02698_gb300 import binding
    from tests.test_oracle_factor_file import _write

    path = tmp_path / "ok.hbf"
    _write(str(path), np.random.default_rng(2), nx=8, ny=8, leaf_pts=16, Lv=2, n_I=2)
    data = path.read_bytes()

    def load(blob):
        p = tmp_path / "x.hbf"
        p.write_bytes(blob)
        h = C.c_void_p()
        st = L.hb_load(str(p).encode(), C.byref(h))
        if st == binding.HB_OK:
            L.hb_destroy(h)
        return st

    expect_ok = binding.HB_OK if torch.cuda.is_available() else binding.HB_ERR_CUDA
    assert load(data) == expect_ok
    header = 8 + 8 * 14 + 8 * 2 * 2 + 8 * 3 * 16 + 8 * 64      # through n_cells
    for cut in (0, 7, 8, 20, 100, header - 1):
        assert load(data[:cut]) == binding.HB_ERR_ARG, cut
    for cut in (header + 8, len(data) // 2, len(data) - 1):
        assert load(data[:cut]) in (binding.HB_ERR_ARG, binding.HB_ERR_CUDA), cut
    big = np.frombuffer(data, dtype=np.uint8).copy()
    big[8:24] = np.frombuffer(np.array([1 << 31, 1 << 31], dtype="<i8").tobytes(), dtype=np.uint8)
    assert load(big.tobytes()) == binding.HB_ERR_ARG        # N_v = 2^62 cells: refused by size
    bad_magic = b"XBFACT01" + data[8:]
    assert load(bad_magic) == binding.HB_ERR_ARG


@pytest.mark.parametrize("N,leaf", [(32, 64), (24, 20), (64, 64), (37, 10), (9, 64), (256, 64)])
def test_host_tree_and_proxy_rows_match_oracle(L, N, leaf):
    """The library's cluster tree and proxy-row rule (host code of hb_create /
    hb_build, Sec. 4.2 and Eq. proxyv2v) equal the oracle's bit for bit,
    without a device."""
    from oracle import tree
    from paper_2210_02698_gb300 import binding
    perm, bounds = binding.host_cluster_tree(N, N, leaf)
    operm, obounds = tree.cluster_tree(N, leaf)
    assert np.array_equal(perm, operm)
    assert len(bounds) == len(obounds) and all(np.array_equal(a, b) for a, b in zip(bounds, obounds))
    rng = np.random.default_rng(N + leaf)
    for lvl in range(1, len(bounds)):
        for _ in range(3):
            k = int(rng.integers(0, (1 << lvl) - 1))
            t0, t1 = int(bounds[lvl][k]), int(bounds[lvl][k + 1])
            s0, s1 = int(bounds[lvl][k + 1]), int(bounds[lvl][k + 2])
            if s1 <= s0 or t1 <= t0:
                continue
            seeds = rng.choice(np.arange(s0, s1), size=min(s1 - s0, int(rng.integers(1, 9))), replace=False)
            for chi, radius in ((20.0, 10.0), (2.0, 3.5)):
                want = tree.proxy_rows(t0, t1, seeds, chi, radius, operm, N)
                got = binding.host_proxy_rows(N, N, leaf, chi, radius, t0, t1, seeds)
                assert np.array_equal(got, want), (lvl, k, chi, radius)


def test_host_tree_on_rectangular_grids(L):
    from paper_2210_02698_gb300 import binding
    for nx, ny, leaf in ((40, 7, 16), (5, 33, 8), (1, 100, 7)):
        perm, bounds = binding.host_cluster_tree(nx, ny, leaf)
        assert sorted(perm.tolist()) == list(range(nx * ny))
        assert bounds[-1][-1] == nx * ny and np.max(np.diff(bounds[-1])) <= leaf
        for l in range(1, len(bounds)):
            assert np.array_equal(bounds[l][::2], bounds[l - 1])
    with pytest.raises(binding.HBError):
        binding.host_cluster_tree(0, 5, 4)


def test_host_segment_tree_matches_oracle(L):
    """The library's segment K-D tree (the column tree of the compressed
    surface operators) equals the oracle prototype's bit for bit: a circle,
    an open square (equal coordinates along its sides) and random points
    with repeated coordinates (ties broken by segment index)."""
    from oracle import curve_butterfly, inclusion
    from paper_2210_02698_gb300 import binding, workloads as W
    rng = np.random.default_rng(12)
    sets = [W.circle_segments((0.5, 0.5), 0.3, 1000)[0],
            inclusion.polyline([(0.1, 0.1), (0.1, 0.9), (0.9, 0.9), (0.9, 0.1)], 333).c,
            np.round(rng.uniform(0, 1, size=(517, 2)), 1)]
    for cen in sets:
        for leaf in (1, 4, 37):
            perm, bounds = binding.host_segment_tree(cen, leaf)
            operm, obounds = curve_butterfly.segment_tree(cen, leaf)
            assert np.array_equal(perm, operm)
            assert len(bounds) == len(obounds) and all(np.array_equal(a, b) for a, b in zip(bounds, obounds))


def test_host_point_proxy_rows_match_oracle_prototype(L):
    """The native two-set proxy rule equals the compressed-inclusion
    prototype's (oracle/curve_butterfly.py) bit for bit: cells as rows with
    segment centres as seeds, and segments as rows with cells as seeds."""
    from types import SimpleNamespace
    from oracle import curve_butterfly as cb, tree
    from paper_2210_02698_gb300 import binding, workloads as W
    N = 32
    g = W.Grid(N)
    x, z = g.centroids()
    vperm, vb = tree.cluster_tree(N, 16)
    cells = np.stack([x, z], axis=1)[vperm]
    cen, _ = W.circle_segments((0.5, 0.5), 0.25, 256)
    sperm, sb = cb.segment_tree(cen, 4)
    segs = cen[sperm]
    rng = np.random.default_rng(5)
    for rows, cols, rb, cbounds in ((cells, segs, vb, sb), (segs, cells, sb, vb)):
        for chi, radius in ((20.0, 10.0 / N), (1.5, 3.0 / N), (0.5, 0.0)):
            obj = SimpleNamespace(chi=chi, radius=radius, rows=SimpleNamespace(pts=rows),
                                  cols=SimpleNamespace(pts=cols))
            for lvl in (1, 3, 5):
                k = int(rng.integers(0, 1 << lvl))
                t0, t1 = int(rb[lvl][k]), int(rb[lvl][k + 1])
                seeds = rng.choice(len(cols), size=int(rng.integers(1, 6)), replace=False)
                want = cb.Butterfly._proxy(obj, t0, t1, seeds)
                got = binding.host_point_proxy_rows(rows, t0, t1, cols[seeds], chi, radius)
                assert np.array_equal(got, want), (lvl, chi, radius)


def test_binding_methods_marshal_through_a_null_handle(L):
    """The binding's handle methods reach the library with well-formed
    arguments: on an Operator whose handle is NULL each call comes back as
    HB_ERR_ARG (null handle) rather than a ctypes argument error."""
    from paper_2210_02698_gb300 import binding
    op = binding.Operator.__new__(binding.Operator)
    op.handle = None
    calls = [lambda: op.launch_shape(False, 1), lambda: op.launch_shape(True, 2),
             lambda: op.record_id_blocks(4), lambda: op.recorded_id_blocks(), lambda: op.info(),
             lambda: op.tree_perm() if hasattr(op, "Nv") else op._call("hb_tree_perm", None),
             lambda: op.set_kernel_timing(True), lambda: op.set_precision(binding.HB_FP64),
             lambda: op.set_omega(2.0), lambda: op.curve_compress(16), lambda: op.curve_info(0)]
    for f in calls:
        with pytest.raises(binding.HBError) as e:
            f()
        assert e.value.status == binding.HB_ERR_ARG
    v = C.c_double()
    assert L.hb_fp64_fma_peak(None, None) == binding.HB_ERR_ARG


def test_table_builder_arguments_need_no_device(L):
    """hb_sweep_tables checks its mesh, sizes and node indices before any
    device call, so the errors come back without a GPU."""
    from paper_2210_02698_gb300 import binding
    M = 16
    n = np.ones((M, M))
    px = pz = np.array([0.25, 0.75])
    tin = np.zeros((1, 46))
    tin[0, 0] = 1.0
    src = np.array([0], dtype=np.int32)
    for bad in ((M, 0.0, 0.1, 2, M, 0, 4), (M, 0.0, -0.1, 2, 12, 0, 4), (4, 0.0, 0.1, 0, 3, 0, 1),
                (M, 0.0, 0.1, 2, 12, 0, 11)):
        with pytest.raises(binding.HBError) as e:
            binding.sweep_tables(*bad, n[:bad[0], :bad[0]], px, pz, src, tin)
        assert e.value.status == binding.HB_ERR_ARG
    with pytest.raises(binding.HBError) as e:
        binding.sweep_tables(M, 0.0, 0.1, 2, 12, 0, 4, n, px, pz, np.array([2], dtype=np.int32), tin)
    assert e.value.status == binding.HB_ERR_ARG        # node index out of range
    bad_t = tin.copy()
    bad_t[0, 0] = 0.0
    with pytest.raises(binding.HBError) as e:
        binding.sweep_tables(M, 0.0, 0.1, 2, 12, 0, 4, n, px, pz, src, bad_t)
    assert e.value.status == binding.HB_ERR_ARG        # S0 = n0^2 must be positive
