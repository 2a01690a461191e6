"""hb_id_batch_noalloc, the entry point for callers that cannot allocate
device memory (code under another framework's memory manager, or on a
latency-critical path that must not take cudaMalloc's implicit
synchronisation).  It must give the same ranks, pivot orders and V matrices
as the allocating hb_id_batch, call after call, although every call shares
one static device array.  Collected last on purpose (file name), so a run
that stops at the first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from paper_2210_02698_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2210_02698_gb300 import build
    build.build()


def _pack(mats):
    import torch
    m = np.array([a.shape[0] for a in mats], dtype=np.int32)
    n = np.array([a.shape[1] for a in mats], dtype=np.int32)
    off = np.concatenate([[0], np.cumsum(m.astype(np.int64) * n)[:-1]]).astype(np.int64)
    flat = np.concatenate([a.T.reshape(-1) for a in mats])
    A = torch.from_numpy(flat).to("cuda")
    rank = torch.zeros(len(mats), dtype=torch.int32, device="cuda")
    skel = torch.full((int(n.sum()),), -1, dtype=torch.int32, device="cuda")
    V = torch.zeros(int((n.astype(np.int64) ** 2).sum()), dtype=torch.complex128, device="cuda")
    return m, n, off, A, rank, skel, V


def _mats(seed, count, m, n, rank, decay):
    A = W.random_id_matrices(count, m, n, rank, decay, seed=seed)
    return [A[b].T.copy() for b in range(count)]


@pytest.mark.parametrize("call", [0])
def test_noalloc_matches_allocating_entry_point_two_calls_in_a_row(call):
    import torch
    from paper_2210_02698_gb300 import binding
    # two different batches back to back: the second must not see the first's metadata
    batches = [_mats(11, 5, 200, 48, 40, 0.7) + _mats(12, 3, 37, 90, 25, 0.5),
               _mats(13, 9, 120, 30, 30, 0.6)]
    stream = torch.cuda.current_stream()
    for mats in batches:
        m, n, off, A1, r1, s1, V1 = _pack(mats)
        _, _, _, A2, r2, s2, V2 = _pack(mats)
        binding.id_batch(A1, m, n, off, 1e-6, r1, s1, V1)
        binding.id_batch_noalloc(A2, m, n, off, 1e-6, r2, s2, V2, stream)
        torch.cuda.synchronize()
        assert torch.equal(r1, r2)
        assert torch.equal(s1, s2)
        # same kernels on the same data: within the ID parity tolerance
        assert float((V1 - V2).abs().max()) <= 1e-12 * max(1.0, float(V1.abs().max()))


def test_noalloc_pinned_host_arrays_may_be_overwritten_on_return():
    """The size and offset arrays may live in page-locked memory; the call
    has consumed them when it returns, so overwriting them at once (before
    the stream has run anything) changes nothing."""
    import torch
    from paper_2210_02698_gb300 import binding
    mats = _mats(21, 6, 150, 40, 32, 0.6) + _mats(22, 4, 60, 70, 40, 0.5)
    m, n, off, A1, r1, s1, V1 = _pack(mats)
    _, _, _, A2, r2, s2, V2 = _pack(mats)
    binding.id_batch(A1, m, n, off, 1e-6, r1, s1, V1)
    torch.cuda.synchronize()
    pm = torch.from_numpy(m).pin_memory()
    pn = torch.from_numpy(n).pin_memory()
    po = torch.from_numpy(off).pin_memory()
    L = binding.lib()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        # keep the stream busy so that its copies cannot have run yet
        torch.cuda._sleep(50_000_000)
        st = L.hb_id_batch_noalloc(len(m), pm.data_ptr(), pn.data_ptr(), po.data_ptr(), C.c_void_p(A2.data_ptr()),
                                   1e-6, C.c_void_p(r2.data_ptr()), C.c_void_p(s2.data_ptr()),
                                   C.c_void_p(V2.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert st == binding.HB_OK
        # a different batch (every matrix 1 x 1 at offset 0: in bounds of
        # every buffer, but with other results) if the copies read it now
        pm.fill_(1)
        pn.fill_(1)
        po.fill_(0)
    torch.cuda.synchronize()
    assert torch.equal(r1, r2)
    assert torch.equal(s1, s2)
    assert float((V1 - V2).abs().max()) <= 1e-12 * max(1.0, float(V1.abs().max()))


@pytest.mark.parametrize("count,shape", [(3000, (4, 3)), (65536, (3, 2))])
def test_noalloc_many_small_matrices(count, shape):
    """Counts above 1024 give several matrices to each thread of the offset
    scan; 65536 is the largest count the static array takes."""
    import torch
    from paper_2210_02698_gb300 import binding
    rng = np.random.default_rng(count)
    mm, nn = shape
    flat = (rng.standard_normal((count, nn, mm)) + 1j * rng.standard_normal((count, nn, mm))).reshape(-1)
    m = np.full(count, mm, dtype=np.int32)
    n = np.full(count, nn, dtype=np.int32)
    off = (np.arange(count, dtype=np.int64) * mm * nn)
    out = []
    for noalloc in (False, True):
        A = torch.from_numpy(flat.copy()).to("cuda")
        rank = torch.zeros(count, dtype=torch.int32, device="cuda")
        skel = torch.full((count * nn,), -1, dtype=torch.int32, device="cuda")
        V = torch.zeros(count * nn * nn, dtype=torch.complex128, device="cuda")
        if noalloc:
            binding.id_batch_noalloc(A, m, n, off, 1e-6, rank, skel, V, torch.cuda.current_stream())
        else:
            binding.id_batch(A, m, n, off, 1e-6, rank, skel, V)
        torch.cuda.synchronize()
        out.append((rank, skel, V))
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])
    assert torch.equal(out[0][2], out[1][2])


def test_noalloc_rejects_counts_beyond_the_static_limit():
    import torch
    from paper_2210_02698_gb300 import binding
    L = binding.lib()
    count = 65537
    m = np.ones(count, dtype=np.int32)
    n = np.ones(count, dtype=np.int32)
    off = np.arange(count, dtype=np.int64)
    # real buffers of the full size; the size check rejects the call before any use
    A = torch.zeros(count, dtype=torch.complex128, device="cuda")
    rank = torch.zeros(count, dtype=torch.int32, device="cuda")
    skel = torch.zeros(count, dtype=torch.int32, device="cuda")
    V = torch.zeros(count, dtype=torch.complex128, device="cuda")
    st = L.hb_id_batch_noalloc(count, m.ctypes.data, n.ctypes.data, off.ctypes.data, C.c_void_p(A.data_ptr()),
                               1e-6, C.c_void_p(rank.data_ptr()), C.c_void_p(skel.data_ptr()),
                               C.c_void_p(V.data_ptr()), None)
    assert st == binding.HB_ERR_ARG
    assert b"65536" in L.hb_last_error(None)
