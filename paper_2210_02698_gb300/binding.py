"""ctypes binding of the C ABI declared in ``include/hb.h``.

Argument marshalling only: every computation runs in ``_lib/libhb.so``.
Tensors passed in are used through their data pointers (``torch.Tensor``
on CUDA for vectors, host numpy arrays for tables and index lists).
``lib()`` raises if the library is missing - there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libhb.so")

HB_OK, HB_ERR_ARG, HB_ERR_CUDA, HB_ERR_OOM, HB_ERR_TIMEOUT, HB_ERR_STATE, HB_ERR_UNSUPPORTED = range(7)
HB_FP64, HB_MIXED_BF16X3 = 0, 1
STATUS = {0: "HB_OK", 1: "HB_ERR_ARG", 2: "HB_ERR_CUDA", 3: "HB_ERR_OOM", 4: "HB_ERR_TIMEOUT",
          5: "HB_ERR_STATE", 6: "HB_ERR_UNSUPPORTED"}

# every symbol include/hb.h declares
EXPORTS = ["hb_create", "hb_build", "hb_set_omega", "hb_save", "hb_load", "hb_apply", "hb_apply_adjoint", "hb_set_precision",
           "hb_set_wait_selftest", "hb_device_alloc_cap",
           "hb_apply_dense", "hb_apply_dense_adjoint", "hb_entries", "hb_curve_set", "hb_curve_operators",
           "hb_apply_inclusion", "hb_curve_compress", "hb_curve_info", "hb_sweep_taylor", "hb_sweep_tables", "hb_id_batch", "hb_id_batch_noalloc",
           "hb_record_id_blocks", "hb_recorded_id_count", "hb_recorded_id_block", "hb_launch_shape", "hb_fp64_fma_peak",
           "hb_shard_rows", "hb_apply_shard", "hb_apply_shard_adjoint", "hb_host_shard_rows",
           "hb_tree_perm", "hb_proxy_rows", "hb_host_cluster_tree", "hb_host_proxy_rows", "hb_host_segment_tree", "hb_host_point_proxy_rows", "hb_info", "hb_rank_profile", "hb_set_kernel_timing",
           "hb_kernel_times", "hb_last_error", "hb_destroy"]


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("y0", C.c_double),
                ("h", C.c_double)]


class Tables(C.Structure):
    _fields_ = [("n_I", C.c_int), ("nodes_x", C.c_void_p), ("nodes_y", C.c_void_p),
                ("tau2", C.c_void_p), ("v0", C.c_void_p), ("v1", C.c_void_p),
                ("n_cells", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("eps", C.c_double), ("leaf", C.c_int), ("chi", C.c_double),
                ("nbr_radius_h", C.c_double), ("precision", C.c_int), ("workspace_mb", C.c_int),
                ("barrier_cycles", C.c_longlong), ("autotune", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("n_v", C.c_longlong), ("levels", C.c_int), ("max_rank", C.c_int),
                ("factor_entries", C.c_longlong), ("factor_bytes_fp64", C.c_longlong),
                ("factor_bytes_mixed", C.c_longlong), ("id_blocks", C.c_longlong),
                ("sampled_entries", C.c_longlong), ("build_ms", C.c_double), ("built", C.c_int),
                ("apply_launches", C.c_int), ("skeleton_rows", C.c_longlong)]


_LIB = None


def lib():
    """Load libhb.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} missing: run paper_2210_02698_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
        L.hb_create.argtypes = [C.POINTER(Grid), C.POINTER(Tables), d, C.POINTER(Options), C.POINTER(vp)]
        L.hb_build.argtypes = [vp]
        L.hb_set_omega.argtypes = [vp, d]
        L.hb_sweep_taylor.argtypes = [i, vp, vp]
        L.hb_curve_compress.argtypes = [vp, i]
        L.hb_curve_info.argtypes = [vp, i, C.POINTER(i), C.POINTER(i), C.POINTER(ll)]
        L.hb_sweep_tables.argtypes = [i, d, d, i, i, i, i, vp, i, vp, vp, i, vp, vp, i, d, vp, vp, vp, vp]
        for f in ("hb_apply", "hb_apply_adjoint", "hb_apply_dense", "hb_apply_dense_adjoint"):
            getattr(L, f).argtypes = [vp, vp, vp, i, vp]
        L.hb_set_precision.argtypes = [vp, i]
        L.hb_save.argtypes = [vp, C.c_char_p]
        L.hb_load.argtypes = [C.c_char_p, vp]
        L.hb_set_wait_selftest.argtypes = [vp, i]
        L.hb_device_alloc_cap.argtypes = [ll, C.POINTER(ll)]
        L.hb_entries.argtypes = [vp, vp, i, vp, i, vp, vp]
        L.hb_curve_set.argtypes = [vp, vp, vp, vp, ll]
        L.hb_curve_operators.argtypes = [vp, vp, vp, vp, vp]
        L.hb_apply_inclusion.argtypes = [vp, vp, vp, i, i, vp]
        L.hb_id_batch.argtypes = [i, vp, vp, vp, vp, d, vp, vp, vp]
        L.hb_id_batch_noalloc.argtypes = [i, vp, vp, vp, vp, d, vp, vp, vp, vp]
        L.hb_launch_shape.argtypes = [vp, i, i, C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(i),
                                      C.POINTER(i), C.POINTER(d), C.POINTER(i)]
        L.hb_fp64_fma_peak.argtypes = [C.POINTER(d), vp]
        L.hb_shard_rows.argtypes = [vp, i, i, C.POINTER(ll), C.POINTER(ll)]
        L.hb_apply_shard.argtypes = [vp, vp, vp, i, i, i, vp]
        L.hb_apply_shard_adjoint.argtypes = [vp, vp, vp, i, i, i, vp]
        L.hb_host_shard_rows.argtypes = [i, i, i, i, i, C.POINTER(ll), C.POINTER(ll)]
        L.hb_record_id_blocks.argtypes = [vp, i]
        L.hb_recorded_id_count.argtypes = [vp, C.POINTER(i)]
        L.hb_recorded_id_block.argtypes = [vp, i, C.POINTER(i), C.POINTER(i), C.POINTER(i), vp, vp, vp,
                                           C.POINTER(i), vp]
        L.hb_tree_perm.argtypes = [vp, vp]
        L.hb_proxy_rows.argtypes = [vp, ll, ll, vp, i, vp, vp]
        L.hb_info.argtypes = [vp, C.POINTER(Stats)]
        L.hb_rank_profile.argtypes = [vp, vp, vp]
        L.hb_host_cluster_tree.argtypes = [i, i, i, vp, vp, C.POINTER(i)]
        L.hb_host_proxy_rows.argtypes = [i, i, i, d, d, ll, ll, vp, i, vp, C.POINTER(ll)]
        L.hb_host_segment_tree.argtypes = [vp, ll, i, vp, vp, C.POINTER(i)]
        L.hb_host_point_proxy_rows.argtypes = [vp, ll, ll, ll, vp, i, d, d, vp, C.POINTER(ll)]
        L.hb_set_kernel_timing.argtypes = [vp, i]
        L.hb_kernel_times.argtypes = [vp, i, vp, vp, vp, vp]
        L.hb_last_error.argtypes = [vp]
        L.hb_last_error.restype = C.c_char_p
        L.hb_destroy.argtypes = [vp]
        L.hb_destroy.restype = None
        for f in EXPORTS:
            if f not in ("hb_last_error", "hb_destroy"):
                getattr(L, f).restype = C.c_int
        _LIB = L
    return _LIB


def sweep_taylor(s2):
    """hb_sweep_taylor: (ns, 15) series S_0..S_4 of n^2 about each source ->
    (ns, 46) Taylor numbers T_2..T_6, B_0..B_4, C_0..C_2."""
    s2 = np.ascontiguousarray(s2, dtype=np.float64)
    if s2.ndim != 2 or s2.shape[1] != 15:
        raise ValueError("s2 must be (ns, 15)")
    out = np.empty((s2.shape[0], 46))
    _check(lib().hb_sweep_taylor(s2.shape[0], s2.ctypes.data, out.ctypes.data))
    return out


def sweep_tables(M, lo, h, w0, w1, roi0, roi1, n_mesh, px, pz, src, taylor, max_iter=400, tol=1e-12):
    """hb_sweep_tables: the tables' columns src of tau^2, v0, v1 (each
    (NI, ns)) and the solves' info (ns, 6), computed on the device."""
    n_mesh = np.ascontiguousarray(n_mesh, dtype=np.float64)
    px = np.ascontiguousarray(px, dtype=np.float64)
    pz = np.ascontiguousarray(pz, dtype=np.float64)
    src = np.ascontiguousarray(src, dtype=np.int32)
    taylor = np.ascontiguousarray(taylor, dtype=np.float64)
    NI, ns = px.size, src.size
    if n_mesh.shape != (M, M) or pz.size != NI or taylor.shape != (ns, 46):
        raise ValueError("n_mesh (M, M), pz like px and taylor (ns, 46) required")
    t2, a0, a1 = (np.empty((NI, ns)) for _ in range(3))
    info = np.empty((ns, 6))
    _check(lib().hb_sweep_tables(int(M), float(lo), float(h), int(w0), int(w1), int(roi0), int(roi1),
                                 n_mesh.ctypes.data, NI, px.ctypes.data, pz.ctypes.data, ns, src.ctypes.data,
                                 taylor.ctypes.data, int(max_iter), float(tol), t2.ctypes.data, a0.ctypes.data,
                                 a1.ctypes.data, info.ctypes.data))
    return t2, a0, a1, info


def device_alloc_cap(cap_bytes=-1):
    """hb_device_alloc_cap: set the cap on the library's live device bytes
    (0: none, negative: unchanged) and return the bytes held now."""
    live = C.c_longlong(0)
    _check(lib().hb_device_alloc_cap(int(cap_bytes), C.byref(live)))
    return live.value


class HBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(st, handle=None):
    if st != HB_OK:
        raise HBError(st, lib().hb_last_error(handle).decode(errors="replace"))


def _device_buf(t, count, name, dtype="torch.complex128"):
    """Check a buffer the library reads or writes on the device: a CUDA,
    contiguous tensor of ``dtype`` with at least ``count`` elements.  Host
    arrays are refused; a raw integer address is passed through unchecked."""
    if isinstance(t, int):
        return t
    if not hasattr(t, "data_ptr") or not getattr(t, "is_cuda", False):
        raise HBError(HB_ERR_ARG, f"{name}: a CUDA tensor is required (got {type(t).__name__})")
    if str(t.dtype) != dtype:
        raise HBError(HB_ERR_ARG, f"{name}: {dtype[6:]} is required (got {t.dtype})")
    if not t.is_contiguous():
        raise HBError(HB_ERR_ARG, f"{name}: a contiguous tensor is required")
    if t.numel() < count:
        raise HBError(HB_ERR_ARG, f"{name}: {t.numel()} elements, {count} needed")
    return t.data_ptr()


def _stream_ptr(stream):
    if stream is None:
        return None
    return getattr(stream, "cuda_stream", stream)


class Operator:
    """Handle owning one discretised HB operator (hb_create .. hb_destroy)."""

    def __init__(self, N, nodes, tau2, v0, v1, n_cells, omega, eps=1e-6, leaf=64, chi=20.0,
                 nbr_radius_h=10.0, precision=HB_MIXED_BF16X3, workspace_mb=0, h=None,
                 x0=0.0, y0=0.0, barrier_cycles=0, autotune=0):
        L = lib()
        self._keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (nodes, tau2, v0, v1, n_cells)]
        nodes, tau2, v0, v1, n_cells = self._keep
        nx, ny = (N, N) if np.isscalar(N) else N
        self.nx, self.ny = nx, ny
        self.Nv = nx * ny
        self.h = (1.0 / nx) if h is None else h
        g = Grid(nx, ny, x0, y0, self.h)
        t = Tables(len(nodes), nodes.ctypes.data, nodes.ctypes.data, tau2.ctypes.data,
                   v0.ctypes.data, v1.ctypes.data, n_cells.ctypes.data)
        o = Options(eps, leaf, chi, nbr_radius_h, precision, workspace_mb, int(barrier_cycles), int(autotune))
        hnd = C.c_void_p()
        _check(L.hb_create(C.byref(g), C.byref(t), float(omega), C.byref(o), C.byref(hnd)))
        self.handle = hnd

    def close(self):
        if getattr(self, "handle", None):
            lib().hb_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _call(self, name, *args):
        _check(getattr(lib(), name)(self.handle, *args), self.handle)

    def save(self, path):
        """Write the built operator to a file (hb_save)."""
        self._call("hb_save", os.fsencode(str(path)))

    @classmethod
    def load(cls, path):
        """A built operator read from a file written by save (hb_load)."""
        L = lib()
        hnd = C.c_void_p()
        _check(L.hb_load(os.fsencode(str(path)), C.byref(hnd)))
        self = cls.__new__(cls)
        self.handle = hnd
        self._keep = []
        with open(path, "rb") as f:           # nx, ny and h from the file's header
            head = f.read(48)
        nx, ny = (int(v) for v in np.frombuffer(head, dtype="<i8", count=2, offset=8))
        self.nx, self.ny, self.Nv = nx, ny, nx * ny
        self.h = float(np.frombuffer(head, dtype="<f8", count=1, offset=40)[0])
        return self

    def build(self):
        self._call("hb_build")

    def set_omega(self, omega):
        """hb_set_omega: the same tables and cluster tree at another frequency;
        the handle is unbuilt afterwards (call build())."""
        self._call("hb_set_omega", float(omega))

    def set_precision(self, p):
        self._call("hb_set_precision", int(p))

    def set_wait_selftest(self, on):
        """Failure-detection self-test of the bounded device waits (see hb.h)."""
        self._call("hb_set_wait_selftest", 1 if on else 0)

    def _vecs(self, a, b, nrhs):
        n = max(int(nrhs), 0) * self.Nv
        return _device_buf(a, n, "input"), _device_buf(b, n, "output")

    def apply(self, s, u, nrhs, stream=None):
        self._call("hb_apply", *self._vecs(s, u, nrhs), int(nrhs), _stream_ptr(stream))

    def apply_adjoint(self, u, s, nrhs, stream=None):
        self._call("hb_apply_adjoint", *self._vecs(u, s, nrhs), int(nrhs), _stream_ptr(stream))

    def shard_rows(self, nranks, rank):
        """hb_shard_rows: the tree positions [lo, hi) of rank `rank` of `nranks`."""
        lo, hi = C.c_longlong(), C.c_longlong()
        self._call("hb_shard_rows", int(nranks), int(rank), C.byref(lo), C.byref(hi))
        return lo.value, hi.value

    def apply_shard(self, s, u, nrhs, nranks, rank, stream=None):
        """hb_apply_shard: this rank's rows of u from the whole input s."""
        self._call("hb_apply_shard", *self._vecs(s, u, nrhs), int(nrhs), int(nranks), int(rank),
                   _stream_ptr(stream))

    def apply_shard_adjoint(self, u, s, nrhs, nranks, rank, stream=None):
        """hb_apply_shard_adjoint: this rank's share of the adjoint on every cell."""
        self._call("hb_apply_shard_adjoint", *self._vecs(u, s, nrhs), int(nrhs), int(nranks), int(rank),
                   _stream_ptr(stream))

    def apply_dense(self, s, u, nrhs, stream=None):
        self._call("hb_apply_dense", *self._vecs(s, u, nrhs), int(nrhs), _stream_ptr(stream))

    def apply_dense_adjoint(self, u, s, nrhs, stream=None):
        self._call("hb_apply_dense_adjoint", *self._vecs(u, s, nrhs), int(nrhs), _stream_ptr(stream))

    def entries(self, rows, cols, out, stream=None):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        cols = np.ascontiguousarray(cols, dtype=np.int64)
        self._call("hb_entries", rows.ctypes.data, len(rows), cols.ctypes.data, len(cols),
                   _device_buf(out, len(rows) * len(cols), "out"), _stream_ptr(stream))

    def set_curve(self, centers, lengths, n_seg):
        """hb_curve_set: the inclusion's segments (centres (ns, 2), lengths,
        n at the centres; host arrays)."""
        c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, 2)
        w = np.ascontiguousarray(lengths, dtype=np.float64)
        n = np.ascontiguousarray(n_seg, dtype=np.float64)
        if not (len(c) == len(w) == len(n)):
            raise ValueError("centers, lengths and n_seg differ in length")
        self._call("hb_curve_set", c.ctypes.data, w.ctypes.data, n.ctypes.data, len(w))
        self.ns = len(w)

    def curve_operators(self, k_s2s=None, k_v2s=None, k_s2v=None, stream=None):
        """hb_curve_operators into device buffers (column-major; None skips)."""
        ns = getattr(self, "ns", 0)
        p = (lambda t, n, name: None if t is None else _device_buf(t, n, name))
        self._call("hb_curve_operators", p(k_s2s, ns * ns, "k_s2s"), p(k_v2s, ns * self.Nv, "k_v2s"),
                   p(k_s2v, ns * self.Nv, "k_s2v"), _stream_ptr(stream))

    def curve_compress(self, leaf_s=16):
        """hb_curve_compress: K^{v2s} and K^{s2v} of the curve as butterflies."""
        self._call("hb_curve_compress", int(leaf_s))

    def curve_info(self, which):
        """hb_curve_info: (levels, max_rank, entries) of the compressed K^{v2s}
        (which = 0) or K^{s2v} (1)."""
        lv, mr, en = C.c_int(), C.c_int(), C.c_longlong()
        self._call("hb_curve_info", int(which), C.byref(lv), C.byref(mr), C.byref(en))
        return lv.value, mr.value, en.value

    def apply_inclusion(self, s, u, nrhs, v2v_dense=False, stream=None):
        """hb_apply_inclusion: u = (K^{v2v} + K^{s2v} (K^{s2s})^{-1} K^{v2s}) h^2 s."""
        self._call("hb_apply_inclusion", *self._vecs(s, u, nrhs), int(nrhs), 1 if v2v_dense else 0,
                   _stream_ptr(stream))

    def tree_perm(self):
        out = np.empty(self.Nv, dtype=np.int64)
        self._call("hb_tree_perm", out.ctypes.data)
        return out

    def proxy_rows(self, t0, t1, seeds):
        seeds = np.ascontiguousarray(seeds, dtype=np.int64)
        out = np.empty(max(t1 - t0, 1), dtype=np.int64)
        cnt = C.c_longlong()
        self._call("hb_proxy_rows", int(t0), int(t1), seeds.ctypes.data, len(seeds), out.ctypes.data,
                   C.byref(cnt))
        return out[:cnt.value].copy()

    def launch_shape(self, adjoint=False, mtiles=1):
        """hb_launch_shape: the mixed apply's launch shape for one direction
        and m-tile count (mode -1 before the first apply at that count)."""
        mode, ib, st, pub, sl, cand = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_int()
        ms = C.c_double()
        self._call("hb_launch_shape", 1 if adjoint else 0, int(mtiles), C.byref(mode), C.byref(ib), C.byref(st),
                   C.byref(pub), C.byref(sl), C.byref(ms), C.byref(cand))
        return {"mode": mode.value, "item_bytes": ib.value, "stages": st.value, "pub_batch": pub.value,
                "slack": sl.value, "tuned_ms": ms.value, "candidates": cand.value}

    def record_id_blocks(self, per_level):
        """hb_record_id_blocks: before build(), keep up to per_level of the
        sampled blocks the ID decomposes at every butterfly level."""
        self._call("hb_record_id_blocks", int(per_level))

    def recorded_id_blocks(self):
        """The kept blocks (hb_recorded_id_block): a list of dicts with the
        level, proxy rows and columns (natural indices), the sampled block A
        (m x n complex128), the rank and the full pivot order."""
        cnt = C.c_int()
        self._call("hb_recorded_id_count", C.byref(cnt))
        out = []
        for q in range(cnt.value):
            lv, m, n, r = C.c_int(), C.c_int(), C.c_int(), C.c_int()
            self._call("hb_recorded_id_block", q, C.byref(lv), C.byref(m), C.byref(n), None, None, None,
                       C.byref(r), None)
            rows = np.empty(m.value, dtype=np.int64)
            cols = np.empty(n.value, dtype=np.int64)
            A = np.empty((n.value, m.value), dtype=np.complex128)   # column-major m x n
            piv = np.empty(n.value, dtype=np.int32)
            self._call("hb_recorded_id_block", q, C.byref(lv), C.byref(m), C.byref(n), rows.ctypes.data,
                       cols.ctypes.data, A.ctypes.data, C.byref(r), piv.ctypes.data)
            out.append({"level": lv.value, "rows": rows, "cols": cols, "A": A.T.copy(), "rank": r.value,
                        "pivots": piv})
        return out

    def info(self):
        s = Stats()
        self._call("hb_info", C.byref(s))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def rank_profile(self):
        """hb_rank_profile: (max, mean) ranks as (L_v+1, L_v+1) arrays indexed
        [HODBF level l][butterfly level k]."""
        n = int(self.info()["levels"]) + 1
        mx = np.zeros((n, n), dtype=np.int32)
        mean = np.zeros((n, n), dtype=np.float64)
        self._call("hb_rank_profile", mx.ctypes.data, mean.ctypes.data)
        return mx, mean

    def set_kernel_timing(self, on):
        self._call("hb_set_kernel_timing", 1 if on else 0)

    def kernel_times(self):
        cap = 32
        names = (C.c_char * 32 * cap)()
        ms = (C.c_double * cap)()
        cnt = (C.c_longlong * cap)()
        ng = C.c_int()
        self._call("hb_kernel_times", cap, C.cast(names, C.c_void_p), C.cast(ms, C.c_void_p),
                   C.cast(cnt, C.c_void_p), C.byref(ng))
        return {bytes(names[i]).split(b"\0")[0].decode(): (ms[i], cnt[i]) for i in range(min(ng.value, cap))}


def host_cluster_tree(nx, ny, leaf):
    """hb_host_cluster_tree: (perm, [bounds of levels 0..L_v]) without a device."""
    lv = C.c_int()
    _check(lib().hb_host_cluster_tree(int(nx), int(ny), int(leaf), None, None, C.byref(lv)))
    perm = np.empty(int(nx) * int(ny), dtype=np.int64)
    bounds = np.empty(sum((1 << l) + 1 for l in range(lv.value + 1)), dtype=np.int64)
    _check(lib().hb_host_cluster_tree(int(nx), int(ny), int(leaf), perm.ctypes.data, bounds.ctypes.data,
                                      C.byref(lv)))
    out, o = [], 0
    for l in range(lv.value + 1):
        out.append(bounds[o:o + (1 << l) + 1].copy())
        o += (1 << l) + 1
    return perm, out


def host_segment_tree(centers, leaf):
    """hb_host_segment_tree: (perm, [bounds of levels 0..L_s]) of the segment K-D tree."""
    c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, 2)
    lv = C.c_int()
    _check(lib().hb_host_segment_tree(c.ctypes.data, len(c), int(leaf), None, None, C.byref(lv)))
    perm = np.empty(len(c), dtype=np.int64)
    bounds = np.empty(sum((1 << l) + 1 for l in range(lv.value + 1)), dtype=np.int64)
    _check(lib().hb_host_segment_tree(c.ctypes.data, len(c), int(leaf), perm.ctypes.data, bounds.ctypes.data,
                                      C.byref(lv)))
    out, o = [], 0
    for l in range(lv.value + 1):
        out.append(bounds[o:o + (1 << l) + 1].copy())
        o += (1 << l) + 1
    return perm, out


def host_point_proxy_rows(rows_xz, t0, t1, seeds_xz, chi, radius):
    """hb_host_point_proxy_rows: proxy positions of rows [t0, t1) for seed points."""
    r = np.ascontiguousarray(rows_xz, dtype=np.float64).reshape(-1, 2)
    sd = np.ascontiguousarray(seeds_xz, dtype=np.float64).reshape(-1, 2)
    out = np.empty(max(int(t1) - int(t0), 1), dtype=np.int64)
    cnt = C.c_longlong()
    _check(lib().hb_host_point_proxy_rows(r.ctypes.data, len(r), int(t0), int(t1), sd.ctypes.data, len(sd),
                                          float(chi), float(radius), out.ctypes.data, C.byref(cnt)))
    return out[:cnt.value].copy()


def host_proxy_rows(nx, ny, leaf, chi, radius, t0, t1, seeds):
    """hb_host_proxy_rows: proxy tree positions of the row node [t0, t1)."""
    seeds = np.ascontiguousarray(seeds, dtype=np.int64)
    out = np.empty(max(int(t1) - int(t0), 1), dtype=np.int64)
    cnt = C.c_longlong()
    _check(lib().hb_host_proxy_rows(int(nx), int(ny), int(leaf), float(chi), float(radius), int(t0), int(t1),
                                    seeds.ctypes.data, len(seeds), out.ctypes.data, C.byref(cnt)))
    return out[:cnt.value].copy()


def _id_args(A, m, n, a_off, rank, skel, V):
    """Host size arrays and checked device buffers of hb_id_batch(_noalloc):
    A (complex128) must hold every matrix, rank (int32) one entry per matrix,
    skel (int32) sum(n), V (complex128) sum(n^2)."""
    m = np.ascontiguousarray(m, dtype=np.int32)
    n = np.ascontiguousarray(n, dtype=np.int32)
    a_off = np.ascontiguousarray(a_off, dtype=np.int64)
    if not (len(m) == len(n) == len(a_off)):
        raise HBError(HB_ERR_ARG, "m, n and a_off differ in length")
    cnt = len(m)
    a_need = int(np.max(a_off + m.astype(np.int64) * n)) if cnt else 0
    n64 = n.astype(np.int64)
    ptrs = (_device_buf(A, a_need, "A"), _device_buf(rank, cnt, "rank", "torch.int32"),
            _device_buf(skel, int(n64.sum()), "skel", "torch.int32"),
            _device_buf(V, int((n64 * n64).sum()), "V"))
    return m, n, a_off, ptrs


def id_batch(A, m, n, a_off, eps, rank, skel, V):
    """hb_id_batch on device buffers (torch tensors) with host size arrays."""
    m, n, a_off, (pA, pr, ps, pV) = _id_args(A, m, n, a_off, rank, skel, V)
    _check(lib().hb_id_batch(len(m), m.ctypes.data, n.ctypes.data, a_off.ctypes.data, pA,
                             float(eps), pr, ps, pV))


def id_batch_noalloc(A, m, n, a_off, eps, rank, skel, V, stream=None):
    """hb_id_batch_noalloc: hb_id_batch without any device allocation."""
    m, n, a_off, (pA, pr, ps, pV) = _id_args(A, m, n, a_off, rank, skel, V)
    _check(lib().hb_id_batch_noalloc(len(m), m.ctypes.data, n.ctypes.data, a_off.ctypes.data, pA,
                                     float(eps), pr, ps, pV, _stream_ptr(stream)))


def fp64_fma_peak(stream=None):
    """hb_fp64_fma_peak: measured FP64 TFLOP/s of the current device."""
    v = C.c_double()
    _check(lib().hb_fp64_fma_peak(C.byref(v), _stream_ptr(stream)))
    return v.value


def host_shard_rows(nx, ny, leaf, nranks, rank):
    """hb_host_shard_rows: a rank's tree positions [lo, hi) without a device."""
    lo, hi = C.c_longlong(), C.c_longlong()
    _check(lib().hb_host_shard_rows(int(nx), int(ny), int(leaf), int(nranks), int(rank), C.byref(lo),
                                    C.byref(hi)))
    return lo.value, hi.value


def load_tables(path):
    z = np.load(path)
    return z["nodes"], z["tau2"], z["v0"], z["v1"]


def operator_for(workload, tables_path, precision=HB_MIXED_BF16X3, **kw):
    """Operator of a workloads.Workload with tables from a stored .npz file."""
    nodes, t2, v0, v1 = load_tables(tables_path)
    return Operator(workload.N, nodes, t2, v0, v1, workload.n_cells(), workload.omega,
                    eps=kw.pop("eps", workload.eps), leaf=kw.pop("leaf", workload.leaf),
                    chi=kw.pop("chi", workload.chi), precision=precision, **kw)
