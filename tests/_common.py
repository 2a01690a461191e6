"""Shared helpers for the tests: stored tables, oracle and GPU operators."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLES = os.path.join(ROOT, "tests", "golden", "tables")


def table_path(medium, n_I=16):
    return os.path.join(TABLES, f"{medium.key}_nI{n_I}.npz")


def load_tables(medium, n_I=16):
    z = np.load(table_path(medium, n_I))
    return {"nodes": z["nodes"], "tau2": z["tau2"], "v0": z["v0"], "v1": z["v1"], "n_I": n_I}


def oracle_op(w, tables=None):
    from oracle import kernel
    tab = tables if tables is not None else load_tables(w.medium)
    return kernel.Operator(w.N, tab, w.omega, w.n_cells())


def gpu_op(w, tables=None, **kw):
    from paper_2210_02698_gb300 import binding
    tab = tables if tables is not None else load_tables(w.medium)
    return binding.Operator(w.N, tab["nodes"], tab["tau2"], tab["v0"], tab["v1"], w.n_cells(),
                            w.omega, eps=kw.pop("eps", w.eps), leaf=kw.pop("leaf", w.leaf),
                            chi=kw.pop("chi", w.chi), **kw)


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "hb.h")).read()
    return sorted(set(re.findall(r"\b(hb_[a-z0-9_]+)\s*\(", txt)))


def to_dev(a):
    """(Nv, nrhs) complex numpy -> CUDA complex128 tensor (nrhs, Nv) = column-major."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).to("cuda")


def from_dev(t):
    return t.cpu().numpy().T.copy()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _dense_part(args):
    """One worker's share of oracle_dense_rows: the columns [c0, c1) of the
    dense sum (or the rows [c0, c1) of the adjoint's), in chunks."""
    import numpy as _np
    w, path, idx, adjoint, c0, c1, chunk = args
    s = _np.load(path, mmap_mode="r")
    og = oracle_op(w)
    out = _np.zeros((len(idx), s.shape[1]), dtype=_np.complex128)
    for a in range(c0, c1, chunk):
        b = _np.arange(a, min(c1, a + chunk))
        if adjoint:
            out += og.block(b, idx).conj().T @ _np.asarray(s[b])
        else:
            out += og.block(idx, b) @ (_np.asarray(s[b]) * og.h ** 2)
    return out * (og.h ** 2 if adjoint else 1.0)


def oracle_dense_rows(w, s, idx, adjoint=False, procs=None, chunk=16384):
    """The oracle's dense sum (oracle.dense.apply) on the rows idx - or its
    adjoint (oracle.dense.adjoint) on the columns idx - for a large grid,
    with the sum over all N_v cells split into `procs` contiguous ranges
    evaluated by worker processes (spawned, so that no CUDA state is
    inherited) and added in range order.  The arithmetic per entry is the
    oracle's own (Operator.block); only the summation is grouped by range."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import tempfile
    procs = procs or max(1, min(16, os.cpu_count() or 1))
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "s.npy")
        np.save(path, np.ascontiguousarray(s))
        Nv = s.shape[0]
        bounds = [Nv * k // procs for k in range(procs + 1)]
        jobs = [(w, path, np.asarray(idx), adjoint, bounds[k], bounds[k + 1], chunk) for k in range(procs)]
        # one BLAS / OpenMP thread per worker (the workers already fill the cores)
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        os.environ.update({k: "1" for k in saved})
        try:
            with cf.ProcessPoolExecutor(procs, mp_context=mp.get_context("spawn")) as ex:
                parts = list(ex.map(_dense_part, jobs))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    return sum(parts[1:], parts[0])
