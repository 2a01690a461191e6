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
    return sorted(set(re.findall(r"\b(hb_[a-z_]+)\s*\(", txt)))


def to_dev(a):
    """(Nv, nrhs) complex numpy -> CUDA complex128 tensor (nrhs, Nv) = column-major."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).T)).to("cuda")


def from_dev(t):
    return t.cpu().numpy().T.copy()


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
