"""Table builder by Lax-Friedrichs WENO sweeping (Sec. 2.3) for media with
no closed-form ingredients (the Gaussian lens).

Test infrastructure (see ``oracle/__init__``).  The numerics live in
``oracle/sweep.c`` (plain C, compiled here with gcc on first use):
factored eikonal (Eq. faceik) and the transport equations Eq. equVs for
v0 (s = -1) and v1 (s = 0), each initialised in a box around the source by
the Taylor expansions Eq. expansionT / expansionV0 / expansionV1 of
``oracle.taylor``, then local cubic interpolation to the Chebyshev nodes
(Sec. 4.1).  This module supplies the Taylor input: the series
n^2 = sum_k S_k of each medium about the source (exact polynomial
arithmetic), passed through the recursions Eq. recursiveT, Eq. recursiveB,
Eq. C0, Eq. C1, Eq. recursiveC.

Pins (tests/test_oracle_sweep.py): on the constant-gradient medium, whose
ingredients are exact in ``oracle.tables``, the mesh errors of tau, v0, v1
fall at the orders the paper states (fifth, third and first order in h0);
on the homogeneous medium the sweeps keep the exact solution; the lens
tables are reciprocal (tau^2, v0, v1 symmetric in observation and source
node) to the discretisation error and v0 stays positive (no caustics).
"""
import ctypes
import hashlib
import math
import os
import subprocess

import numpy as np

from . import chebyshev, taylor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sweep.c")
BUILD = os.path.join(HERE, "_build")
B0_2D = 1.0 / (2.0 * math.sqrt(math.pi))
TAYLOR_LEN = 46
_lib = None


# -ffp-contract=off: every a*b + c rounds twice, as written, on every
# architecture (GCC contracts it into one fused multiply-add by default where
# the hardware has one), so the oracle's results are the same on x86 and Arm
CFLAGS = ["-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared"]


def compile_library():
    """gcc CFLAGS [-fopenmp] oracle/sweep.c; cached by source and flags."""
    with open(SRC, "rb") as f:
        tag = hashlib.sha256(f.read() + " ".join(CFLAGS).encode()).hexdigest()[:12]
    out = os.path.join(BUILD, f"libhbsweep_{tag}.so")
    if os.path.exists(out):
        return out
    os.makedirs(BUILD, exist_ok=True)
    tmp = out + f".{os.getpid()}.tmp"
    base = ["gcc", *CFLAGS, SRC, "-o", tmp, "-lm"]
    r = subprocess.run(base[:len(CFLAGS) + 1] + ["-fopenmp"] + base[len(CFLAGS) + 1:], capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, out)
    return out


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(compile_library())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        ci, cd = ctypes.c_int, ctypes.c_double
        L.hb_oracle_sweep_tables.argtypes = [ci, cd, cd, ci, ci, ci, ci, dp, ci, dp, dp, ci, ip, dp, ci, cd, dp, dp,
                                             dp, dp]
        L.hb_oracle_sweep_tables.restype = ctypes.c_int
        L.hb_oracle_sweep_fields.argtypes = [ci, cd, cd, ci, ci, ci, ci, dp, cd, cd, dp, ci, cd, dp, dp, dp, dp]
        L.hb_oracle_sweep_fields.restype = ctypes.c_int
        L.hb_oracle_sweep_set_order.argtypes = [ci]
        L.hb_oracle_sweep_set_order.restype = None
        L.hb_oracle_sweep_visit_order.argtypes = [ci, ci, ctypes.POINTER(ctypes.c_longlong)]
        L.hb_oracle_sweep_visit_order.restype = None
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------ series of n^2 about r0 ----
def _pmul(A, B, P):
    """Product of two polynomials given as homogeneous pieces [H_0..H_P]."""
    out = [np.zeros(d + 1) for d in range(P + 1)]
    for a in range(P + 1):
        for b in range(P + 1 - a):
            out[a + b] = out[a + b] + taylor.mul(A[a], B[b])
    return out


def n2_series(medium, x0, z0, P):
    """S_0..S_P with n(r0 + (X, Z))^2 = sum_k S_k(X, Z) + O(|(X, Z)|^(P+1))."""
    if medium.kind == "homogeneous":
        S = [np.zeros(k + 1) for k in range(P + 1)]
        S[0][0] = medium.n0 ** 2
        return S
    if medium.kind == "gradient":
        return taylor.n2_series_gradient(medium.c0 + medium.g * z0, medium.g, P)
    if medium.kind == "lens":
        # n = 1 + a E0 exp(q), q = -(2 dx X + 2 dz Z + X^2 + Z^2) / w^2
        a, w = medium.amp, medium.w
        dx, dz = x0 - medium.center[0], z0 - medium.center[1]
        E0 = math.exp(-(dx * dx + dz * dz) / (w * w))
        q = [np.zeros(k + 1) for k in range(P + 1)]
        q[1] = np.array([-2 * dx, -2 * dz]) / (w * w)
        if P >= 2:
            q[2] = np.array([-1.0, 0.0, -1.0]) / (w * w)
        E = [np.zeros(k + 1) for k in range(P + 1)]
        E[0][0] = 1.0
        term = [x.copy() for x in E]
        for m in range(1, P + 1):
            term = [t / m for t in _pmul(term, q, P)]
            E = [e + t for e, t in zip(E, term)]
        E = [E0 * e for e in E]
        nser = [a * e for e in E]
        nser[0] = nser[0] + 1.0
        return _pmul(nser, nser, P)
    raise NotImplementedError(medium.kind)


def taylor_input(medium, x0, z0, P_T=6):
    """The 46 Taylor numbers of one source: T_2..T_6, B_0..B_4, C_0..C_2."""
    S = n2_series(medium, x0, z0, P_T - 2)
    T, B, C = taylor.recursions(S, P_T)
    parts = [T[k] for k in range(2, P_T + 1)] + [B[k] for k in range(0, P_T - 1)] + [C[k] for k in range(0, 3)]
    out = np.concatenate([np.asarray(p, dtype=np.float64).reshape(-1) for p in parts])
    assert out.size == TAYLOR_LEN
    return out


# ------------------------------------------------------------------ mesh ----
def mesh(h0, margin):
    """Mesh x_i = lo + i h0 covering [-m, 1 + m], m = max(margin, 38 h0)
    (M points a side); the window [w0, w1] of the transports (the unit
    square plus 14 points a side) and, in window indices, the region of
    interest [roi0, roi1] (the unit square plus the two points a side the
    cubic interpolation may use)."""
    k = max(int(math.ceil(margin / h0)), 38)
    n1 = int(round(1.0 / h0))
    M = n1 + 1 + 2 * k
    w0, w1 = k - 14, k + n1 + 14
    return M, -k * h0, w0, w1, 12, 12 + n1 + 4


def mesh_n(medium, M, lo, h0):
    c = lo + h0 * np.arange(M)
    X, Z = np.meshgrid(c, c)         # [j][i] = (x_i, z_j)
    return np.ascontiguousarray(medium.n(X, Z), dtype=np.float64), X, Z


class _Order:
    """Sweep order of the calls inside the block: rows (default) or
    anti-diagonals (``wavefront``), restored to rows on exit."""

    def __init__(self, wavefront):
        self.wavefront = wavefront

    def __enter__(self):
        lib().hb_oracle_sweep_set_order(1 if self.wavefront else 0)

    def __exit__(self, *exc):
        lib().hb_oracle_sweep_set_order(0)


def visit_order(o, M, wavefront=False):
    """The points (j M + i) in the order sweep o visits them."""
    out = np.empty(M * M, dtype=np.int64)
    with _Order(wavefront):
        lib().hb_oracle_sweep_visit_order(o, M, out.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)))
    return out


def fields(medium, x0, z0, h0, margin=0.3, max_iter=500, tol=1e-12, wavefront=False):
    """Mesh fields of one source: tau^2, v0, v1 (each [j][i] on the mesh;
    v0 and v1 are NaN outside the transport window), the mesh coordinates
    and (iterations, last update) of the three solves.  ``wavefront``: sweep
    anti-diagonal by anti-diagonal instead of row by row (same fixed point)."""
    M, lo, w0, w1, roi0, roi1 = mesh(h0, margin)
    n, X, Z = mesh_n(medium, M, lo, h0)
    tin = taylor_input(medium, x0, z0)
    Mw = w1 - w0 + 1
    t2 = np.empty((M, M))
    a0 = np.empty((Mw, Mw))
    a1 = np.empty((Mw, Mw))
    info = np.empty(6)
    with _Order(wavefront):
        r = lib().hb_oracle_sweep_fields(M, lo, h0, w0, w1, roi0, roi1, _p(n), x0, z0, _p(tin), max_iter, tol,
                                         _p(t2), _p(a0), _p(a1), _p(info))
    if r != 0:
        raise RuntimeError("sweep failed")
    v0 = np.full((M, M), np.nan)
    v1 = np.full((M, M), np.nan)
    v0[w0:w1 + 1, w0:w1 + 1] = a0
    v1[w0:w1 + 1, w0:w1 + 1] = a1
    return t2, v0, v1, X, Z, info


def build_tables(medium, n_I, h0=1.0 / 256, margin=0.3, max_iter=400, tol=1e-12, sources=None):
    """F^c tables (Sec. 4.1) by sweeping: dict with 'nodes', 'tau2', 'v0',
    'v1' (N_I x N_I, row = observation node, column = source node) and
    'info' (per source: iterations and last updates of the three solves).
    With ``sources`` only those columns are computed (N_I x len(sources))."""
    xn = chebyshev.nodes(n_I)
    NI = n_I * n_I
    px = np.ascontiguousarray(np.tile(xn, n_I))
    pz = np.ascontiguousarray(np.repeat(xn, n_I))
    # contiguous: the C builder reads the indices as one array
    src = np.arange(NI, dtype=np.int32) if sources is None else np.ascontiguousarray(sources, dtype=np.int32)
    ns = len(src)
    M, lo, w0, w1, roi0, roi1 = mesh(h0, margin)
    n, _, _ = mesh_n(medium, M, lo, h0)
    tin = np.ascontiguousarray(np.stack([taylor_input(medium, px[j], pz[j]) for j in src]))
    t2 = np.empty((NI, ns))
    a0 = np.empty((NI, ns))
    a1 = np.empty((NI, ns))
    info = np.empty((ns, 6))
    r = lib().hb_oracle_sweep_tables(M, lo, h0, w0, w1, roi0, roi1, _p(n), NI, _p(px), _p(pz), ns,
                                     src.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _p(tin), max_iter, tol,
                                     _p(t2), _p(a0), _p(a1), _p(info))
    if r != 0:
        raise RuntimeError("sweep failed")
    # diagonal: tau^2 = 0, v0 = B0, v1 = C0 (the value of v1 at the source)
    for k, j in enumerate(src):
        t2[j, k] = 0.0
        a0[j, k] = B0_2D
        a1[j, k] = tin[k, 40]
    return {"nodes": xn, "tau2": t2, "v0": a0, "v1": a1, "n_I": n_I, "info": info}
