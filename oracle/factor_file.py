"""Test infrastructure (oracle): the CPU butterfly apply over a factor file.

Reads the file that ``hb_save`` writes - its format is documented with
``hb_save`` in include/hb.h; the file is data, no code is shared - and
applies the compressed operator with plain numpy products, block by block:

    u = K~ (h^2 s),   K~ = D + sum over the HODBF blocks of
                      P_o K^L W^L ... W^1 V^0 P_s^T       (Sec. 4.2, Sec. 4.2.1,
                                                         Eq. butterfly_mat)

with D the dense diagonal leaf blocks, and the exact adjoint
s = h^2 K~^H u (reversed order, conjugate-transposed blocks).  Level-0
blocks act on the points of leaf j of the column node, a level-k transfer
block (i, j) on the stacked skeleton vectors of the level k-1 blocks
((i/2) 2^(L-k+1) + 2j, + 1), and the K^L block i writes leaf i of the row
node.  FP64 throughout; only tests/ and bench.py use it.
"""
from __future__ import annotations

import numpy as np

MAGIC = b"HBFACT01"


class FactorFile:
    """The operator stored in a factor file (see module docstring)."""

    def __init__(self, path):
        with open(path, "rb") as f:
            buf = f.read()
        self._buf = buf
        self._pos = 0
        if self._raw(8) != MAGIC:
            raise ValueError("not an HB factor file")
        self.nx, self.ny = self._ints(2)
        self.x0, self.y0, self.h, self.omega = self._reals(4)
        self.eps, self.chi, self.nbr_radius_h = self._reals(3)
        self.leaf, self.precision, self.workspace_mb, self.barrier_cycles = self._ints(4)
        self.n_I = int(self._ints(1)[0])
        NI = self.n_I * self.n_I
        self.nodes_x = self._reals(self.n_I)
        self.nodes_y = self._reals(self.n_I)
        self.tau2 = self._reals(NI * NI).reshape(NI, NI)
        self.v0 = self._reals(NI * NI).reshape(NI, NI)
        self.v1 = self._reals(NI * NI).reshape(NI, NI)
        self.Nv = int(self.nx) * int(self.ny)
        self.n_cells = self._reals(self.Nv)
        self.Lv = int(self._ints(1)[0])
        self.perm = self._ints(self.Nv)                  # tree position -> natural index
        self.bounds = [self._ints((1 << l) + 1) for l in range(self.Lv + 1)]
        nfac = int(self._ints(1)[0])
        self.arena = self._reals(2 * nfac).view(np.complex128)
        self.leaf_off = self._ints(1 << self.Lv)
        self.butterflies = []
        for _ in range(int(self._ints(1)[0])):
            l, oi, si, L = (int(v) for v in self._ints(4))
            rank, f_off = [], []
            for _k in range(L + 1):
                rf = self._ints(2 * (1 << L)).reshape(-1, 2)
                rank.append(rf[:, 0].copy())
                f_off.append(rf[:, 1].copy())
            kl_off = self._ints(1 << L)
            self.butterflies.append({"l": l, "oi": oi, "si": si, "L": L, "rank": rank, "f_off": f_off,
                                     "kl_off": kl_off})
        if self._pos != len(buf):
            raise ValueError("trailing bytes in the factor file")
        del self._buf

    # ------------------------------------------------------------ reading
    def _raw(self, n):
        b = self._buf[self._pos:self._pos + n]
        if len(b) != n:
            raise ValueError("truncated factor file")
        self._pos += n
        return b

    def _ints(self, n):
        return np.frombuffer(self._raw(8 * n), dtype="<i8").astype(np.int64)

    def _reals(self, n):
        return np.frombuffer(self._raw(8 * n), dtype="<f8").copy()

    # ------------------------------------------------------------- blocks
    def node(self, level, idx):
        """Tree positions [lo, hi) of node idx at a tree level."""
        b = self.bounds[level]
        return int(b[idx]), int(b[idx + 1])

    def block(self, off, rows, cols):
        """The column-major rows x cols block at an arena offset."""
        return self.arena[off:off + rows * cols].reshape(cols, rows).T

    def _leaf_rows(self, t):
        lo, hi = self.node(self.Lv, t)
        return lo, hi

    # -------------------------------------------------------------- apply
    def apply(self, s):
        """u = K~ (h^2 s); s, u: (N_v, nrhs) complex128 in natural order."""
        s = np.asarray(s, dtype=np.complex128).reshape(self.Nv, -1)
        x = self.h * self.h * s[self.perm]               # tree order
        y = np.zeros_like(x)
        for t in range(1 << self.Lv):
            lo, hi = self._leaf_rows(t)
            y[lo:hi] += self.block(int(self.leaf_off[t]), hi - lo, hi - lo) @ x[lo:hi]
        for b in self.butterflies:
            L, rank, f_off = b["L"], b["rank"], b["f_off"]
            z = []
            for j in range(1 << L):                       # V^0
                lo, hi = self._leaf_rows((b["si"] << L) + j)
                z.append(self.block(int(f_off[0][j]), int(rank[0][j]), hi - lo) @ x[lo:hi])
            for k in range(1, L + 1):                     # W^k
                w = 1 << (L - k)
                nz = [None] * (1 << L)
                for i in range(1 << k):
                    for j in range(w):
                        q1 = (i // 2) * (2 * w) + 2 * j
                        inp = np.vstack([z[q1], z[q1 + 1]])
                        q = i * w + j
                        nz[q] = self.block(int(f_off[k][q]), int(rank[k][q]), inp.shape[0]) @ inp
                z = nz
            for i in range(1 << L):                       # K^L
                lo, hi = self._leaf_rows((b["oi"] << L) + i)
                y[lo:hi] += self.block(int(b["kl_off"][i]), hi - lo, int(rank[L][i])) @ z[i]
        u = np.empty_like(y)
        u[self.perm] = y
        return u

    def apply_adjoint(self, u):
        """s = h^2 K~^H u; u, s: (N_v, nrhs) complex128 in natural order."""
        u = np.asarray(u, dtype=np.complex128).reshape(self.Nv, -1)
        y = u[self.perm]
        x = np.zeros_like(y)
        for t in range(1 << self.Lv):
            lo, hi = self._leaf_rows(t)
            x[lo:hi] += self.block(int(self.leaf_off[t]), hi - lo, hi - lo).conj().T @ y[lo:hi]
        for b in self.butterflies:
            L, rank, f_off = b["L"], b["rank"], b["f_off"]
            z = []
            for i in range(1 << L):                       # K^L^H
                lo, hi = self._leaf_rows((b["oi"] << L) + i)
                z.append(self.block(int(b["kl_off"][i]), hi - lo, int(rank[L][i])).conj().T @ y[lo:hi])
            for k in range(L, 0, -1):                     # W^k^H, back to level k - 1
                w = 1 << (L - k)
                nz = [None] * (1 << L)
                for i in range(1 << k):
                    for j in range(w):
                        q1 = (i // 2) * (2 * w) + 2 * j
                        r1, r2 = int(rank[k - 1][q1]), int(rank[k - 1][q1 + 1])
                        q = i * w + j
                        v = self.block(int(f_off[k][q]), int(rank[k][q]), r1 + r2).conj().T @ z[q]
                        for qq, part in ((q1, v[:r1]), (q1 + 1, v[r1:])):
                            nz[qq] = part if nz[qq] is None else nz[qq] + part
                z = nz
            for j in range(1 << L):                       # V^0^H
                lo, hi = self._leaf_rows((b["si"] << L) + j)
                x[lo:hi] += self.block(int(f_off[0][j]), int(rank[0][j]), hi - lo).conj().T @ z[j]
        s = np.empty_like(x)
        s[self.perm] = self.h * self.h * x
        return s
