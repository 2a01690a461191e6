"""The inclusion operators in compressed form (Sec. 4.2: the K^{s2v},
K^{v2s} and K^{s2s} items; Sec. 4.2.3, Sec. 4.2.4): a prototype of the
compressed path, checked against the dense operators of ``inclusion``.

Test infrastructure (see ``oracle/__init__``).  Slow; for small grids.

Trees.  Cells: the cluster tree T_{H_v} of ``tree.cluster_tree``.  Segments:
a K-D tree T_{H_s} over the segment centres built by the same rule on real
coordinates (split the longer side of the bounding box, order by
(coordinate, index), first child ceil(n/2)).

Butterflies (Sec. 4.2.1, as ``butterfly`` builds them for K^{v2v}): the
butterfly of K(o, s), o the node oi and s the node si at level l0 of the row
and column trees, with L levels: at level 0 the ID of K(tau_hat, nu) for
every node nu of the column tree at level l0 + L below s, with tau = o; at
level k = 1..L the ID of [K(tau_hat, nu1_bar) K(tau_hat, nu2_bar)] for tau at
level l0 + k below o and nu at level l0 + L - k below s; K^L = K(tau_i,
nu_bar) at level l0 + L below o.  Proxy rows tau_hat (Eq. proxyv2v): the
rows of tau whose points lie within ``radius`` h of a seed column's point,
plus m = min(|tau|, ceil(chi |seeds|)) rows of tau at a uniform stride in
tree order; all of tau at k = L.

Operators:
  * K^{s2v} and K^{v2s}: one butterfly each with o, s the roots and
    L = min(L_v, L_s) levels, the trees cut at level L;
  * K^{s2s}: an HODBF over T_{H_s} (siblings at level l: a butterfly with
    L_s - l levels; dense leaf blocks, holding the self terms);
  * the total field U = K^{v2v} I + K^{s2v} P with K^{s2s} P = K^{v2s} I
    (Eq. m_v2v_inclu), the surface system solved by GMRES with the HODBF
    matvec (the paper inverts the HODBF by cited work; an iterative solve
    reaches the same P to its tolerance).
Reading: the paper states these items and their complexities, not their
proxy rules; the volume rule with the other set's points as seeds is used.
"""
import math

import numpy as np
from scipy.sparse import linalg as spla

from . import cpqr, inclusion, tree


def segment_tree(centres, leaf):
    """(perm, bounds) of the K-D tree over the segment centres: perm[p] is
    the segment at tree position p, bounds[l] the 2^l + 1 node boundaries."""
    c = np.asarray(centres, dtype=np.float64)
    ns = len(c)
    L = tree.num_levels(ns, leaf)
    nodes, bounds = [np.arange(ns)], [np.array([0, ns])]
    for _ in range(L):
        nxt = []
        for P in nodes:
            if len(P) == 0:
                nxt += [P, P]
                continue
            w = c[P].max(axis=0) - c[P].min(axis=0)
            coord = c[P, 0] if w[0] >= w[1] else c[P, 1]
            P = P[np.lexsort((P, coord))]
            n1 = (len(P) + 1) // 2
            nxt += [P[:n1], P[n1:]]
        nodes = nxt
        bounds.append(np.concatenate([[0], np.cumsum([len(P) for P in nodes])]))
    return np.concatenate([np.sort(P) for P in nodes]), bounds


class Side:
    """One index set in tree order: points (tree order), tree bounds."""

    def __init__(self, points, perm, bounds):
        self.perm, self.bounds = perm, bounds
        self.pts = np.asarray(points)[perm]

    def node(self, level, i):
        b = self.bounds[level]
        return int(b[i]), int(b[i + 1])


class Butterfly:
    """K(o, s) between node oi of ``rows`` and node si of ``cols`` at level
    l0, L levels; K(rpos, cpos) evaluates a block by tree positions."""

    def __init__(self, K, rows, cols, l0, oi, si, L, eps, chi, radius):
        self.K, self.rows, self.cols = K, rows, cols
        self.l0, self.oi, self.si, self.L = l0, oi, si, L
        self.eps, self.chi, self.radius = eps, chi, radius
        self._build()

    def _proxy(self, t0, t1, seeds):
        size = t1 - t0
        m = min(size, int(math.ceil(self.chi * len(seeds))))
        if m >= size:
            return np.arange(t0, t1)
        uni = t0 + (np.arange(m) * size) // m
        pos = np.arange(t0, t1)
        d2 = ((self.rows.pts[pos][:, None, :] - self.cols.pts[np.asarray(seeds)][None, :, :]) ** 2).sum(axis=-1)
        return np.union1d(uni, pos[(d2 <= self.radius ** 2).any(axis=1)])

    def _build(self):
        l0, L, oi, si = self.l0, self.L, self.oi, self.si
        self.V0, self.W, self.KL, skel = {}, {}, {}, {}
        t0, t1 = self.rows.node(l0, oi)
        for j in range(1 << L):
            cols = np.arange(*self.cols.node(l0 + L, (si << L) + j))
            rows = np.arange(t0, t1) if L == 0 else self._proxy(t0, t1, cols)
            sk, V, _ = cpqr.cpqr_id(self.K(rows, cols), self.eps)
            self.V0[j], skel[(0, 0, j)] = V, cols[sk]
        for k in range(1, L + 1):
            for i in range(1 << k):
                a0, a1 = self.rows.node(l0 + k, (oi << k) + i)
                for j in range(1 << (L - k)):
                    cols = np.concatenate([skel[(k - 1, i // 2, 2 * j)], skel[(k - 1, i // 2, 2 * j + 1)]])
                    rows = np.arange(a0, a1) if k == L else self._proxy(a0, a1, cols)
                    sk, Wm, _ = cpqr.cpqr_id(self.K(rows, cols), self.eps)
                    self.W[(k, i, j)], skel[(k, i, j)] = Wm, cols[sk]
        for i in range(1 << L):
            a0, a1 = self.rows.node(l0 + L, (oi << L) + i)
            self.KL[i] = self.K(np.arange(a0, a1), skel[(L, i, 0)])
        self.skel = skel

    def apply(self, x, y):
        """y[rows of o] += K(o, s) x[cols of s]; x, y in tree order."""
        l0, L, oi, si = self.l0, self.L, self.oi, self.si
        xh = {}
        for j in range(1 << L):
            n0, n1 = self.cols.node(l0 + L, (si << L) + j)
            xh[(0, 0, j)] = self.V0[j] @ x[n0:n1]
        for k in range(1, L + 1):
            for i in range(1 << k):
                for j in range(1 << (L - k)):
                    xin = np.concatenate([xh[(k - 1, i // 2, 2 * j)], xh[(k - 1, i // 2, 2 * j + 1)]])
                    xh[(k, i, j)] = self.W[(k, i, j)] @ xin
        for i in range(1 << L):
            a0, a1 = self.rows.node(l0 + L, (oi << L) + i)
            y[a0:a1] += self.KL[i] @ xh[(L, i, 0)]

    def entries(self):
        return (sum(V.size for V in self.V0.values()) + sum(W.size for W in self.W.values())
                + sum(K.size for K in self.KL.values()))

    def max_rank_by_level(self):
        out = [0] * (self.L + 1)
        for (k, _i, _j), s in self.skel.items():
            out[k] = max(out[k], len(s))
        return out


class CompressedInclusion:
    """K^{s2v}, K^{v2s} (butterflies) and K^{s2s} (HODBF) of a curve in the
    medium of the oracle operator ``op`` (a ``kernel.Operator``)."""

    def __init__(self, op, curve, n_of, leaf_v, leaf_s, eps, chi=20.0, radius_h=10.0):
        self.op, self.curve, self.eps = op, curve, eps
        tab, w = op.tab, op.omega
        vperm, vb = tree.cluster_tree(op.N, leaf_v)
        sperm, sb = segment_tree(curve.c, leaf_s)
        self.Ls = len(sb) - 1
        L = min(len(vb), len(sb)) - 1
        cells = np.stack([op.px, op.pz], axis=1)
        self.V = Side(cells, vperm, vb)
        self.S = Side(curve.c, sperm, sb)
        Vc, Sc = Side(cells, vperm, vb[:L + 1]), Side(curve.c, sperm, sb[:L + 1])
        cw = curve.w[sperm]                                   # lengths in tree order
        nseg = n_of(curve.c[sperm, 0], curve.c[sperm, 1])
        rad = radius_h * op.h

        # the entries, evaluated once in tree order (small grids only); the
        # butterflies read their sampled blocks from these
        G_vs = inclusion.green(tab, w, self.V.pts, self.S.pts)           # g(r_i, r^s_j)
        G_sv = inclusion.green(tab, w, self.S.pts, self.V.pts)           # g(r^s_i, r_j)
        G_ss = inclusion.green(tab, w, self.S.pts, self.S.pts)
        K_ss = -G_ss * cw[None, :]
        K_ss[np.arange(len(cw)), np.arange(len(cw))] = inclusion.s2s_self(cw, w, nseg)
        K_vs = G_vs * cw[None, :]

        def k_s2v(r, c):
            return K_vs[np.ix_(r, c)]

        def k_v2s(r, c):
            return G_sv[np.ix_(r, c)]

        def k_s2s(r, c):
            return K_ss[np.ix_(r, c)]

        self.s2v = Butterfly(k_s2v, Vc, Sc, 0, 0, 0, L, eps, chi, rad)
        self.v2s = Butterfly(k_v2s, Sc, Vc, 0, 0, 0, L, eps, chi, rad)
        self.s2s = []
        for l in range(1, self.Ls + 1):
            for p in range(1 << (l - 1)):
                for d in (0, 1):
                    self.s2s.append(Butterfly(k_s2s, self.S, self.S, l, 2 * p + d, 2 * p + 1 - d,
                                              self.Ls - l, eps, chi, rad))
        self.s2s_leaves = []
        for i in range(1 << self.Ls):
            pos = np.arange(*self.S.node(self.Ls, i))
            self.s2s_leaves.append(k_s2s(pos, pos))

    def s2s_apply(self, p):
        """K^{s2s} p, tree order."""
        y = np.zeros_like(p, dtype=np.complex128)
        for i, D in enumerate(self.s2s_leaves):
            a0, a1 = self.S.node(self.Ls, i)
            y[a0:a1] += D @ p[a0:a1]
        for bf in self.s2s:
            bf.apply(p, y)
        return y

    def total_field(self, s, v2v, tol=1e-12):
        """U = v2v + K^{s2v} (K^{s2s})^{-1} K^{v2s} I, I = s h^2 (natural order
        in and out; v2v = K^{v2v} I given)."""
        s = np.asarray(s, dtype=np.complex128)
        s = s[:, None] if s.ndim == 1 else s
        Ns, Nv = len(self.curve.w), self.op.Nv
        x = (s * self.op.h ** 2)[self.V.perm]
        U = np.zeros((Nv, s.shape[1]), dtype=np.complex128)
        for r in range(s.shape[1]):
            uinc = np.zeros(Ns, dtype=np.complex128)
            self.v2s.apply(x[:, r], uinc)
            A = spla.LinearOperator((Ns, Ns), matvec=self.s2s_apply, dtype=np.complex128)
            P, info = spla.gmres(A, uinc, rtol=tol, atol=0.0, restart=Ns, maxiter=Ns)
            if info != 0:
                raise RuntimeError(f"GMRES did not converge ({info})")
            y = np.zeros(Nv, dtype=np.complex128)
            self.s2v.apply(P, y)
            U[self.V.perm, r] = y
        return np.asarray(v2v) + U
