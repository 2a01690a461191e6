"""K^{s2v} (cells <- curve segments) as a single butterfly (Sec. 4.2, the
K^{s2v} item; Sec. 4.2.3): a prototype of the compressed surface-to-volume
operator, checked against the dense K^{s2v} of ``inclusion``.

Test infrastructure (see ``oracle/__init__``).  Slow; for small grids.

Trees.  Rows: the cell cluster tree T_{H_v} of ``tree.cluster_tree``.
Columns: a K-D tree over the segment centres built by the same rule on real
coordinates (split the longer side of the bounding box, order by
(coordinate, index), first child ceil(n/2)).  The butterfly of K(o, s) with
o, s the roots has L = min(L_v, L_s) levels (Sec. 4.2), T_o and T_s being the
two trees cut at level L.

Factors (Sec. 4.2.1, as in ``butterfly`` for K^{v2v}): at level 0 the ID of
K(tau_hat, nu) for every leaf nu of T_s with tau = o; at level k = 1..L the ID
of [K(tau_hat, nu1_bar) K(tau_hat, nu2_bar)] for tau at level k of T_o and nu
at level L - k of T_s; K^L = K(tau_i, nu_bar) at the leaves of T_o.  Proxy
rows tau_hat (Eq. proxyv2v read for a curve): the cells of tau within
``radius`` h of a seed segment centre plus m = min(|tau|, ceil(chi |seeds|))
cells of tau at a uniform stride in tree order; all of tau at k = L.
Readings: the paper states the K^{s2v} item and its complexity, not the
proxy rule for it; the volume rule with segment centres as seeds is used.
"""
import math

import numpy as np

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


class S2VButterfly:
    def __init__(self, op, curve, leaf_v, leaf_s, eps, chi=20.0, radius=10.0):
        self.op, self.curve, self.eps, self.chi, self.radius = op, curve, eps, chi, radius
        self.vperm, vb = tree.cluster_tree(op.N, leaf_v)
        self.sperm, sb = segment_tree(curve.c, leaf_s)
        self.L = L = min(len(vb), len(sb)) - 1
        self.vb, self.sb = vb[:L + 1], sb[:L + 1]
        x, z = op.px, op.pz
        self.cells = np.stack([x, z], axis=1)
        self._build()

    def _vnode(self, level, i):
        return int(self.vb[level][i]), int(self.vb[level][i + 1])

    def _snode(self, level, j):
        return int(self.sb[level][j]), int(self.sb[level][j + 1])

    def K(self, rows, cols):
        """K^{s2v}[rows, cols] for tree positions (cells, segments)."""
        r = self.cells[self.vperm[np.asarray(rows)]]
        sidx = self.sperm[np.asarray(cols)]
        sub = inclusion.Curve(self.curve.c[sidx], self.curve.w[sidx])
        return inclusion.K_s2v(self.op.tab, self.op.omega, sub, r)

    def _proxy(self, t0, t1, seeds):
        size = t1 - t0
        m = min(size, int(math.ceil(self.chi * len(seeds))))
        if m >= size:
            return np.arange(t0, t1)
        uni = t0 + (np.arange(m) * size) // m
        pos = np.arange(t0, t1)
        pc = self.cells[self.vperm[pos]]
        sc = self.curve.c[self.sperm[np.asarray(seeds)]]
        d2 = ((pc[:, None, :] - sc[None, :, :]) ** 2).sum(axis=-1)
        near = pos[(d2 <= (self.radius * self.op.h) ** 2).any(axis=1)]
        return np.union1d(uni, near)

    def _build(self):
        L = self.L
        self.V0, self.W, self.KL, skel = {}, {}, {}, {}
        t0, t1 = self._vnode(0, 0)
        for j in range(1 << L):
            n0, n1 = self._snode(L, j)
            cols = np.arange(n0, n1)
            rows = np.arange(t0, t1) if L == 0 else self._proxy(t0, t1, cols)
            sk, V, _ = cpqr.cpqr_id(self.K(rows, cols), self.eps)
            self.V0[j], skel[(0, 0, j)] = V, cols[sk]
        for k in range(1, L + 1):
            for i in range(1 << k):
                a0, a1 = self._vnode(k, i)
                for j in range(1 << (L - k)):
                    cols = np.concatenate([skel[(k - 1, i // 2, 2 * j)], skel[(k - 1, i // 2, 2 * j + 1)]])
                    rows = np.arange(a0, a1) if k == L else self._proxy(a0, a1, cols)
                    sk, Wm, _ = cpqr.cpqr_id(self.K(rows, cols), self.eps)
                    self.W[(k, i, j)], skel[(k, i, j)] = Wm, cols[sk]
        for i in range(1 << L):
            a0, a1 = self._vnode(L, i)
            self.KL[i] = self.K(np.arange(a0, a1), skel[(L, i, 0)])
        self.skel = skel

    def apply(self, p):
        """u = K^{s2v} p: p over the segments (natural order, (N_s, nrhs)),
        u over the cells (natural order)."""
        p = np.asarray(p, dtype=np.complex128)
        p = p[:, None] if p.ndim == 1 else p
        x = p[self.sperm]
        L = self.L
        xh = {}
        for j in range(1 << L):
            n0, n1 = self._snode(L, j)
            xh[(0, 0, j)] = self.V0[j] @ x[n0:n1]
        for k in range(1, L + 1):
            for i in range(1 << k):
                for j in range(1 << (L - k)):
                    xin = np.concatenate([xh[(k - 1, i // 2, 2 * j)], xh[(k - 1, i // 2, 2 * j + 1)]])
                    xh[(k, i, j)] = self.W[(k, i, j)] @ xin
        y = np.zeros((self.op.Nv, p.shape[1]), dtype=np.complex128)
        for i in range(1 << L):
            a0, a1 = self._vnode(L, i)
            y[a0:a1] = self.KL[i] @ xh[(L, i, 0)]
        u = np.empty_like(y)
        u[self.vperm] = y
        return u

    def factor_entries(self):
        return (sum(V.size for V in self.V0.values()) + sum(W.size for W in self.W.values())
                + sum(K.size for K in self.KL.values()))

    def max_rank_by_level(self):
        """The largest skeleton size at each butterfly level k = 0..L."""
        out = [0] * (self.L + 1)
        for (k, _i, _j), s in self.skel.items():
            out[k] = max(out[k], len(s))
        return out
