"""Plain HODBF / column-wise butterfly construction and apply (Sec. 4.2).

Test infrastructure (see ``oracle/__init__``).  Slow; for small grids.

HODBF layout (Sec. 4.2, K^{v2v} item): for siblings tau1, tau2 at level l of
the cluster tree, K(tau1, tau2) and K(tau2, tau1) are butterflies with
L = L_v - l levels; the leaf diagonal blocks K(tau, tau) stay dense.

Butterfly of K(o, s) (Sec. 4.2.1):
* level 0: for each leaf nu of T_s and tau = o, the ID of the proxy block
  K(tau_hat, nu) ~ K(tau_hat, nu_bar) V_{tau,nu}  (Eq. proxy, l = 0);
* level l = 1..L: for tau at level l of T_o, nu at level L-l of T_s with
  children nu1, nu2: the ID of [K(tau_hat, nu1_bar) K(tau_hat, nu2_bar)] ~
  K(tau_hat, nu_bar) W_{tau,nu}, nui_bar the skeletons of (p_tau, nui)
  (Eq. transfer_computation, Eq. proxy); at l = L the proxy set is tau itself;
* K^L = diag(K(tau_i, nu_bar)) over the leaves tau_i of T_o with nu = s.
Apply (Eq. butterfly_mat): y = K^L W^L ... W^1 V^0 x, i.e.
  xh0[nu] = V_{o,nu} x(nu);  xhl[tau,nu] = W_{tau,nu} [xh(p_tau,nu1); xh(p_tau,nu2)];
  y(tau_i) = K(tau_i, nu_bar) xhL[tau_i, s].
All indices here are tree positions; x and y are in tree order.
"""
import numpy as np

from . import cpqr, tree


class HODBF:
    def __init__(self, op, leaf, eps, chi, radius):
        self.op = op
        self.perm, self.bounds = tree.cluster_tree(op.N, leaf)
        self.Lv = len(self.bounds) - 1
        self.eps, self.chi, self.radius = eps, chi, radius
        self.bfs = []
        for l in range(1, self.Lv + 1):
            for p in range(1 << (l - 1)):
                for d in (0, 1):
                    self.bfs.append(self._build(l, 2 * p + d, 2 * p + 1 - d))
        self.leaves = []
        for i in range(1 << self.Lv):
            t0, t1 = self.node(self.Lv, i)
            nat = self.perm[t0:t1]
            self.leaves.append(op.block(nat, nat))

    def node(self, level, idx):
        b = self.bounds[level]
        return int(b[idx]), int(b[idx + 1])

    def K(self, rows, cols):
        return self.op.block(self.perm[np.asarray(rows)], self.perm[np.asarray(cols)])

    def _build(self, l, oi, si):
        L = self.Lv - l
        skel = {}
        V0 = {}
        W = {}
        for j in range(1 << L):
            t0, t1 = self.node(l, oi)
            n0, n1 = self.node(l + L, si * (1 << L) + j)
            cols = np.arange(n0, n1)
            if L == 0:
                rows = np.arange(t0, t1)
            else:
                rows = tree.proxy_rows(t0, t1, cols, self.chi, self.radius, self.perm, self.op.N)
            sk, V, _ = cpqr.cpqr_id(self.K(rows, cols), self.eps)
            V0[j] = V
            skel[(0, 0, j)] = cols[sk]
        for k in range(1, L + 1):
            for i in range(1 << k):
                t0, t1 = self.node(l + k, oi * (1 << k) + i)
                for j in range(1 << (L - k)):
                    cols = np.concatenate([skel[(k - 1, i // 2, 2 * j)],
                                           skel[(k - 1, i // 2, 2 * j + 1)]])
                    if k == L:
                        rows = np.arange(t0, t1)
                    else:
                        rows = tree.proxy_rows(t0, t1, cols, self.chi, self.radius,
                                               self.perm, self.op.N)
                    sk, Wm, _ = cpqr.cpqr_id(self.K(rows, cols), self.eps)
                    W[(k, i, j)] = Wm
                    skel[(k, i, j)] = cols[sk]
        KL = {}
        for i in range(1 << L):
            t0, t1 = self.node(l + L, oi * (1 << L) + i)
            KL[i] = self.K(np.arange(t0, t1), skel[(L, i, 0)])
        return dict(l=l, oi=oi, si=si, L=L, V0=V0, W=W, KL=KL, skel=skel)

    def apply_tree(self, x):
        """y = K x with x, y in tree order, shape (N_v, nrhs)."""
        y = np.zeros_like(x, dtype=np.complex128)
        for i, D in enumerate(self.leaves):
            t0, t1 = self.node(self.Lv, i)
            y[t0:t1] += D @ x[t0:t1]
        for bf in self.bfs:
            l, oi, si, L = bf["l"], bf["oi"], bf["si"], bf["L"]
            xh = {}
            for j in range(1 << L):
                n0, n1 = self.node(l + L, si * (1 << L) + j)
                xh[(0, 0, j)] = bf["V0"][j] @ x[n0:n1]
            for k in range(1, L + 1):
                for i in range(1 << k):
                    for j in range(1 << (L - k)):
                        xin = np.concatenate([xh[(k - 1, i // 2, 2 * j)],
                                              xh[(k - 1, i // 2, 2 * j + 1)]])
                        xh[(k, i, j)] = bf["W"][(k, i, j)] @ xin
            for i in range(1 << L):
                t0, t1 = self.node(l + L, oi * (1 << L) + i)
                y[t0:t1] += bf["KL"][i] @ xh[(L, i, 0)]
        return y

    def apply(self, s):
        """u = K (s h^2), natural order in and out (Eq. m_v2v)."""
        s = np.asarray(s, dtype=np.complex128)
        if s.ndim == 1:
            s = s[:, None]
        x = s[self.perm] * self.op.h ** 2
        y = self.apply_tree(x)
        u = np.empty_like(y)
        u[self.perm] = y
        return u

    def factor_entries(self):
        e = sum(D.size for D in self.leaves)
        for bf in self.bfs:
            e += sum(V.size for V in bf["V0"].values())
            e += sum(Wm.size for Wm in bf["W"].values())
            e += sum(Km.size for Km in bf["KL"].values())
        return e
