"""K-D cluster tree of the cell centroids and the proxy-row rule (Sec. 4.2).

Test infrastructure (see ``oracle/__init__``).

Cluster tree (Sec. 4.2): the centroid set is bisected recursively into two
halves of (nearly) equal size down to a leaf size, giving a complete binary
tree T_Hv of L_v levels.  Readings, shared with the library as a spec:
* L_v is the smallest L >= 0 with ceil(N_v / 2^L) <= leaf;
* a node is split along x if its bounding box (in cell units) is at least as
  wide in x as in z, else along z; its points are ordered by (coordinate,
  natural index) and the first ceil(n/2) go to the first child;
* the points of a leaf are listed in natural order.
Tree order is the concatenation of the leaves; each node is a contiguous
range of tree positions.

Proxy rows (Eq. proxyv2v): for a block (tau, nu) with seed columns S
(the skeleton union nu1_bar U nu2_bar, or at butterfly level 0 the points of
nu itself), tau_hat = (U_{i in S} n_i) ^ tau  U  f_tau, with n_i the centroids
within radius*h of r_i and f_tau chi*|S| points of tau picked uniformly.
Readings: f_tau takes m = min(|tau|, ceil(chi*|S|)) points at tree positions
t0 + floor(k*|tau|/m), k = 0..m-1 (a deterministic uniform stride; the
paper's "near the boundary of tau" is not reproduced); if m = |tau| the
proxy set is all of tau; the result is sorted by tree position.
"""
import math

import numpy as np


def num_levels(Nv, leaf):
    L = 0
    while -(-Nv // (1 << L)) > leaf:
        L += 1
    return L


def cluster_tree(N, leaf):
    """Return (perm, bounds): perm[p] = natural index at tree position p;
    bounds[l] = array of 2^l + 1 range boundaries of the level-l nodes."""
    Nv = N * N
    Lv = num_levels(Nv, leaf)
    a = np.arange(Nv) % N
    b = np.arange(Nv) // N
    nodes = [np.arange(Nv)]
    bounds = [np.array([0, Nv])]
    for _level in range(Lv):
        nxt = []
        for P in nodes:
            n = len(P)
            wa = a[P].max() - a[P].min() if n else 0
            wb = b[P].max() - b[P].min() if n else 0
            coord = a[P] if wa >= wb else b[P]
            order = np.lexsort((P, coord))     # primary: coord, secondary: index
            P = P[order]
            n1 = (n + 1) // 2
            nxt += [P[:n1], P[n1:]]
        nodes = nxt
        sizes = np.array([len(P) for P in nodes])
        bounds.append(np.concatenate([[0], np.cumsum(sizes)]))
    perm = np.concatenate([np.sort(P) for P in nodes])
    return perm, bounds


def proxy_rows(t0, t1, seeds, chi, radius, perm, N):
    """Eq. proxyv2v for row node tau = tree positions [t0, t1); ``seeds`` are
    tree positions.  Returns sorted tree positions."""
    size = t1 - t0
    m = min(size, int(math.ceil(chi * len(seeds))))
    if m >= size:
        return np.arange(t0, t1)
    uni = t0 + (np.arange(m) * size) // m
    pos = np.arange(t0, t1)
    a = perm[pos] % N
    b = perm[pos] // N
    sa = perm[np.asarray(seeds)] % N
    sb = perm[np.asarray(seeds)] // N
    d2 = (a[:, None] - sa[None, :]) ** 2 + (b[:, None] - sb[None, :]) ** 2
    near = pos[(d2 <= radius * radius).any(axis=1)]
    return np.union1d(uni, near)
