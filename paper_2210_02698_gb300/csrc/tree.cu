// tree.cu - host side K-D cluster tree of the cell centroids and the
// proxy-row rule (Sec. 4.2; Eq. proxyv2v).
//
// Cluster tree (Sec. 4.2): the centroids are bisected recursively into two
// halves down to the leaf size, a complete binary tree of L_v levels, L_v the
// smallest L with ceil(N_v / 2^L) <= leaf.  A node is split along x when its
// bounding box (in cells) is at least as wide in x as in z, else along z; its
// points are ordered by (coordinate, natural index) and the first ceil(n/2)
// form the first child.  Leaf points are listed in natural order.  Tree order
// concatenates the leaves, so every node is a contiguous range of positions.
//
// Proxy rows (Eq. proxyv2v): for row node tau = positions [t0, t1) and seed
// columns S, tau_hat = (neighbours within R h of S, inside tau) U f_tau with
// f_tau the m = min(|tau|, ceil(chi |S|)) positions t0 + floor(k |tau| / m);
// when m = |tau| the proxy set is tau itself.  Sorted by position.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "hb_internal.cuh"

namespace hb {

void tree_build(hb_ctx* c) {
  const long long Nv = c->Nv;
  const int nx = c->nx;
  int Lv = 0;
  while ((Nv + (1LL << Lv) - 1) / (1LL << Lv) > c->opt.leaf) ++Lv;
  c->Lv = Lv;
  std::vector<long long> P((size_t)Nv);
  std::iota(P.begin(), P.end(), 0LL);
  c->bounds.assign(Lv + 1, {});
  c->bounds[0] = {0, Nv};
  std::vector<std::pair<long long, long long>> keyed;
  for (int l = 0; l < Lv; ++l) {
    const std::vector<long long>& B = c->bounds[l];
    std::vector<long long> nb;
    nb.reserve(B.size() * 2);
    nb.push_back(0);
    for (size_t k = 0; k + 1 < B.size(); ++k) {
      long long s = B[k], e = B[k + 1], n = e - s;
      long long amin = 1LL << 62, amax = -1, bmin = 1LL << 62, bmax = -1;
      for (long long i = s; i < e; ++i) {
        long long a = P[i] % nx, b = P[i] / nx;
        amin = std::min(amin, a);
        amax = std::max(amax, a);
        bmin = std::min(bmin, b);
        bmax = std::max(bmax, b);
      }
      const bool splitx = n == 0 || (amax - amin) >= (bmax - bmin);
      keyed.resize((size_t)n);
      for (long long i = 0; i < n; ++i) {
        long long p = P[s + i];
        keyed[i] = {splitx ? p % nx : p / nx, p};
      }
      std::sort(keyed.begin(), keyed.end());
      for (long long i = 0; i < n; ++i) P[s + i] = keyed[i].second;
      nb.push_back(s + (n + 1) / 2);
      nb.push_back(e);
    }
    c->bounds[l + 1] = nb;
  }
  const std::vector<long long>& leaves = c->bounds[Lv];
  for (size_t k = 0; k + 1 < leaves.size(); ++k) std::sort(P.begin() + leaves[k], P.begin() + leaves[k + 1]);
  c->perm = P;
  c->iperm.assign((size_t)Nv, 0);
  for (long long i = 0; i < Nv; ++i) c->iperm[P[i]] = i;
}

void segment_tree_build(const double* cx, const double* cz, long long ns, int leaf, std::vector<long long>& perm,
                        std::vector<std::vector<long long>>& bounds) {
  int L = 0;
  while ((ns + (1LL << L) - 1) / (1LL << L) > leaf) ++L;
  std::vector<std::vector<long long>> nodes(1);
  nodes[0].resize((size_t)ns);
  std::iota(nodes[0].begin(), nodes[0].end(), 0LL);
  bounds.assign(1, {0, ns});
  std::vector<std::pair<double, long long>> keyed;
  for (int l = 0; l < L; ++l) {
    std::vector<std::vector<long long>> nxt;
    nxt.reserve(nodes.size() * 2);
    std::vector<long long> nb{0};
    for (const std::vector<long long>& P : nodes) {
      std::vector<long long> a, b;
      if (!P.empty()) {
        double xmin = cx[P[0]], xmax = xmin, zmin = cz[P[0]], zmax = zmin;
        for (long long i : P) {
          xmin = std::min(xmin, cx[i]);
          xmax = std::max(xmax, cx[i]);
          zmin = std::min(zmin, cz[i]);
          zmax = std::max(zmax, cz[i]);
        }
        const bool splitx = (xmax - xmin) >= (zmax - zmin);
        keyed.resize(P.size());
        for (size_t i = 0; i < P.size(); ++i) keyed[i] = {splitx ? cx[P[i]] : cz[P[i]], P[i]};
        std::sort(keyed.begin(), keyed.end());
        const size_t n1 = (P.size() + 1) / 2;
        for (size_t i = 0; i < keyed.size(); ++i) (i < n1 ? a : b).push_back(keyed[i].second);
      }
      nb.push_back(nb.back() + (long long)a.size());
      nb.push_back(nb.back() + (long long)b.size());
      nxt.push_back(std::move(a));
      nxt.push_back(std::move(b));
    }
    nodes = std::move(nxt);
    bounds.push_back(std::move(nb));
  }
  perm.clear();
  for (std::vector<long long>& P : nodes) {
    std::sort(P.begin(), P.end());
    perm.insert(perm.end(), P.begin(), P.end());
  }
}

void point_proxy_rows(const double* rows_xz, long long t0, long long t1, const double* seeds_xz, int nseeds,
                      double chi, double radius, std::vector<long long>& out) {
  out.clear();
  const long long size = t1 - t0;
  const long long m = std::min(size, (long long)std::ceil(chi * (double)nseeds));
  if (m >= size) {
    out.resize((size_t)size);
    std::iota(out.begin(), out.end(), t0);
    return;
  }
  for (long long k = 0; k < m; ++k) out.push_back(t0 + (k * size) / m);
  const double R2 = radius * radius;
  for (long long pos = t0; pos < t1; ++pos) {
    const double x = rows_xz[2 * pos], z = rows_xz[2 * pos + 1];
    for (int s = 0; s < nseeds; ++s) {
      const double dx = x - seeds_xz[2 * s], dz = z - seeds_xz[2 * s + 1];
      if (dx * dx + dz * dz <= R2) {
        out.push_back(pos);
        break;
      }
    }
  }
  std::sort(out.begin(), out.end());
  out.erase(std::unique(out.begin(), out.end()), out.end());
}

void proxy_rows(const hb_ctx* c, long long t0, long long t1, const long long* seeds, int nseeds,
                std::vector<long long>& out, std::vector<int>& stamp, int stamp_id) {
  out.clear();
  const long long size = t1 - t0;
  const long long m = std::min(size, (long long)std::ceil(c->opt.chi * (double)nseeds));
  if (m >= size) {
    out.resize((size_t)size);
    std::iota(out.begin(), out.end(), t0);
    return;
  }
  auto mark = [&](long long pos) {
    if (stamp[pos] != stamp_id) {
      stamp[pos] = stamp_id;
      out.push_back(pos);
    }
  };
  for (long long k = 0; k < m; ++k) mark(t0 + (k * size) / m);
  const double R = c->opt.nbr_radius_h;
  const int Ri = (int)std::floor(R);
  const double R2 = R * R;
  const int nx = c->nx, ny = c->ny;
  for (int s = 0; s < nseeds; ++s) {
    const long long nat = c->perm[seeds[s]];
    const int as = (int)(nat % nx), bs = (int)(nat / nx);
    for (int db = -Ri; db <= Ri; ++db) {
      const int b = bs + db;
      if (b < 0 || b >= ny) continue;
      for (int da = -Ri; da <= Ri; ++da) {
        const int a = as + da;
        if (a < 0 || a >= nx) continue;
        if ((double)(da * da + db * db) > R2) continue;
        const long long pos = c->iperm[(long long)b * nx + a];
        if (pos >= t0 && pos < t1) mark(pos);
      }
    }
  }
  std::sort(out.begin(), out.end());
}

}  // namespace hb
