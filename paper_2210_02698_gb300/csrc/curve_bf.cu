// curve_bf.cu - the volume / curve operators of an inclusion in compressed
// form (Sec. 3.2 and the K^{v2s}, K^{s2v} items of Sec. 4.2): each is one
// butterfly (Sec. 4.2.1) between the cells' cluster tree and the segments'
// K-D tree, both cut at L = min(L_v, L_s) levels, built on the device and
// applied by the FP64 step tasks of the volume operator.
//
// Butterfly of K(rows, cols) (roots o, s; L levels):
// * level 0: for every column node nu at level L, the ID (Eq. ID) of
//   K(tau_hat, nu) with tau = o - the skeleton columns of nu and
//   V_nu (rank x |nu|);
// * level k = 1..L: for tau at level k below o and nu at level L - k below
//   s, the ID of [K(tau_hat, nu1_bar) K(tau_hat, nu2_bar)] (nu1_bar, nu2_bar:
//   the children's skeletons at level k - 1, under tau's parent) -
//   W (rank x (r1 + r2)) and the skeleton of (tau, nu);
// * K^L_tau = K(tau, skeleton of (tau, s)) for tau at level L;
// tau_hat = the proxy rows of tau (Eq. proxyv2v with the other set's
// points as seeds: the rows within nbr_radius_h h of a seed column, plus
// ceil(chi |seeds|) rows of tau at a uniform stride; all of tau at k = L).
// Apply: xh(0, nu) = V_nu x(nu); xh(k, tau, nu) = W [xh(nu1); xh(nu2)];
// y(tau) = K^L_tau xh(L, tau).  K^{v2s}_ij = g(r^s_i, r_j) (rows: segments,
// columns: cells), K^{s2v}_ij = g(r_i, r^s_j) w_j (rows: cells, columns:
// segments), g = v0 f0 + v1 f1 interpolated at the points (inclusion.cu).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <vector>

#include "hb_internal.cuh"

namespace hb {
namespace {

// one side of a butterfly: points and weights in tree order, tree bounds
struct BfSide {
  std::vector<long long> perm;                  // tree position -> natural index
  std::vector<std::vector<long long>> bounds;   // [level] node boundaries (2^l + 1)
  std::vector<double> xz;                       // (x, z) of tree position p at 2p, 2p + 1
  std::vector<double> w;                        // weight of tree position p (empty: 1)
  long long size() const { return (long long)perm.size(); }
};

struct CurveBfly {
  int L = 0;
  long long nrows = 0, ncols = 0, xh_rows = 0, entries = 0;
  std::vector<int> step_begin;
  std::vector<int> max_rank;    // per butterfly level
  Task* d_tasks = nullptr;
  double2* d_F = nullptr;
  long long* d_rperm = nullptr;
  long long* d_cperm = nullptr;
  int cap = 0;                  // right-hand sides the vectors hold
  double2* d_x = nullptr;
  double2* d_y = nullptr;
  double2* d_xh = nullptr;
};

void free_bfly(CurveBfly* B) {
  if (!B) return;
  for (void* p : {(void*)B->d_tasks, (void*)B->d_F, (void*)B->d_rperm, (void*)B->d_cperm, (void*)B->d_x,
                  (void*)B->d_y, (void*)B->d_xh})
    dev_free(p);
  delete B;
}

// a device array freed on scope exit
template <class T>
struct DevBuf {
  T* p = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { dev_free(p); }
  T* take() {
    T* q = p;
    p = nullptr;
    return q;
  }
};

template <class T>
void to_dev(DevBuf<T>& d, const std::vector<T>& v) {
  d.p = upload(v);
}

// x[p R + r] = scale * src[r ld + perm[p]]
__global__ void gather_tree_kernel(const double2* __restrict__ src, long long ld, const long long* __restrict__ perm,
                                   long long n, int R, double scale, double2* __restrict__ x) {
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n * R;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long p = idx / R;
    const int r = (int)(idx % R);
    const double2 v = src[(size_t)r * ld + perm[p]];
    x[idx] = make_double2(scale * v.x, scale * v.y);
  }
}

// dst[r ld + perm[p]] (= or +=) y[p R + r]
__global__ void scatter_tree_kernel(const double2* __restrict__ y, const long long* __restrict__ perm, long long n,
                                    int R, double2* __restrict__ dst, long long ld, int accumulate) {
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n * R;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long p = idx / R;
    const int r = (int)(idx % R);
    double2* o = dst + (size_t)r * ld + perm[p];
    const double2 v = y[idx];
    *o = accumulate ? make_double2(o->x + v.x, o->y + v.y) : v;
  }
}

// One copy per CTA: rows [row0, row0 + rows) of the column-major block at
// src + src_off (ld src_ld, cols columns) to a rows x cols block at dst_off.
struct RowChunk {
  long long src_off, dst_off;
  int src_ld, rows, cols, row0;
};
__global__ void rechunk_kernel(const double2* __restrict__ src, const RowChunk* __restrict__ ch,
                               double2* __restrict__ dst) {
  const RowChunk c = ch[blockIdx.x];
  for (long long e = threadIdx.x; e < (long long)c.rows * c.cols; e += blockDim.x) {
    const long long col = e / c.rows, r = e % c.rows;
    dst[c.dst_off + e] = src[c.src_off + col * c.src_ld + c.row0 + r];
  }
}

unsigned grid_for(long long total) {
  return (unsigned)std::max<long long>(1, std::min<long long>((total + 255) / 256, 152LL * 8));
}

// The sampled blocks K(rows[b], cols[b]) (rows on side R, columns on side C,
// column weights C.w) into d_out, block b column-major at off[b].
void eval_blocks(const hb_ctx* c, const BfSide& R, const BfSide& C, const std::vector<std::vector<long long>>& rows,
                 const std::vector<std::vector<long long>>& cols, const std::vector<long long>& off, double2* d_out) {
  std::vector<double2> obs;
  std::vector<GreenCol> jobs;
  for (size_t b = 0; b < rows.size(); ++b) {
    const long long obs0 = (long long)obs.size(), m = (long long)rows[b].size();
    for (long long p : rows[b]) obs.push_back(make_double2(R.xz[2 * p], R.xz[2 * p + 1]));
    for (size_t t = 0; t < cols[b].size(); ++t) {
      const long long q = cols[b][t];
      GreenCol J{};
      J.obs0 = obs0;
      J.out_off = off[b] + (long long)t * m;
      J.src = make_double2(C.xz[2 * q], C.xz[2 * q + 1]);
      J.w = C.w.empty() ? 1.0 : C.w[(size_t)q];
      J.m = (int)m;
      jobs.push_back(J);
    }
  }
  if (jobs.empty()) return;
  DevBuf<double2> d_obs;
  DevBuf<GreenCol> d_jobs;
  to_dev(d_obs, obs);
  to_dev(d_jobs, jobs);
  green_jobs(c, d_obs.p, d_jobs.p, (long long)jobs.size(), d_out, 0);
  HB_CUDA(cudaDeviceSynchronize());
}

// The IDs of one level's blocks (column-major in d_A at aoff): ranks,
// pivot orders (the skeleton first) and V = rank x n (ld rank) into a new
// buffer *V at voff.
void id_level(const hb_ctx* c, double2* d_A, const std::vector<int>& m, const std::vector<int>& n,
              const std::vector<long long>& aoff, std::vector<int>& rank, std::vector<std::vector<int>>& piv,
              DevBuf<double2>& V, std::vector<long long>& voff) {
  const int cnt = (int)m.size();
  std::vector<long long> soff((size_t)cnt);
  long long sacc = 0;
  int max_n = 0;
  for (int b = 0; b < cnt; ++b) {
    soff[(size_t)b] = sacc;
    sacc += n[(size_t)b];
    max_n = std::max(max_n, n[(size_t)b]);
  }
  // the ID kernel keeps 28 bytes per column of a block in shared memory
  if (max_n > 8000)
    throw Error{HB_ERR_UNSUPPORTED,
                "a curve butterfly block with more than 8000 columns (too few tree levels: more segments or a "
                "smaller leaf_s)"};
  DevBuf<int> d_m, d_n, d_rank, d_perm;
  DevBuf<long long> d_a, d_s, d_v;
  to_dev(d_m, m);
  to_dev(d_n, n);
  to_dev(d_a, aoff);
  to_dev(d_s, soff);
  d_rank.p = dev_alloc<int>((size_t)cnt);
  d_perm.p = dev_alloc<int>((size_t)sacc);
  id_batch(cnt, d_m.p, d_n.p, d_a.p, d_A, c->opt.eps, d_rank.p, d_perm.p, d_s.p, max_n, 0);
  HB_CUDA(cudaDeviceSynchronize());
  rank.assign((size_t)cnt, 0);
  std::vector<int> perm((size_t)sacc);
  HB_CUDA(cudaMemcpy(rank.data(), d_rank.p, sizeof(int) * cnt, cudaMemcpyDeviceToHost));
  HB_CUDA(cudaMemcpy(perm.data(), d_perm.p, sizeof(int) * sacc, cudaMemcpyDeviceToHost));
  piv.assign((size_t)cnt, {});
  voff.assign((size_t)cnt, 0);
  long long vacc = 0;
  for (int b = 0; b < cnt; ++b) {
    piv[(size_t)b].assign(perm.begin() + soff[(size_t)b], perm.begin() + soff[(size_t)b] + n[(size_t)b]);
    voff[(size_t)b] = vacc;
    vacc += (long long)rank[(size_t)b] * n[(size_t)b];
  }
  to_dev(d_v, voff);
  V.p = dev_alloc<double2>((size_t)std::max<long long>(vacc, 1));
  emit_v(cnt, d_m.p, d_n.p, d_a.p, d_A, d_rank.p, d_perm.p, d_s.p, d_v.p, 1, V.p, nullptr, 0);
  HB_CUDA(cudaDeviceSynchronize());
}

// One butterfly K(rows on R, columns on C), both trees cut at L levels.
CurveBfly* build_bfly(const hb_ctx* c, const BfSide& R, const BfSide& C, int L) {
  const double chi = c->opt.chi, radius = c->opt.nbr_radius_h * c->h;
  std::unique_ptr<CurveBfly, void (*)(CurveBfly*)> B(new CurveBfly(), free_bfly);
  B->L = L;
  B->nrows = R.size();
  B->ncols = C.size();
  B->max_rank.assign((size_t)L + 1, 0);
  std::vector<std::vector<std::vector<long long>>> skel((size_t)L + 1);
  std::vector<std::vector<long long>> xh_off((size_t)L + 1);
  std::vector<Task> tasks;
  std::vector<int> sb{0};
  std::vector<std::pair<double2*, long long>> parts;   // factor buffers in arena order (device, size)
  auto free_parts = [&]() {
    for (auto& q : parts) dev_free(q.first);
    parts.clear();
  };
  long long fbase = 0, xh = 0;
  try {
    const int nb = 1 << L;   // blocks per level: 2^k row nodes x 2^(L-k) column nodes
    for (int k = 0; k <= L; ++k) {
      std::vector<std::vector<long long>> rows((size_t)nb), cols((size_t)nb);
      const int nj = 1 << (L - k);
      for (int i = 0; i < (1 << k); ++i) {
        const long long a0 = R.bounds[(size_t)k][(size_t)i], a1 = R.bounds[(size_t)k][(size_t)i + 1];
        for (int j = 0; j < nj; ++j) {
          const size_t b = (size_t)i * nj + j;
          if (k == 0) {
            for (long long q = C.bounds[(size_t)L][(size_t)j]; q < C.bounds[(size_t)L][(size_t)j + 1]; ++q)
              cols[b].push_back(q);
          } else {
            const size_t c1 = (size_t)(i / 2) * (2 * nj) + 2 * j;
            cols[b] = skel[(size_t)k - 1][c1];
            cols[b].insert(cols[b].end(), skel[(size_t)k - 1][c1 + 1].begin(), skel[(size_t)k - 1][c1 + 1].end());
          }
          if (a1 <= a0 || cols[b].empty()) throw Error{HB_ERR_UNSUPPORTED, "an empty tree node in a curve butterfly"};
          if (k == L) {
            for (long long p = a0; p < a1; ++p) rows[b].push_back(p);
          } else {
            std::vector<double> seeds;
            for (long long q : cols[b]) {
              seeds.push_back(C.xz[2 * q]);
              seeds.push_back(C.xz[2 * q + 1]);
            }
            point_proxy_rows(R.xz.data(), a0, a1, seeds.data(), (int)cols[b].size(), chi, radius, rows[b]);
          }
        }
      }
      std::vector<int> m((size_t)nb), n((size_t)nb);
      std::vector<long long> aoff((size_t)nb);
      long long aacc = 0;
      for (int b = 0; b < nb; ++b) {
        m[(size_t)b] = (int)rows[(size_t)b].size();
        n[(size_t)b] = (int)cols[(size_t)b].size();
        aoff[(size_t)b] = aacc;
        aacc += (long long)m[(size_t)b] * n[(size_t)b];
      }
      DevBuf<double2> d_A, V;
      d_A.p = dev_alloc<double2>((size_t)aacc);
      eval_blocks(c, R, C, rows, cols, aoff, d_A.p);
      std::vector<int> rank;
      std::vector<std::vector<int>> piv;
      std::vector<long long> voff;
      id_level(c, d_A.p, m, n, aoff, rank, piv, V, voff);
      skel[(size_t)k].resize((size_t)nb);
      xh_off[(size_t)k].resize((size_t)nb);
      long long lsize = 0;
      for (int b = 0; b < nb; ++b) {
        const int r = rank[(size_t)b];
        for (int t = 0; t < r; ++t) skel[(size_t)k][(size_t)b].push_back(cols[(size_t)b][(size_t)piv[(size_t)b][(size_t)t]]);
        xh_off[(size_t)k][(size_t)b] = xh;
        xh += r;
        B->max_rank[(size_t)k] = std::max(B->max_rank[(size_t)k], r);
        Task t{};
        t.y_off = xh_off[(size_t)k][(size_t)b];
        t.r_out = r;
        t.y_buf = 2;
        if (k == 0) {
          t.nterm = 1;
          t.x_buf = 0;
          t.f_off[0] = fbase + voff[(size_t)b];
          t.x_off[0] = cols[(size_t)b].front();   // the column node's first tree position
          t.r_in[0] = n[(size_t)b];
        } else {
          const int i = b / nj, j = b % nj;
          const size_t c1 = (size_t)(i / 2) * (2 * nj) + 2 * j;
          const int r1 = (int)skel[(size_t)k - 1][c1].size(), r2 = (int)skel[(size_t)k - 1][c1 + 1].size();
          t.nterm = 2;
          t.x_buf = 2;
          t.f_off[0] = fbase + voff[(size_t)b];
          t.f_off[1] = fbase + voff[(size_t)b] + (long long)r * r1;
          t.x_off[0] = xh_off[(size_t)k - 1][c1];
          t.x_off[1] = xh_off[(size_t)k - 1][c1 + 1];
          t.r_in[0] = r1;
          t.r_in[1] = r2;
        }
        tasks.push_back(t);
        lsize += (long long)r * n[(size_t)b];
      }
      sb.push_back((int)tasks.size());
      parts.push_back({V.take(), lsize});
      fbase += lsize;
    }
    // K^L_tau = K(tau, skeleton of (tau, s)), tau at level L
    std::vector<std::vector<long long>> rows((size_t)nb), cols((size_t)nb);
    std::vector<long long> koff((size_t)nb);
    long long kacc = 0;
    for (int i = 0; i < nb; ++i) {
      for (long long p = R.bounds[(size_t)L][(size_t)i]; p < R.bounds[(size_t)L][(size_t)i + 1]; ++p)
        rows[(size_t)i].push_back(p);
      cols[(size_t)i] = skel[(size_t)L][(size_t)i];
      koff[(size_t)i] = kacc;
      kacc += (long long)rows[(size_t)i].size() * (long long)cols[(size_t)i].size();
      Task t{};
      t.y_off = R.bounds[(size_t)L][(size_t)i];
      t.r_out = (int)rows[(size_t)i].size();
      t.y_buf = 1;
      t.nterm = 1;
      t.x_buf = 2;
      t.f_off[0] = fbase + koff[(size_t)i];
      t.x_off[0] = xh_off[(size_t)L][(size_t)i];
      t.r_in[0] = (int)cols[(size_t)i].size();
      tasks.push_back(t);
    }
    sb.push_back((int)tasks.size());
    DevBuf<double2> KL;
    KL.p = dev_alloc<double2>((size_t)std::max<long long>(kacc, 1));
    eval_blocks(c, R, C, rows, cols, koff, KL.p);
    parts.push_back({KL.take(), kacc});
    fbase += kacc;
    // the factor arena, in task order
    DevBuf<double2> F;
    F.p = dev_alloc<double2>((size_t)std::max<long long>(fbase, 1));
    long long at = 0;
    for (auto& q : parts) {
      if (q.second) HB_CUDA(cudaMemcpy(F.p + at, q.first, sizeof(double2) * q.second, cudaMemcpyDeviceToDevice));
      at += q.second;
    }
    free_parts();
    // tasks of more than CHUNK output rows split by rows (more CTAs per
    // step: a level has only 2^L tasks), each chunk's factor rows copied to
    // a block of their own (the tasks read F with the leading dimension
    // r_out)
    constexpr int CHUNK = 16;
    std::vector<Task> split;
    std::vector<RowChunk> chunks;
    std::vector<int> sb2{0};
    long long nf = 0;
    for (size_t st = 0; st + 1 < sb.size(); ++st) {
      for (int q = sb[st]; q < sb[st + 1]; ++q) {
        const Task& t = tasks[(size_t)q];
        const int cols = t.r_in[0] + (t.nterm == 2 ? t.r_in[1] : 0);
        for (int r0 = 0; r0 < t.r_out; r0 += CHUNK) {
          const int cr = std::min(CHUNK, t.r_out - r0);
          Task u = t;
          u.y_off = t.y_off + r0;
          u.r_out = cr;
          u.f_off[0] = nf;
          if (t.nterm == 2) u.f_off[1] = nf + (long long)cr * t.r_in[0];
          split.push_back(u);
          chunks.push_back(RowChunk{t.f_off[0], nf, t.r_out, cr, cols, r0});
          nf += (long long)cr * cols;
        }
      }
      sb2.push_back((int)split.size());
    }
    B->d_F = dev_alloc<double2>((size_t)std::max<long long>(nf, 1));
    if (!chunks.empty()) {
      DevBuf<RowChunk> d_ch;
      to_dev(d_ch, chunks);
      for (size_t b0 = 0; b0 < chunks.size(); b0 += (1u << 30)) {
        const unsigned n = (unsigned)std::min<size_t>(chunks.size() - b0, 1u << 30);
        rechunk_kernel<<<n, 256>>>(F.p, d_ch.p + b0, B->d_F);
        HB_CHECK_LAUNCH();
      }
      HB_CUDA(cudaDeviceSynchronize());
    }
    tasks.swap(split);
    sb.swap(sb2);
    B->entries = fbase;
    B->xh_rows = xh;
    B->step_begin = sb;
    B->d_tasks = upload(tasks);
    B->d_rperm = upload(R.perm);
    B->d_cperm = upload(C.perm);
    HB_CUDA(cudaDeviceSynchronize());
  } catch (...) {
    free_parts();
    throw;
  }
  return B.release();
}

}  // namespace

void curve_bf_free(hb_ctx* c) {
  for (int q = 0; q < 2; ++q) {
    free_bfly(static_cast<CurveBfly*>(c->curve_bf[q]));
    c->curve_bf[q] = nullptr;
  }
}

void curve_compress(hb_ctx* c, int leaf_s) {
  if (c->ns == 0) throw Error{HB_ERR_STATE, "no curve set (hb_curve_set)"};
  if (leaf_s < 1) throw arg_error("leaf_s must be >= 1");
  const long long ns = c->ns;
  // the two sides: cells (the cluster tree) and segments (their K-D tree)
  BfSide cells, segs;
  cells.perm = c->perm;
  cells.bounds = c->bounds;
  cells.xz.resize((size_t)c->Nv * 2);
  for (long long p = 0; p < c->Nv; ++p) {
    const long long q = c->perm[(size_t)p];
    cells.xz[(size_t)(2 * p)] = c->x0 + ((double)(q % c->nx) + 0.5) * c->h;
    cells.xz[(size_t)(2 * p + 1)] = c->y0 + ((double)(q / c->nx) + 0.5) * c->h;
  }
  std::vector<double2> cen((size_t)ns);
  std::vector<double> len((size_t)ns), cx((size_t)ns), cz((size_t)ns);
  HB_CUDA(cudaMemcpy(cen.data(), c->d_seg, sizeof(double2) * ns, cudaMemcpyDeviceToHost));
  HB_CUDA(cudaMemcpy(len.data(), c->d_segw, sizeof(double) * ns, cudaMemcpyDeviceToHost));
  for (long long i = 0; i < ns; ++i) {
    cx[(size_t)i] = cen[(size_t)i].x;
    cz[(size_t)i] = cen[(size_t)i].y;
  }
  segment_tree_build(cx.data(), cz.data(), ns, leaf_s, segs.perm, segs.bounds);
  segs.xz.resize((size_t)ns * 2);
  segs.w.resize((size_t)ns);
  for (long long p = 0; p < ns; ++p) {
    const long long q = segs.perm[(size_t)p];
    segs.xz[(size_t)(2 * p)] = cx[(size_t)q];
    segs.xz[(size_t)(2 * p + 1)] = cz[(size_t)q];
    segs.w[(size_t)p] = len[(size_t)q];
  }
  const int L = std::min((int)cells.bounds.size(), (int)segs.bounds.size()) - 1;
  curve_bf_free(c);
  // K^{v2s}: rows segments, columns cells (unweighted); K^{s2v}: rows
  // cells, columns segments weighted by their lengths
  CurveBfly* v2s = build_bfly(c, segs, cells, L);
  CurveBfly* s2v = nullptr;
  try {
    s2v = build_bfly(c, cells, segs, L);
  } catch (...) {
    free_bfly(v2s);
    throw;
  }
  c->curve_bf[0] = v2s;
  c->curve_bf[1] = s2v;
  // the dense forms are not needed any more
  dev_free(c->d_kv2s);
  dev_free(c->d_ks2v);
  c->d_kv2s = c->d_ks2v = nullptr;
}

void curve_bf_apply(hb_ctx* c, int which, const double2* x_nat, long long ldx, double scale, double2* y_nat,
                    long long ldy, int accumulate, int nrhs, cudaStream_t st) {
  CurveBfly* B = static_cast<CurveBfly*>(c->curve_bf[which]);
  if (!B) throw Error{HB_ERR_STATE, "no compressed curve operator"};
  if (B->cap < nrhs) {
    for (void* p : {(void*)B->d_x, (void*)B->d_y, (void*)B->d_xh}) dev_free(p);
    B->d_x = B->d_y = B->d_xh = nullptr;
    B->cap = 0;
    B->d_x = dev_alloc<double2>((size_t)B->ncols * nrhs);
    B->d_y = dev_alloc<double2>((size_t)B->nrows * nrhs);
    B->d_xh = dev_alloc<double2>((size_t)std::max<long long>(B->xh_rows, 1) * nrhs);
    B->cap = nrhs;
    HB_CUDA(cudaDeviceSynchronize());
  }
  gather_tree_kernel<<<grid_for(B->ncols * nrhs), 256, 0, st>>>(x_nat, ldx, B->d_cperm, B->ncols, nrhs, scale, B->d_x);
  HB_CHECK_LAUNCH();
  for (size_t s = 0; s + 1 < B->step_begin.size(); ++s)
    run_tasks_fp64(B->d_tasks + B->step_begin[s], B->step_begin[s + 1] - B->step_begin[s], B->d_F, B->d_x, B->d_y,
                   B->d_xh, nrhs, st);
  scatter_tree_kernel<<<grid_for(B->nrows * nrhs), 256, 0, st>>>(B->d_y, B->d_rperm, B->nrows, nrhs, y_nat, ldy,
                                                                 accumulate);
  HB_CHECK_LAUNCH();
}

void curve_bf_info(const hb_ctx* c, int which, int* levels, int* max_rank, long long* entries) {
  const CurveBfly* B = static_cast<const CurveBfly*>(c->curve_bf[which]);
  if (!B) throw Error{HB_ERR_STATE, "no compressed curve operator (hb_curve_compress)"};
  *levels = B->L;
  *max_rank = *std::max_element(B->max_rank.begin(), B->max_rank.end());
  *entries = B->entries;
}

}  // namespace hb
