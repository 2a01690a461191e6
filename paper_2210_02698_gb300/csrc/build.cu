// build.cu - host orchestration of the HODBF / butterfly construction
// (Sec. 4.2, Sec. 4.2.1, Eq. transfer_computation, Eq. proxy,
// Eq. butterfly_factors, Eq. proxyv2v) and of the apply task plans.
//
// HODBF (Sec. 4.2, K^{v2v} item): for siblings tau1, tau2 at level l of the
// cluster tree, K(tau1, tau2) and K(tau2, tau1) are butterflies with
// L = L_v - l levels; the 2^{L_v} leaf diagonal blocks stay dense.
// Construction runs butterfly level by butterfly level for all butterflies
// at once: for every block (tau, nu) of level k the host forms the column set
// (level 0: the points of nu; k > 0: nu1_bar U nu2_bar, the skeletons of
// (p_tau, nu1), (p_tau, nu2)) and the proxy rows (Eq. proxyv2v; tau itself at
// k = L), the device evaluates all sampled blocks (entries.cu) and their
// interpolative decompositions (cpqr.cu), and the skeletons come back to the
// host for the next level.  K^L = K(tau_i, nu_bar) and the dense leaves are
// evaluated straight into the factor arena.
//
// Apply plans.  Forward (Eq. butterfly_mat): step 0 = V^0 of every butterfly
// and the dense leaves (y = D x); step t = W^t of the butterflies with L >= t
// and K^L (y += ...) of those with L = t - 1.  Adjoint (reverse order,
// conjugate transposes): step 0 = K^L^H and D^H; step u = W^{L-u+1}^H; step
// L + 1 = V^0^H (y += ...).  Each butterfly's V^0^H lands in its own step,
// so outputs of one step never overlap and the sum order is fixed.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <cmath>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "hb_internal.cuh"

namespace hb {

#ifndef HB_LEAF_NG
#define HB_LEAF_NG 8
#endif
#ifndef HB_NG
#define HB_NG 4
#endif
constexpr int LEAF_NG = HB_LEAF_NG;   // n-tiles per group of the leaf-output tasks (mixed apply)
constexpr int BLOCK_NG = HB_NG;       // n-tiles per group of the other tasks
// Cones: levels 0 .. min(L, CONE_M) of every butterfly (forward; adjoint: its
// first CONE_M + 1 steps) split into groups closed under their dependencies.
// Forward: level k block (i, j) reads level k - 1 blocks (i/2, 2j), (i/2, 2j+1),
// so the blocks with j >> (m - k) == c (m = min(L, CONE_M)) need only x and
// one another.  Adjoint: the step writing level L - d pair (p, .) reads level
// L - d + 1 blocks (2p + cc, j), so the blocks with row >> (m - d) == a do.
constexpr int CONE_M = 3;

struct BlockRec {
  int rank = 0;
  int ncols = 0;
  long long f_off = -1;
  long long xh_off = -1;
  long long xh_tile = -1;        // native layout: first padded row tile
  std::vector<long long> skel;   // tree positions, pivot order
};

struct Butterfly {
  int l, oi, si, L;
  std::vector<std::vector<BlockRec>> lev;   // lev[k][i * 2^(L-k) + j]
  std::vector<long long> kl_off;            // K^L factor offset per leaf i of T_o
};

struct Job {
  int bf, k, i, j;
  std::vector<long long> rows, cols;        // tree positions
};

namespace {

struct Segment {
  double2* ptr;
  long long count;
  long long global_off;
};

long long node_lo(const hb_ctx* c, int level, long long idx) { return c->bounds[level][idx]; }
long long node_hi(const hb_ctx* c, int level, long long idx) { return c->bounds[level][idx + 1]; }

void form_job(const hb_ctx* c, const std::vector<Butterfly>& bfs, Job& jb, std::vector<int>& stamp,
              int stamp_id) {
  const Butterfly& b = bfs[jb.bf];
  const int k = jb.k, L = b.L;
  const long long t0 = node_lo(c, b.l + k, ((long long)b.oi << k) + jb.i);
  const long long t1 = node_hi(c, b.l + k, ((long long)b.oi << k) + jb.i);
  jb.cols.clear();
  if (k == 0) {
    const long long n0 = node_lo(c, b.l + L, ((long long)b.si << L) + jb.j);
    const long long n1 = node_hi(c, b.l + L, ((long long)b.si << L) + jb.j);
    for (long long p = n0; p < n1; ++p) jb.cols.push_back(p);
  } else {
    const long long w = 1LL << (L - k + 1);
    const BlockRec& a = b.lev[k - 1][(jb.i / 2) * w + 2 * jb.j];
    const BlockRec& bb = b.lev[k - 1][(jb.i / 2) * w + 2 * jb.j + 1];
    jb.cols.insert(jb.cols.end(), a.skel.begin(), a.skel.end());
    jb.cols.insert(jb.cols.end(), bb.skel.begin(), bb.skel.end());
  }
  if (k == L) {
    jb.rows.resize((size_t)(t1 - t0));
    for (long long p = t0; p < t1; ++p) jb.rows[p - t0] = p;
  } else {
    proxy_rows(c, t0, t1, jb.cols.data(), (int)jb.cols.size(), jb.rows, stamp, stamp_id);
  }
}

}  // namespace

static void make_plans(hb_ctx* c, std::vector<Butterfly>& bfs, const std::vector<long long>& leaf_off);

void build(hb_ctx* c) {
  const auto t_begin = std::chrono::steady_clock::now();
  const int Lv = c->Lv;
  cudaStream_t st = 0;
  std::vector<Butterfly> bfs;
  for (int l = 1; l <= Lv; ++l)
    for (long long p = 0; p < (1LL << (l - 1)); ++p)
      for (int d = 0; d < 2; ++d) {
        Butterfly b;
        b.l = l;
        b.oi = (int)(2 * p + d);
        b.si = (int)(2 * p + 1 - d);
        b.L = Lv - l;
        b.lev.assign(b.L + 1, std::vector<BlockRec>((size_t)1 << b.L));
        bfs.push_back(std::move(b));
      }

  const long long ws_bytes = (long long)(c->opt.workspace_mb > 0 ? c->opt.workspace_mb : 2048) << 20;
  const long long ws_elems = ws_bytes / (long long)sizeof(double2);
  double2* d_A = dev_alloc<double2>((size_t)ws_elems);
  std::vector<Segment> segs;
  long long nfac = 0;
  long long id_blocks = 0, sampled = 0;
  int max_rank = 0;
#ifdef _OPENMP
  const int nthreads = omp_get_max_threads();
#else
  const int nthreads = 1;
#endif
  std::vector<std::vector<int>> stamps((size_t)nthreads, std::vector<int>((size_t)c->Nv, -1));
  const int Lmax = Lv - 1;
  int stamp_base = 0;

  for (int k = 0; k <= Lmax; ++k) {
    std::vector<Job> desc;
    for (int bi = 0; bi < (int)bfs.size(); ++bi) {
      const Butterfly& b = bfs[bi];
      if (b.L < k) continue;
      for (int i = 0; i < (1 << k); ++i)
        for (int j = 0; j < (1 << (b.L - k)); ++j) desc.push_back(Job{bi, k, i, j, {}, {}});
    }
    // blocks of this level kept for hb_record_id_blocks: every step-th job
    const size_t rec_step = c->id_rec_per_level > 0
                                ? std::max<size_t>(1, desc.size() / (size_t)c->id_rec_per_level)
                                : 0;
    auto recorded = [&](size_t q) {
      return rec_step && q % rec_step == 0 && q / rec_step < (size_t)c->id_rec_per_level;
    };
    const size_t JC = 8192;
    for (size_t j0 = 0; j0 < desc.size(); j0 += JC) {
      const size_t j1 = std::min(desc.size(), j0 + JC);
#pragma omp parallel for schedule(dynamic, 16)
      for (long long q = (long long)j0; q < (long long)j1; ++q) {
#ifdef _OPENMP
        const int tid = omp_get_thread_num();
#else
        const int tid = 0;
#endif
        form_job(c, bfs, desc[q], stamps[tid], stamp_base + (int)(q - j0) + 1);
      }
      stamp_base += (int)(j1 - j0) + 1;
      if (stamp_base > (1 << 30)) {
        for (auto& s : stamps) std::fill(s.begin(), s.end(), -1);
        stamp_base = 0;
      }
      // workspace chunks
      size_t q0 = j0;
      while (q0 < j1) {
        size_t q1 = q0;
        long long used = 0;
        while (q1 < j1) {
          long long e = (long long)desc[q1].rows.size() * (long long)desc[q1].cols.size();
          if (q1 > q0 && used + e > ws_elems) break;
          if (e > ws_elems) throw Error{HB_ERR_OOM, "sampled block exceeds the build workspace"};
          used += e;
          ++q1;
        }
        const int cnt = (int)(q1 - q0);
        BlockBatchHost B;
        std::vector<int> hm(cnt), hn(cnt);
        std::vector<long long> haoff(cnt), hsoff(cnt);
        long long aoff = 0, soff = 0;
        int max_n = 1;
        std::vector<std::pair<int, size_t>> rec_here;   // (t, index in c->id_recs)
        for (int t = 0; t < cnt; ++t) {
          Job& jb = desc[q0 + t];
          std::vector<long long> rn(jb.rows.size()), cn(jb.cols.size());
          for (size_t a = 0; a < rn.size(); ++a) rn[a] = c->perm[jb.rows[a]];
          for (size_t a = 0; a < cn.size(); ++a) cn[a] = c->perm[jb.cols[a]];
          if (recorded(q0 + t)) {
            IdRecord rec;
            rec.level = k;
            rec.rows = rn;
            rec.cols = cn;
            rec_here.push_back({t, c->id_recs.size()});
            c->id_recs.push_back(std::move(rec));
          }
          add_block(B, c, rn.data(), (long long)rn.size(), cn.data(), (long long)cn.size(), aoff);
          hm[t] = (int)rn.size();
          hn[t] = (int)cn.size();
          haoff[t] = aoff;
          hsoff[t] = soff;
          aoff += (long long)hm[t] * hn[t];
          soff += hn[t];
          max_n = std::max(max_n, hn[t]);
        }
        sampled += aoff;
        id_blocks += cnt;
        run_blocks(c, B, d_A, st);
        for (const auto& rh : rec_here) {   // the samples as the ID receives them
          IdRecord& rec = c->id_recs[rh.second];
          rec.A.resize((size_t)hm[rh.first] * hn[rh.first]);
          HB_CUDA(cudaMemcpyAsync(rec.A.data(), d_A + haoff[rh.first], sizeof(double2) * rec.A.size(),
                                  cudaMemcpyDeviceToHost, st));
        }
        int* d_m = upload(hm);
        int* d_n = upload(hn);
        long long* d_aoff = upload(haoff);
        long long* d_soff = upload(hsoff);
        int* d_rank = dev_alloc<int>(cnt);
        int* d_perm = dev_alloc<int>((size_t)soff);
        id_batch(cnt, d_m, d_n, d_aoff, d_A, c->opt.eps, d_rank, d_perm, d_soff, max_n, st);
        std::vector<int> hrank(cnt), hperm((size_t)soff);
        HB_CUDA(cudaMemcpyAsync(hrank.data(), d_rank, sizeof(int) * cnt, cudaMemcpyDeviceToHost, st));
        HB_CUDA(cudaMemcpyAsync(hperm.data(), d_perm, sizeof(int) * soff, cudaMemcpyDeviceToHost, st));
        HB_CUDA(cudaStreamSynchronize(st));
        for (const auto& rh : rec_here) {
          IdRecord& rec = c->id_recs[rh.second];
          rec.rank = hrank[rh.first];
          rec.piv.assign(hperm.begin() + hsoff[rh.first], hperm.begin() + hsoff[rh.first] + hn[rh.first]);
        }
        std::vector<long long> hvoff(cnt);
        long long vacc = 0;
        for (int t = 0; t < cnt; ++t) {
          Job& jb = desc[q0 + t];
          Butterfly& b = bfs[jb.bf];
          BlockRec& br = b.lev[jb.k][(size_t)jb.i * (1u << (b.L - jb.k)) + jb.j];
          const int r = hrank[t];
          br.rank = r;
          br.ncols = hn[t];
          br.f_off = nfac + vacc;
          br.skel.resize(r);
          for (int a = 0; a < r; ++a) br.skel[a] = jb.cols[hperm[hsoff[t] + a]];
          hvoff[t] = vacc;
          vacc += ((long long)r * hn[t] + 1) & ~1LL;   // blocks start at even offsets (16-byte TMA alignment)
          max_rank = std::max(max_rank, r);
        }
        double2* seg = dev_alloc<double2>((size_t)vacc);
        long long* d_voff = upload(hvoff);
        emit_v(cnt, d_m, d_n, d_aoff, d_A, d_rank, d_perm, d_soff, d_voff, 1, seg, nullptr, st);
        HB_CUDA(cudaStreamSynchronize(st));
        segs.push_back(Segment{seg, vacc, nfac});
        nfac += vacc;
        for (void* p : {(void*)d_m, (void*)d_n, (void*)d_aoff, (void*)d_soff, (void*)d_rank, (void*)d_perm,
                        (void*)d_voff})
          dev_free(p);
        for (int t = 0; t < cnt; ++t) {
          std::vector<long long>().swap(desc[q0 + t].rows);
        }
        q0 = q1;
      }
    }
  }

  // K^L blocks and dense leaves, evaluated straight into factor segments
  struct EJob {
    std::vector<long long> rows, cols;   // natural indices
    long long* target;
  };
  std::vector<EJob> ejobs;
  for (auto& b : bfs) {
    b.kl_off.assign((size_t)1 << b.L, -1);
    for (long long i = 0; i < (1LL << b.L); ++i) {
      const long long t0 = node_lo(c, b.l + b.L, ((long long)b.oi << b.L) + i);
      const long long t1 = node_hi(c, b.l + b.L, ((long long)b.oi << b.L) + i);
      EJob e;
      for (long long p = t0; p < t1; ++p) e.rows.push_back(c->perm[p]);
      for (long long p : b.lev[b.L][(size_t)i].skel) e.cols.push_back(c->perm[p]);
      e.target = &b.kl_off[(size_t)i];
      ejobs.push_back(std::move(e));
    }
  }
  std::vector<long long> leaf_off((size_t)1 << Lv, -1);
  for (long long t = 0; t < (1LL << Lv); ++t) {
    EJob e;
    for (long long p = node_lo(c, Lv, t); p < node_hi(c, Lv, t); ++p) e.rows.push_back(c->perm[p]);
    e.cols = e.rows;
    e.target = &leaf_off[(size_t)t];
    ejobs.push_back(std::move(e));
  }
  {
    size_t q0 = 0;
    while (q0 < ejobs.size()) {
      size_t q1 = q0;
      long long used = 0;
      while (q1 < ejobs.size()) {
        long long e = (long long)ejobs[q1].rows.size() * (long long)ejobs[q1].cols.size();
        if (q1 > q0 && used + e > ws_elems) break;
        used += e;
        ++q1;
      }
      BlockBatchHost B;
      long long off = 0;
      for (size_t q = q0; q < q1; ++q) {
        EJob& e = ejobs[q];
        add_block(B, c, e.rows.data(), (long long)e.rows.size(), e.cols.data(), (long long)e.cols.size(), off);
        *e.target = nfac + off;
        off += ((long long)e.rows.size() * (long long)e.cols.size() + 1) & ~1LL;
      }
      double2* seg = dev_alloc<double2>((size_t)off);
      run_blocks(c, B, seg, st);
      segs.push_back(Segment{seg, off, nfac});
      nfac += off;
      sampled += off;
      q0 = q1;
    }
  }
  dev_free(d_A);

  // pack the arenas
  c->n_factor = nfac;
  // 16 spare elements: 1D bulk copies round their size up to 16 bytes
  c->d_f64 = dev_alloc<double2>((size_t)nfac + 16);
  HB_CUDA(cudaMemset(c->d_f64, 0, sizeof(double2) * ((size_t)nfac + 16)));
  for (const Segment& s : segs) {
    if (s.count) HB_CUDA(cudaMemcpyAsync(c->d_f64 + s.global_off, s.ptr, sizeof(double2) * s.count,
                                         cudaMemcpyDeviceToDevice, st));
  }
  HB_CUDA(cudaStreamSynchronize(st));
  for (const Segment& s : segs) dev_free(s.ptr);

  // the factor index (what hb_save writes) and the apply plans
  c->bidx.clear();
  for (const Butterfly& b : bfs) {
    BflyIndex x;
    x.l = b.l;
    x.oi = b.oi;
    x.si = b.si;
    x.L = b.L;
    x.rank.assign((size_t)b.L + 1, {});
    x.f_off.assign((size_t)b.L + 1, {});
    for (int k = 0; k <= b.L; ++k)
      for (const BlockRec& br : b.lev[(size_t)k]) {
        x.rank[(size_t)k].push_back(br.rank);
        x.f_off[(size_t)k].push_back(br.f_off);
      }
    x.kl_off = b.kl_off;
    c->bidx.push_back(std::move(x));
  }
  c->leaf_off = leaf_off;
  make_plans(c, bfs, leaf_off);
  c->stats.id_blocks = id_blocks;
  c->stats.sampled_entries = sampled;
  c->stats.build_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_begin).count();
}

// Apply plans from the factor index: FP64 step lists, native arenas and the
// mixed-apply plans of both directions; statistics of the factors.
static void make_plans(hb_ctx* c, std::vector<Butterfly>& bfs, const std::vector<long long>& leaf_off) {
  const int Lv = c->Lv;
  const int Lmax = Lv - 1;
  cudaStream_t st = 0;
  int max_rank = 0;
  for (const Butterfly& b : bfs)
    for (const auto& lev : b.lev)
      for (const BlockRec& br : lev) max_rank = std::max(max_rank, br.rank);

  // xh offsets (FP64 path: packed rows; native layout: padded row tiles)
  long long xh = 0, xht = 0;
  for (auto& b : bfs)
    for (int k = 0; k <= b.L; ++k)
      for (auto& br : b.lev[k]) {
        br.xh_off = xh;
        xh += br.rank;
        br.xh_tile = xht;
        xht += (br.rank + 7) / 8;
      }
  c->xh_rows = xh;
  c->xh_tiles = xht;

  // task plans
  for (int dir = 0; dir < 2; ++dir) {
    std::vector<std::vector<Task>> steps((size_t)Lv + 1);
    // tree-position rows of each task's row node (the rows it serves; a shard
    // of the operator computes the tasks whose rows meet its own)
    std::vector<std::vector<std::pair<long long, long long>>> srows((size_t)Lv + 1);
    auto push = [&](int step, const Task& tk, long long lo, long long hi) {
      steps[(size_t)step].push_back(tk);
      srows[(size_t)step].push_back({lo, hi});
    };
    auto node_rows = [&](int level, long long idx) { return std::make_pair(node_lo(c, level, idx), node_hi(c, level, idx)); };
    auto mk = [](long long y_off, int r_out, unsigned char y_buf, unsigned char acc) {
      Task t{};
      t.y_off = y_off;
      t.r_out = r_out;
      t.y_buf = y_buf;
      t.accumulate = acc;
      t.nterm = 1;
      return t;
    };
    for (long long t = 0; t < (1LL << Lv); ++t) {
      const long long p0 = node_lo(c, Lv, t);
      const int sz = (int)(node_hi(c, Lv, t) - p0);
      Task tk = mk(p0, sz, 1, 0);
      tk.f_off[0] = leaf_off[(size_t)t];
      tk.x_off[0] = p0;
      tk.r_in[0] = sz;
      tk.x_buf = 0;
      tk.conj_t = (unsigned char)dir;
      tk.kind = 0;
      // the adjoint's outputs are columns: every shard adds its rows' share
      push(0, tk, dir == 0 ? p0 : 0, dir == 0 ? p0 + sz : c->Nv);
    }
    for (auto& b : bfs) {
      const int L = b.L;
      for (int k = 0; k <= L + 1; ++k) {
        if (dir == 0) {
          if (k == 0) {
            for (int j = 0; j < (1 << L); ++j) {
              const BlockRec& br = b.lev[0][(size_t)j];
              const long long n0 = node_lo(c, b.l + L, ((long long)b.si << L) + j);
              const int nn = (int)(node_hi(c, b.l + L, ((long long)b.si << L) + j) - n0);
              Task tk = mk(br.xh_off, br.rank, 2, 0);
              tk.f_off[0] = br.f_off;
              tk.x_buf = 0;
              tk.x_off[0] = n0;
              tk.r_in[0] = nn;
              tk.kind = 1;
              const auto rr = node_rows(b.l, b.oi);
              push(0, tk, rr.first, rr.second);
            }
          } else if (k <= L) {
            const int w = 1 << (L - k);
            for (int i = 0; i < (1 << k); ++i)
              for (int j = 0; j < w; ++j) {
                const BlockRec& br = b.lev[k][(size_t)i * w + j];
                const BlockRec& c1 = b.lev[k - 1][(size_t)(i / 2) * (2 * w) + 2 * j];
                const BlockRec& c2 = b.lev[k - 1][(size_t)(i / 2) * (2 * w) + 2 * j + 1];
                Task tk = mk(br.xh_off, br.rank, 2, 0);
                tk.f_off[0] = br.f_off;
                tk.x_buf = 2;
                tk.x_off[0] = c1.xh_off;
                tk.r_in[0] = c1.rank + c2.rank;
                tk.kind = 2;
                const auto rr = node_rows(b.l + k, ((long long)b.oi << k) + i);
                push(k, tk, rr.first, rr.second);
              }
          } else {
            for (int i = 0; i < (1 << L); ++i) {
              const BlockRec& br = b.lev[L][(size_t)i];
              const long long t0 = node_lo(c, b.l + L, ((long long)b.oi << L) + i);
              const int sz = (int)(node_hi(c, b.l + L, ((long long)b.oi << L) + i) - t0);
              Task tk = mk(t0, sz, 1, 1);
              tk.f_off[0] = b.kl_off[(size_t)i];
              tk.x_buf = 2;
              tk.x_off[0] = br.xh_off;
              tk.r_in[0] = br.rank;
              tk.kind = 3;
              push(L + 1, tk, t0, t0 + sz);
            }
          }
        } else {
          if (k == 0) {
            for (int i = 0; i < (1 << L); ++i) {
              const BlockRec& br = b.lev[L][(size_t)i];
              const long long t0 = node_lo(c, b.l + L, ((long long)b.oi << L) + i);
              const int sz = (int)(node_hi(c, b.l + L, ((long long)b.oi << L) + i) - t0);
              Task tk = mk(br.xh_off, br.rank, 2, 0);
              tk.f_off[0] = b.kl_off[(size_t)i];
              tk.x_buf = 0;
              tk.x_off[0] = t0;
              tk.r_in[0] = sz;
              tk.conj_t = 1;
              tk.kind = 3;
              push(0, tk, t0, t0 + sz);
            }
          } else if (k <= L) {
            const int t = L - k + 1;            // adjoint of W^t
            const int w = 1 << (L - t);
            for (int p = 0; p < (1 << (t - 1)); ++p)
              for (int j = 0; j < w; ++j) {
                const BlockRec& o1 = b.lev[t - 1][(size_t)p * (2 * w) + 2 * j];
                const BlockRec& o2 = b.lev[t - 1][(size_t)p * (2 * w) + 2 * j + 1];
                Task tk = mk(o1.xh_off, o1.rank + o2.rank, 2, 0);
                tk.nterm = 2;
                for (int cc = 0; cc < 2; ++cc) {
                  const BlockRec& br = b.lev[t][(size_t)(2 * p + cc) * w + j];
                  tk.f_off[cc] = br.f_off;
                  tk.x_off[cc] = br.xh_off;
                  tk.r_in[cc] = br.rank;
                }
                tk.x_buf = 2;
                tk.conj_t = 1;
                tk.kind = 2;
                const auto rr = node_rows(b.l + t - 1, ((long long)b.oi << (t - 1)) + p);
                push(k, tk, rr.first, rr.second);
              }
          } else {
            for (int j = 0; j < (1 << L); ++j) {
              const BlockRec& br = b.lev[0][(size_t)j];
              const long long n0 = node_lo(c, b.l + L, ((long long)b.si << L) + j);
              const int nn = (int)(node_hi(c, b.l + L, ((long long)b.si << L) + j) - n0);
              Task tk = mk(n0, nn, 1, 1);
              tk.f_off[0] = br.f_off;
              tk.x_buf = 2;
              tk.x_off[0] = br.xh_off;
              tk.r_in[0] = br.rank;
              tk.conj_t = 1;
              tk.kind = 1;
              push(L + 1, tk, 0, c->Nv);   // column outputs: every shard adds its share
            }
          }
        }
      }
    }
    c->tasks_h[dir].clear();
    c->task_rows[dir].clear();
    std::vector<int> begins;
    for (size_t q = 0; q < steps.size(); ++q) {
      begins.push_back((int)c->tasks_h[dir].size());
      c->tasks_h[dir].insert(c->tasks_h[dir].end(), steps[q].begin(), steps[q].end());
      c->task_rows[dir].insert(c->task_rows[dir].end(), srows[q].begin(), srows[q].end());
    }
    begins.push_back((int)c->tasks_h[dir].size());
    c->step_begin[dir] = begins;
    c->d_tasks[dir] = upload(c->tasks_h[dir]);
  }

  // native arenas and plans of the mixed apply
  {
    auto tiles8 = [](long long r) { return (r + 7) / 8; };
    const long long nleaf = 1LL << Lv;
    c->leaf_tile.assign((size_t)nleaf + 1, 0);
    for (long long t = 0; t < nleaf; ++t)
      c->leaf_tile[(size_t)t + 1] = c->leaf_tile[(size_t)t] + tiles8(node_hi(c, Lv, t) - node_lo(c, Lv, t));
    c->nv_tiles = c->leaf_tile[(size_t)nleaf];
    {
      std::vector<long long> pp((size_t)c->nv_tiles * 8, -1);
      for (long long t = 0; t < nleaf; ++t)
        for (long long p = node_lo(c, Lv, t); p < node_hi(c, Lv, t); ++p)
          pp[(size_t)(c->leaf_tile[(size_t)t] * 8 + (p - node_lo(c, Lv, t)))] = c->perm[(size_t)p];
      c->d_pperm = upload(pp);
    }
    auto leaf_size = [&](long long t) { return (int)(node_hi(c, Lv, t) - node_lo(c, Lv, t)); };
    // butterfly index of (HODBF level l, node oi as the row set / si as the column set)
    auto bf_of_o = [&](int l, long long oi) { return (int)(((1LL << (l - 1)) - 1) * 2 + (oi >> 1) * 2 + (oi & 1)); };
    auto bf_of_s = [&](int l, long long si) {
      const long long p = si >> 1;
      const int d = 1 - (int)(si & 1);   // o = 2p + d, s = 2p + 1 - d
      return (int)(((1LL << (l - 1)) - 1) * 2 + p * 2 + d);
    };
    for (int dir = 0; dir < 2; ++dir) {
      std::vector<NatBlock> nb;
      long long ntile = 0;
      // n-tiles per group: 4, and LEAF_NG for the many-term leaf outputs,
      // whose accumulation chains are long (smaller groups balance better)
      int ng = BLOCK_NG;
      // a native block of op(F) with outputs (r1 | r2) and inputs (k1 | k2)
      auto nat = [&](long long src, int ld, int r1, int r2, int k1, int k2) {
        NatBlock B{};
        B.src_off = src;
        B.tile0 = ntile;
        B.ld = ld;
        B.conj = dir;
        B.r1 = r1;
        B.r2 = r2;
        B.k1 = k1;
        B.k2 = k2;
        B.ng = ng;
        ntile += (tiles8(r1) + tiles8(r2)) * (tiles8(k1) + tiles8(k2));
        nb.push_back(B);
        return B.tile0;
      };
      auto term = [](long long f_tile, long long x_tile, long long ks, int x_buf) {
        NatTerm tm{};
        tm.f_tile = f_tile;
        tm.x_tile = x_tile;
        tm.ks = (int)ks;
        tm.x_buf = x_buf;
        return tm;
      };
      std::vector<NatTask> nt;
      // first cone id of every butterfly: 2^(L - min(L, CONE_M)) cones each
      std::vector<long long> cone_base(bfs.size() + 1, 0);
      for (size_t bi = 0; bi < bfs.size(); ++bi)
        cone_base[bi + 1] = cone_base[bi] + (1LL << (bfs[bi].L - std::min(bfs[bi].L, CONE_M)));
      auto task = [&](long long y_tile, long long ntl, int depth, int y_buf) {
        NatTask t;
        t.y_tile = y_tile;
        t.nt = (int)ntl;
        t.depth = depth;
        t.y_buf = y_buf;
        t.ng = ng;
        return t;
      };
      if (dir == 0) {
        // depth k: V^0 (k = 0) and W^k of every butterfly with L >= k
        for (int k = 0; k <= Lmax; ++k)
          for (size_t bi = 0; bi < bfs.size(); ++bi) {
            const Butterfly& b = bfs[bi];
            if (b.L < k) continue;
            const int w = 1 << (b.L - k);
            for (int i = 0; i < (1 << k); ++i)
              for (int j = 0; j < w; ++j) {
                const BlockRec& br = b.lev[k][(size_t)i * w + j];
                NatTask t = task(br.xh_tile, tiles8(br.rank), k, 2);
                t.tc_out = (k == b.L);   // lev[L] is read only by the leaf outputs (K^L)
                t.row_lo = node_lo(c, b.l + k, ((long long)b.oi << k) + i);
                t.row_hi = node_hi(c, b.l + k, ((long long)b.oi << k) + i);
                {
                  const int m = std::min(b.L, CONE_M);
                  if (k <= m) {
                    t.cone = cone_base[bi] + (j >> (m - k));
                    t.cone_level = k;
                  }
                }
                if (k == 0) {
                  const long long leaf = ((long long)b.si << b.L) + j;
                  const int nn = leaf_size(leaf);
                  t.terms.push_back(term(nat(br.f_off, br.rank, br.rank, 0, nn, 0), c->leaf_tile[(size_t)leaf],
                                         tiles8(nn), 0));
                } else {
                  const size_t q1 = (size_t)(i / 2) * (2 * w) + 2 * j;
                  const BlockRec& c1 = b.lev[k - 1][q1];
                  const BlockRec& c2 = b.lev[k - 1][q1 + 1];
                  t.terms.push_back(term(nat(br.f_off, br.rank, br.rank, 0, c1.rank, c2.rank), c1.xh_tile,
                                         tiles8(c1.rank) + tiles8(c2.rank), 2));
                }
                nt.push_back(std::move(t));
              }
          }
        // last depth: y(leaf t) = D_t x(t) + sum over levels of K^L x_hat
        ng = LEAF_NG;
        for (long long t = 0; t < nleaf; ++t) {
          const int sz = leaf_size(t);
          NatTask o = task(c->leaf_tile[(size_t)t], tiles8(sz), Lmax + 1, 1);
          o.row_lo = node_lo(c, Lv, t);
          o.row_hi = node_hi(c, Lv, t);
          o.terms.push_back(term(nat(leaf_off[(size_t)t], sz, sz, 0, sz, 0), c->leaf_tile[(size_t)t], tiles8(sz), 0));
          // terms in the order their inputs are produced (HODBF level Lv,
          // whose K^L input is written at depth 0, first): a dataflow launch
          // can start the leaf outputs before the deepest butterflies finish
          for (int l = Lv; l >= 1; --l) {
            const long long oi = t >> (Lv - l);
            const Butterfly& b = bfs[(size_t)bf_of_o(l, oi)];
            const long long i = t - (oi << b.L);
            const BlockRec& br = b.lev[b.L][(size_t)i];
            o.terms.push_back(term(nat(b.kl_off[(size_t)i], sz, sz, 0, br.rank, 0), br.xh_tile, tiles8(br.rank), 2));
          }
          nt.push_back(std::move(o));
        }
      } else {
        // depth 0: K^L^H
        for (size_t bi = 0; bi < bfs.size(); ++bi) {
          const Butterfly& b = bfs[bi];
          for (int i = 0; i < (1 << b.L); ++i) {
            const BlockRec& br = b.lev[b.L][(size_t)i];
            const long long leaf = ((long long)b.oi << b.L) + i;
            const int sz = leaf_size(leaf);
            NatTask t = task(br.xh_tile, tiles8(br.rank), 0, 2);
            t.tc_out = (b.L == 0);   // lev[0] is read only by the leaf outputs (V^0^H)
            t.row_lo = node_lo(c, b.l + b.L, ((long long)b.oi << b.L) + i);
            t.row_hi = node_hi(c, b.l + b.L, ((long long)b.oi << b.L) + i);
            t.cone = cone_base[bi] + (i >> std::min(b.L, CONE_M));
            t.cone_level = 0;
            t.terms.push_back(term(nat(b.kl_off[(size_t)i], sz, br.rank, 0, sz, 0), c->leaf_tile[(size_t)leaf],
                                   tiles8(sz), 0));
            nt.push_back(std::move(t));
          }
        }
        // depth d: W^{L-d+1}^H, writing the pair of level L-d blocks
        for (int d = 1; d <= Lmax; ++d)
          for (size_t bi = 0; bi < bfs.size(); ++bi) {
            const Butterfly& b = bfs[bi];
            if (b.L < d) continue;
            const int tl = b.L - d + 1;
            const int w = 1 << (b.L - tl);
            for (int p = 0; p < (1 << (tl - 1)); ++p)
              for (int j = 0; j < w; ++j) {
                const size_t q1 = (size_t)p * (2 * w) + 2 * j;
                const BlockRec& o1 = b.lev[tl - 1][q1];
                const BlockRec& o2 = b.lev[tl - 1][q1 + 1];
                NatTask t = task(o1.xh_tile, tiles8(o1.rank) + tiles8(o2.rank), d, 2);
                t.tc_out = (tl == 1);   // writes lev[0], read only by the leaf outputs
                t.row_lo = node_lo(c, b.l + tl - 1, ((long long)b.oi << (tl - 1)) + p);
                t.row_hi = node_hi(c, b.l + tl - 1, ((long long)b.oi << (tl - 1)) + p);
                {
                  const int m = std::min(b.L, CONE_M);
                  if (d <= m) {
                    t.cone = cone_base[bi] + (p >> (m - d));
                    t.cone_level = d;
                  }
                }
                for (int cc = 0; cc < 2; ++cc) {
                  const BlockRec& br = b.lev[tl][(size_t)(2 * p + cc) * w + j];
                  t.terms.push_back(term(nat(br.f_off, br.rank, o1.rank, o2.rank, br.rank, 0), br.xh_tile,
                                         tiles8(br.rank), 2));
                }
                nt.push_back(std::move(t));
              }
          }
        // last depth: y(leaf t) = D_t^H x(t) + sum over levels of V^0^H x_hat
        ng = LEAF_NG;
        for (long long t = 0; t < nleaf; ++t) {
          const int sz = leaf_size(t);
          NatTask o = task(c->leaf_tile[(size_t)t], tiles8(sz), Lmax + 1, 1);
          o.row_lo = 0;   // column outputs: every shard adds its rows' share
          o.row_hi = c->Nv;
          o.terms.push_back(term(nat(leaf_off[(size_t)t], sz, sz, 0, sz, 0), c->leaf_tile[(size_t)t], tiles8(sz), 0));
          for (int l = Lv; l >= 1; --l) {   // inputs in the order they are produced (as above)
            const long long si = t >> (Lv - l);
            const Butterfly& b = bfs[(size_t)bf_of_s(l, si)];
            const long long j = t - (si << b.L);
            const BlockRec& br = b.lev[0][(size_t)j];
            o.terms.push_back(term(nat(br.f_off, br.rank, sz, 0, br.rank, 0), br.xh_tile, tiles8(br.rank), 2));
          }
          nt.push_back(std::move(o));
        }
      }
      c->nat_tiles[dir] = ntile;
      c->d_nat[dir] = dev_alloc<uint4>((size_t)std::max<long long>(ntile, 1) * 32);
      nat_convert(c->d_f64, nb, c->d_nat[dir], st);
      HB_CUDA(cudaStreamSynchronize(st));
      // the leaf outputs again, for the tensor-core leaf kernel: chains of up
      // to 64 outputs, each term's block in the operand layout (4 KB per 8
      // inputs); the terms and blocks are those of the native tasks above
      {
        std::vector<TcBlock> tb;
        std::vector<TcChainHost> tch;
        long long units = 0;
        std::map<long long, const NatBlock*> by_tile;
        for (const NatBlock& B : nb) by_tile[B.tile0] = &B;
        for (const NatTask& L : nt) {
          if (L.y_buf != 1) continue;
          const int rows = 8 * L.nt;
          for (int o0 = 0; o0 < rows; o0 += 64) {
            TcChainHost ch;
            ch.y_tile = L.y_tile + o0 / 8;
            ch.nout = std::min(64, rows - o0);
            for (const NatTerm& tm : L.terms) {
              const NatBlock& B = *by_tile.at(tm.f_tile);
              TcBlock t{};
              t.src_off = B.src_off;
              t.unit0 = units;
              t.ld = B.ld;
              t.conj = B.conj;
              t.o0 = o0;
              t.nout = std::max(0, std::min(64, B.r1 - o0));
              t.k = B.k1;
              tb.push_back(t);
              ch.terms.push_back(TcTerm{units, tm.x_tile, tm.ks, tm.x_buf});
              units += tm.ks;
            }
            tch.push_back(std::move(ch));
          }
        }
        c->d_tc[dir] = dev_alloc<uint4>((size_t)std::max<long long>(units, 1) * 256);
        tc_convert(c->d_f64, tb, c->d_tc[dir], st);
        c->tc_plan[dir] = tc_plan_build(std::move(tch));
      }
      flow_plan_build(nt, &c->flow_plan[dir]);
    }
  }
  HB_CUDA(cudaDeviceSynchronize());

  c->max_rank = max_rank;
  c->stats.max_rank = max_rank;
  c->stats.factor_entries = c->n_factor;
  c->stats.factor_bytes_fp64 = c->n_factor * (long long)sizeof(double2);
  c->stats.factor_bytes_mixed = c->nat_tiles[0] * 512;
  c->stats.skeleton_rows = c->xh_rows;
  // mixed-precision apply of up to 32 right-hand sides in the default
  // shape: the gather and one step launch per dependency depth (the last one
  // writes u)
  c->stats.apply_launches = 1 + flow_plan_depths(c->flow_plan[0]);
}

// hb_load: the apply plans of a factor index read from a file (the arena
// c->d_f64, c->bidx and c->leaf_off are in place).
void plans_from_index(hb_ctx* c) {
  std::vector<Butterfly> bfs;
  for (const BflyIndex& x : c->bidx) {
    Butterfly b;
    b.l = x.l;
    b.oi = x.oi;
    b.si = x.si;
    b.L = x.L;
    b.lev.assign((size_t)x.L + 1, std::vector<BlockRec>((size_t)1 << x.L));
    for (int k = 0; k <= x.L; ++k)
      for (size_t j = 0; j < b.lev[(size_t)k].size(); ++j) {
        b.lev[(size_t)k][j].rank = x.rank[(size_t)k][j];
        b.lev[(size_t)k][j].f_off = x.f_off[(size_t)k][j];
      }
    b.kl_off = x.kl_off;
    bfs.push_back(std::move(b));
  }
  make_plans(c, bfs, c->leaf_off);
}

}  // namespace hb
