// api.cu - the extern "C" entry points declared in include/hb.h.  Argument
// checks, error capture (no exception crosses the ABI) and dispatch to the
// kernels of entries.cu, cpqr.cu, build.cu and apply.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "hb_internal.cuh"

// ------------------------------------------------- allocation registry ----
namespace {
struct Registry {
  std::mutex m;
  std::unordered_map<void*, size_t> bytes;
  long long live = 0;
  long long cap = 0;   // 0: no cap
};
Registry& registry() {
  static Registry* r = new Registry();   // never destroyed: frees may come late
  return *r;
}
thread_local std::vector<void*>* g_build_allocs = nullptr;
}  // namespace

namespace hb {

void* registry_alloc(size_t bytes) {
  Registry& r = registry();
  {
    std::lock_guard<std::mutex> lock(r.m);
    if (r.cap > 0 && r.live + (long long)bytes > r.cap)
      throw Error{HB_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes exceeds the cap of " +
                                  std::to_string(r.cap) + " bytes (hb_device_alloc_cap)"};
  }
  void* p = nullptr;
  const cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error{e == cudaErrorMemoryAllocation ? HB_ERR_OOM : HB_ERR_CUDA,
                "cudaMalloc(" + std::to_string(bytes) + " bytes): " + cudaGetErrorString(e)};
  }
  {
    std::lock_guard<std::mutex> lock(r.m);
    r.bytes[p] = bytes;
    r.live += (long long)bytes;
  }
  if (g_build_allocs) g_build_allocs->push_back(p);
  return p;
}

void registry_free(void* p) {
  Registry& r = registry();
  {
    std::lock_guard<std::mutex> lock(r.m);
    auto it = r.bytes.find(p);
    if (it != r.bytes.end()) {
      r.live -= (long long)it->second;
      r.bytes.erase(it);
    }
  }
  if (g_build_allocs) {
    auto it = std::find(g_build_allocs->begin(), g_build_allocs->end(), p);
    if (it != g_build_allocs->end()) g_build_allocs->erase(it);
  }
  cudaFree(p);
}

BuildAllocs::BuildAllocs() { g_build_allocs = new std::vector<void*>(); }

BuildAllocs::~BuildAllocs() {
  delete g_build_allocs;
  g_build_allocs = nullptr;
}

void BuildAllocs::free_all() {
  std::vector<void*> v;
  v.swap(*g_build_allocs);
  for (void* p : v) registry_free(p);
}

}  // namespace hb

namespace {

thread_local std::string g_err;   // errors of calls without a handle

template <class F>
hb_status guarded(hb_ctx* c, F&& f) {
  try {
    f();
    return HB_OK;
  } catch (const hb::Error& e) {
    (c ? c->err : g_err) = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    (c ? c->err : g_err) = "host allocation failed";
    return HB_ERR_OOM;
  } catch (...) {
    (c ? c->err : g_err) = "unexpected C++ exception";
    return HB_ERR_CUDA;
  }
}

void free_all(hb_ctx* c) {
  for (void* p : {(void*)c->d_nodes, (void*)c->d_tab, (void*)c->d_LX, (void*)c->d_LZ, (void*)c->d_H[0],
                  (void*)c->d_H[1], (void*)c->d_ncell, (void*)c->d_self, (void*)c->d_perm, (void*)c->d_f64,
                  (void*)c->d_nat[0], (void*)c->d_nat[1], (void*)c->d_pperm, (void*)c->d_mx,
                  (void*)c->d_mxh, c->d_x, c->d_y, (void*)c->d_dense_part, (void*)c->d_flags, (void*)c->d_mx_tc,
                  (void*)c->d_tc[0], (void*)c->d_tc[1]})
    hb::dev_free(p);
  hb::dev_free(c->d_xh);
  hb::dev_free(c->d_tasks[0]);
  hb::dev_free(c->d_tasks[1]);
  hb::flow_plan_free(c->flow_plan[0]);
  hb::flow_plan_free(c->flow_plan[1]);
  hb::tc_plan_free(c->tc_plan[0]);
  hb::tc_plan_free(c->tc_plan[1]);
  hb::shard_cache_free(c);
  hb::curve_free(c);
  if (c->h_err) cudaFreeHost(c->h_err);
}

// Everything hb_build made - factors, apply plans, recorded ID blocks, row
// shards and the apply scratch sized by the ranks - freed, so that the
// handle can be built again; the tables, the cluster tree, the options and
// the error word stay.
void release_build(hb_ctx* c) {
  HB_CUDA(cudaDeviceSynchronize());
  for (void* p : {(void*)c->d_f64, (void*)c->d_nat[0], (void*)c->d_nat[1], (void*)c->d_tc[0], (void*)c->d_tc[1],
                  (void*)c->d_pperm, (void*)c->d_mx, (void*)c->d_mxh, (void*)c->d_mx_tc, (void*)c->d_flags,
                  c->d_x, c->d_y, c->d_xh, (void*)c->d_tasks[0], (void*)c->d_tasks[1]})
    hb::dev_free(p);
  c->d_f64 = nullptr;
  c->d_nat[0] = c->d_nat[1] = c->d_tc[0] = c->d_tc[1] = nullptr;
  c->d_pperm = nullptr;
  c->d_mx = c->d_mxh = c->d_mx_tc = nullptr;
  c->d_flags = c->d_epoch = nullptr;
  c->d_x = c->d_y = c->d_xh = nullptr;
  c->cap_rhs = 0;
  c->d_tasks[0] = c->d_tasks[1] = nullptr;
  for (int d = 0; d < 2; ++d) {
    hb::flow_plan_free(c->flow_plan[d]);
    c->flow_plan[d] = nullptr;
    hb::tc_plan_free(c->tc_plan[d]);
    c->tc_plan[d] = nullptr;
    c->step_begin[d].clear();
    c->tasks_h[d].clear();
    c->task_rows[d].clear();
    c->nat_tiles[d] = 0;
  }
  hb::shard_cache_free(c);
  c->bidx.clear();
  c->leaf_off.clear();
  c->leaf_tile.clear();
  c->id_recs.clear();
  c->n_factor = 0;
  c->nv_tiles = c->xh_tiles = c->xh_rows = 0;
  c->max_rank = 0;
  const long long nv = c->stats.n_v;
  const int lv = c->stats.levels;
  c->stats = hb_stats{};
  c->stats.n_v = nv;
  c->stats.levels = lv;
  c->built = false;
}

void check_vec_args(hb_ctx* c, const void* a, const void* b, int nrhs) {
  if (!c) throw hb::arg_error("null handle");
  if (!a || !b) throw hb::arg_error("null vector pointer");
  if (a == b) throw hb::arg_error("input and output must not alias");
  if (nrhs < 1 || nrhs > 1024) throw hb::arg_error("nrhs=%d outside [1, 1024]", nrhs);
}

}  // namespace

extern "C" {

}  // extern "C"

namespace hb {
// Validate the inputs, copy them, upload the tables and build the cluster
// tree; throws hb::Error.  Shared by hb_create and hb_load.
hb_ctx* create_ctx(const hb_grid* grid, const hb_tables* tables, double omega, const hb_options* opts) {
  if (!grid || !tables || !opts) throw hb::arg_error("null argument");
  if (grid->nx < 1 || grid->ny < 1 || !(grid->h > 0)) throw hb::arg_error("bad grid");
  if ((long long)grid->nx * grid->ny > (1LL << 31)) throw hb::arg_error("grid too large");
  if (tables->n_I < 2 || tables->n_I > 16)
    throw hb::Error{tables->n_I < 2 ? HB_ERR_ARG : HB_ERR_UNSUPPORTED, "n_I must be in [2, 16]"};
  if (!tables->nodes_x || !tables->nodes_y || !tables->tau2 || !tables->v0 || !tables->v1 || !tables->n_cells)
    throw hb::arg_error("null table pointer");
  if (!(omega > 0) || !std::isfinite(omega)) throw hb::arg_error("omega must be positive");
  if (!(opts->eps > 0) || opts->leaf < 1 || !(opts->chi > 0) || !(opts->nbr_radius_h >= 0))
    throw hb::arg_error("bad options (eps > 0, leaf >= 1, chi > 0, radius >= 0)");
  if (opts->precision != HB_FP64 && opts->precision != HB_MIXED_BF16X3)
    throw hb::arg_error("unknown precision %d", opts->precision);
  if (opts->autotune < 0 || opts->autotune > 6) throw hb::arg_error("autotune must be 0 .. 6");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    throw hb::Error{HB_ERR_CUDA, "no CUDA device"};
  }
  hb_ctx* c = new hb_ctx();
  try {
    c->nx = grid->nx;
    c->ny = grid->ny;
    c->Nv = (long long)grid->nx * grid->ny;
    c->x0 = grid->x0;
    c->y0 = grid->y0;
    c->h = grid->h;
    c->omega = omega;
    c->nI = tables->n_I;
    c->NI = tables->n_I * tables->n_I;
    c->opt = *opts;
    c->nodes_x.assign(tables->nodes_x, tables->nodes_x + c->nI);
    c->nodes_y.assign(tables->nodes_y, tables->nodes_y + c->nI);
    const double* src[3] = {tables->tau2, tables->v0, tables->v1};
    for (int q = 0; q < 3; ++q) c->tab[q].assign(src[q], src[q] + (size_t)c->NI * c->NI);
    c->n_cells.assign(tables->n_cells, tables->n_cells + c->Nv);
    for (double v : c->n_cells)
      if (!(v > 0) || !std::isfinite(v)) throw hb::arg_error("n_cells must be positive");
    hb::setup_tables(c);
    hb::tree_build(c);
    c->stats.n_v = c->Nv;
    c->stats.levels = c->Lv;
  } catch (...) {
    free_all(c);
    delete c;
    throw;
  }
  return c;
}
}  // namespace hb

extern "C" {

hb_status hb_create(const hb_grid* grid, const hb_tables* tables, double omega, const hb_options* opts,
                    hb_handle* out) {
  hb_ctx* c = nullptr;
  hb_status st = guarded(nullptr, [&] {
    if (!out) throw hb::arg_error("null argument");
    *out = nullptr;
    c = hb::create_ctx(grid, tables, omega, opts);
  });
  if (st != HB_OK) return st;
  *out = c;
  return HB_OK;
}

hb_status hb_save(hb_handle h, const char* path) {
  return guarded(h, [&] {
    if (!h || !path) throw hb::arg_error("null argument");
    if (!h->built) throw hb::Error{HB_ERR_STATE, "hb_save before hb_build"};
    hb::save_file(h, path);
  });
}

hb_status hb_load(const char* path, hb_handle* out) {
  hb_ctx* c = nullptr;
  hb_status st = guarded(nullptr, [&] {
    if (!path || !out) throw hb::arg_error("null argument");
    *out = nullptr;
    c = hb::load_file(path, &hb::create_ctx);
  });
  if (st != HB_OK) return st;
  *out = c;
  return HB_OK;
}

hb_status hb_build(hb_handle h) {
  return guarded(h, [&] {
    if (!h) throw hb::arg_error("null handle");
    if (h->built) throw hb::Error{HB_ERR_STATE, "already built"};
    hb::BuildAllocs allocs;
    hb::NvtxRange nr("hb_build");
    try {
      hb::build(h);
    } catch (...) {
      // a failed build frees what it allocated and leaves the handle unbuilt
      cudaDeviceSynchronize();
      cudaGetLastError();
      allocs.free_all();
      h->d_f64 = nullptr;
      h->d_tasks[0] = h->d_tasks[1] = nullptr;
      h->d_nat[0] = h->d_nat[1] = nullptr;
      h->d_tc[0] = h->d_tc[1] = nullptr;
      h->d_pperm = nullptr;
      for (int d = 0; d < 2; ++d) {
        hb::flow_plan_free(h->flow_plan[d]);
        h->flow_plan[d] = nullptr;
        hb::tc_plan_free(h->tc_plan[d]);
        h->tc_plan[d] = nullptr;
      }
      h->id_recs.clear();
      throw;
    }
    h->built = true;
  });
}

hb_status hb_set_omega(hb_handle h, double omega) {
  return guarded(h, [&] {
    if (!h) throw hb::arg_error("null handle");
    if (!(omega > 0) || !std::isfinite(omega)) throw hb::arg_error("omega must be positive");
    // the curve, if any, is assembled again at the new frequency
    std::vector<double> cen, len, nseg;
    const long long ns = h->ns;
    if (ns > 0) {
      std::vector<double2> c2((size_t)ns);
      len.resize((size_t)ns);
      nseg.resize((size_t)ns);
      HB_CUDA(cudaMemcpy(c2.data(), h->d_seg, sizeof(double2) * ns, cudaMemcpyDeviceToHost));
      HB_CUDA(cudaMemcpy(len.data(), h->d_segw, sizeof(double) * ns, cudaMemcpyDeviceToHost));
      HB_CUDA(cudaMemcpy(nseg.data(), h->d_segn, sizeof(double) * ns, cudaMemcpyDeviceToHost));
      for (const double2& v : c2) {
        cen.push_back(v.x);
        cen.push_back(v.y);
      }
    }
    release_build(h);
    hb::curve_free(h);
    h->omega = omega;
    hb::compute_self(h);
    if (ns > 0) hb::curve_set(h, cen.data(), len.data(), nseg.data(), ns);
  });
}

hb_status hb_curve_compress(hb_handle h, int leaf_s) {
  return guarded(h, [&] {
    if (!h) throw hb::arg_error("null handle");
    hb::NvtxRange nr("hb_curve_compress");
    hb::curve_compress(h, leaf_s);
  });
}

hb_status hb_curve_info(hb_handle h, int which, int* levels, int* max_rank, long long* entries) {
  return guarded(h, [&] {
    if (!h || !levels || !max_rank || !entries) throw hb::arg_error("null argument");
    if (which != 0 && which != 1) throw hb::arg_error("which must be 0 (K^{v2s}) or 1 (K^{s2v})");
    hb::curve_bf_info(h, which, levels, max_rank, entries);
  });
}

hb_status hb_sweep_taylor(int ns, const double* s2, double* taylor) {
  return guarded(nullptr, [&] {
    if (ns < 0) throw hb::arg_error("ns must be >= 0");
    if (ns > 0 && (!s2 || !taylor)) throw hb::arg_error("null argument");
    for (int k = 0; k < ns; ++k) hb::sweep_taylor_one(s2 + (size_t)k * 15, taylor + (size_t)k * 46);
  });
}

hb_status hb_sweep_tables(int M, double lo, double h, int w0, int w1, int roi0, int roi1, const double* n_mesh,
                          int NI, const double* px, const double* pz, int ns, const int* src, const double* taylor,
                          int max_iter, double tol, double* tau2, double* v0, double* v1, double* info) {
  return guarded(nullptr, [&] {
    hb::NvtxRange nr("hb_sweep_tables");
    hb::sweep_tables(M, lo, h, w0, w1, roi0, roi1, n_mesh, NI, px, pz, ns, src, taylor, max_iter, tol, tau2, v0, v1,
                     info);
  });
}

hb_status hb_record_id_blocks(hb_handle h, int per_level) {
  return guarded(h, [&] {
    if (!h) throw hb::arg_error("null handle");
    if (per_level < 0) throw hb::arg_error("per_level must be >= 0");
    if (h->built) throw hb::Error{HB_ERR_STATE, "hb_record_id_blocks must come before hb_build"};
    h->id_rec_per_level = per_level;
    h->id_recs.clear();
  });
}

hb_status hb_recorded_id_count(hb_handle h, int* count) {
  return guarded(h, [&] {
    if (!h || !count) throw hb::arg_error("null argument");
    *count = (int)h->id_recs.size();
  });
}

hb_status hb_recorded_id_block(hb_handle h, int index, int* level, int* m, int* n, long long* rows,
                               long long* cols, void* A, int* rank, int* pivots) {
  return guarded(h, [&] {
    if (!h || !level || !m || !n || !rank) throw hb::arg_error("null argument");
    if (index < 0 || index >= (int)h->id_recs.size())
      throw hb::arg_error("record %d out of range (%d kept)", index, (int)h->id_recs.size());
    const hb::IdRecord& r = h->id_recs[(size_t)index];
    *level = r.level;
    *m = (int)r.rows.size();
    *n = (int)r.cols.size();
    *rank = r.rank;
    if (rows) std::copy(r.rows.begin(), r.rows.end(), rows);
    if (cols) std::copy(r.cols.begin(), r.cols.end(), cols);
    if (A) std::copy(r.A.begin(), r.A.end(), static_cast<double2*>(A));
    if (pivots) std::copy(r.piv.begin(), r.piv.end(), pivots);
  });
}

hb_status hb_launch_shape(hb_handle h, int adjoint, int mtiles, int* mode, int* item_bytes, int* stages,
                          int* pub_batch, int* slack, double* tuned_ms, int* candidates) {
  return guarded(h, [&] {
    if (!h || !mode || !item_bytes || !stages || !pub_batch || !slack || !tuned_ms || !candidates)
      throw hb::arg_error("null argument");
    if (adjoint != 0 && adjoint != 1) throw hb::arg_error("adjoint must be 0 or 1");
    if (mtiles != 1 && mtiles != 2) throw hb::arg_error("mtiles must be 1 or 2");
    if (!h->built || !h->flow_plan[adjoint]) throw hb::Error{HB_ERR_STATE, "not built"};
    hb::flow_shape(h->flow_plan[adjoint], mtiles, mode, item_bytes, stages, pub_batch, slack, tuned_ms, candidates);
  });
}

hb_status hb_device_alloc_cap(long long cap_bytes, long long* live_bytes) {
  return guarded(nullptr, [&] {
    Registry& r = registry();
    std::lock_guard<std::mutex> lock(r.m);
    if (cap_bytes >= 0) r.cap = cap_bytes;
    if (live_bytes) *live_bytes = r.live;
  });
}

hb_status hb_apply(hb_handle h, const void* s, void* u, int nrhs, void* stream) {
  return guarded(h, [&] {
    check_vec_args(h, s, u, nrhs);
    if (!h->built) throw hb::Error{HB_ERR_STATE, "hb_apply before hb_build"};
    hb::apply_bf(h, (const double2*)s, (double2*)u, nrhs, 0, h->opt.precision, (cudaStream_t)stream);
  });
}

hb_status hb_apply_adjoint(hb_handle h, const void* u, void* s, int nrhs, void* stream) {
  return guarded(h, [&] {
    check_vec_args(h, u, s, nrhs);
    if (!h->built) throw hb::Error{HB_ERR_STATE, "hb_apply_adjoint before hb_build"};
    hb::apply_bf(h, (const double2*)u, (double2*)s, nrhs, 1, h->opt.precision, (cudaStream_t)stream);
  });
}

hb_status hb_shard_rows(hb_handle h, int nranks, int rank, long long* lo, long long* hi) {
  return guarded(h, [&] {
    if (!h || !lo || !hi) throw hb::arg_error("null argument");
    hb::shard_rows(h, nranks, rank, lo, hi);
  });
}

hb_status hb_apply_shard(hb_handle h, const void* s, void* u, int nrhs, int nranks, int rank, void* stream) {
  return guarded(h, [&] {
    check_vec_args(h, s, u, nrhs);
    if (!h->built) throw hb::Error{HB_ERR_STATE, "hb_apply_shard before hb_build"};
    hb::apply_bf_shard(h, (const double2*)s, (double2*)u, nrhs, 0, h->opt.precision, nranks, rank,
                       (cudaStream_t)stream);
  });
}

hb_status hb_apply_shard_adjoint(hb_handle h, const void* u, void* s, int nrhs, int nranks, int rank, void* stream) {
  return guarded(h, [&] {
    check_vec_args(h, u, s, nrhs);
    if (!h->built) throw hb::Error{HB_ERR_STATE, "hb_apply_shard_adjoint before hb_build"};
    hb::apply_bf_shard(h, (const double2*)u, (double2*)s, nrhs, 1, h->opt.precision, nranks, rank,
                       (cudaStream_t)stream);
  });
}

hb_status hb_set_precision(hb_handle h, int precision) {
  return guarded(h, [&] {
    if (!h) throw hb::arg_error("null handle");
    if (precision != HB_FP64 && precision != HB_MIXED_BF16X3) throw hb::arg_error("unknown precision");
    h->opt.precision = precision;
  });
}

hb_status hb_set_wait_selftest(hb_handle h, int on) {
  return guarded(h, [&] {
    if (!h) throw hb::arg_error("null handle");
    h->wait_selftest = on != 0;
  });
}

hb_status hb_apply_dense(hb_handle h, const void* s, void* u, int nrhs, void* stream) {
  return guarded(h, [&] {
    check_vec_args(h, s, u, nrhs);
    hb::dense_apply(h, (const double2*)s, (double2*)u, nrhs, 0, (cudaStream_t)stream);
  });
}

hb_status hb_apply_dense_adjoint(hb_handle h, const void* u, void* s, int nrhs, void* stream) {
  return guarded(h, [&] {
    check_vec_args(h, u, s, nrhs);
    hb::dense_apply(h, (const double2*)u, (double2*)s, nrhs, 1, (cudaStream_t)stream);
  });
}

hb_status hb_entries(hb_handle h, const long long* rows, int m, const long long* cols, int n, void* out,
                     void* stream) {
  return guarded(h, [&] {
    if (!h || !rows || !cols || !out) throw hb::arg_error("null argument");
    if (m < 1 || n < 1) throw hb::arg_error("m, n must be >= 1");
    for (int i = 0; i < m; ++i)
      if (rows[i] < 0 || rows[i] >= h->Nv) throw hb::arg_error("row index %lld out of range", rows[i]);
    for (int j = 0; j < n; ++j)
      if (cols[j] < 0 || cols[j] >= h->Nv) throw hb::arg_error("column index %lld out of range", cols[j]);
    hb::eval_entries(h, rows, m, cols, n, (double2*)out, (cudaStream_t)stream);
  });
}

hb_status hb_rank_profile(hb_handle h, int* max_rank, double* mean_rank) {
  return guarded(h, [&] {
    if (!h || !max_rank || !mean_rank) throw hb::arg_error("null argument");
    if (!h->built) throw hb::Error{HB_ERR_STATE, "hb_rank_profile before hb_build"};
    const int n = h->Lv + 1;
    std::vector<long long> sum((size_t)n * n, 0), cnt((size_t)n * n, 0);
    std::fill(max_rank, max_rank + (size_t)n * n, 0);
    for (const hb::BflyIndex& b : h->bidx) {
      if (b.l < 1 || b.l > h->Lv || b.L < 0 || b.l + b.L > h->Lv || (int)b.rank.size() != b.L + 1)
        throw hb::Error{HB_ERR_STATE, "inconsistent factor index"};
      for (int k = 0; k <= b.L; ++k)
        for (int r : b.rank[(size_t)k]) {
          const size_t at = (size_t)b.l * n + k;
          max_rank[at] = std::max(max_rank[at], r);
          sum[at] += r;
          cnt[at] += 1;
        }
    }
    for (size_t i = 0; i < (size_t)n * n; ++i) mean_rank[i] = cnt[i] ? (double)sum[i] / (double)cnt[i] : 0.0;
  });
}

hb_status hb_curve_set(hb_handle h, const double* centers, const double* lengths, const double* n_seg,
                       long long ns) {
  return guarded(h, [&] {
    if (!h) throw hb::arg_error("null handle");
    hb::curve_set(h, centers, lengths, n_seg, ns);
  });
}

hb_status hb_curve_operators(hb_handle h, void* k_s2s, void* k_v2s, void* k_s2v, void* stream) {
  return guarded(h, [&] {
    if (!h) throw hb::arg_error("null handle");
    hb::curve_operators(h, (double2*)k_s2s, (double2*)k_v2s, (double2*)k_s2v, (cudaStream_t)stream);
  });
}

hb_status hb_apply_inclusion(hb_handle h, const void* s, void* u, int nrhs, int v2v_dense, void* stream) {
  return guarded(h, [&] {
    check_vec_args(h, s, u, nrhs);
    hb::apply_inclusion(h, (const double2*)s, (double2*)u, nrhs, v2v_dense, (cudaStream_t)stream);
  });
}

hb_status hb_id_batch(int count, const int* m, const int* n, const long long* a_off, void* A, double eps,
                      int* rank, int* skel, void* V) {
  return guarded(nullptr, [&] {
    if (count < 0 || (count > 0 && (!m || !n || !a_off || !A || !rank || !skel || !V)))
      throw hb::arg_error("bad hb_id_batch arguments");
    if (!(eps >= 0)) throw hb::arg_error("eps must be >= 0");
    if (count == 0) return;
    std::vector<long long> soff(count), voff(count);
    long long sacc = 0, vacc = 0;
    int max_n = 0;
    for (int b = 0; b < count; ++b) {
      if (m[b] < 1 || n[b] < 1) throw hb::arg_error("matrix %d has an empty dimension", b);
      soff[b] = sacc;
      voff[b] = vacc;
      sacc += n[b];
      vacc += (long long)n[b] * n[b];
      max_n = std::max(max_n, n[b]);
    }
    int* d_m = hb::upload(std::vector<int>(m, m + count));
    int* d_n = hb::upload(std::vector<int>(n, n + count));
    long long* d_a = hb::upload(std::vector<long long>(a_off, a_off + count));
    long long* d_s = hb::upload(soff);
    long long* d_v = hb::upload(voff);
    int* d_perm = hb::dev_alloc<int>(sacc);
    hb::id_batch(count, d_m, d_n, d_a, (double2*)A, eps, rank, d_perm, d_s, max_n, 0);
    hb::emit_v(count, d_m, d_n, d_a, (const double2*)A, rank, d_perm, d_s, d_v, 0, (double2*)V, nullptr, 0);
    HB_CUDA(cudaMemcpy(skel, d_perm, sizeof(int) * sacc, cudaMemcpyDeviceToDevice));
    HB_CUDA(cudaDeviceSynchronize());
    hb::dev_free(d_perm);
    for (void* p : {(void*)d_m, (void*)d_n, (void*)d_a, (void*)d_s, (void*)d_v}) hb::dev_free(p);
  });
}

hb_status hb_id_batch_noalloc(int count, const int* m, const int* n, const long long* a_off, void* A, double eps,
                              int* rank, int* skel, void* V, void* stream) {
  return guarded(nullptr, [&] {
    if (count < 0 || (count > 0 && (!m || !n || !a_off || !A || !rank || !skel || !V)))
      throw hb::arg_error("bad hb_id_batch_noalloc arguments");
    if (!(eps >= 0)) throw hb::arg_error("eps must be >= 0");
    hb::id_batch_noalloc(count, m, n, a_off, (double2*)A, eps, rank, skel, (double2*)V, (cudaStream_t)stream);
  });
}

hb_status hb_tree_perm(hb_handle h, long long* perm_out) {
  return guarded(h, [&] {
    if (!h || !perm_out) throw hb::arg_error("null argument");
    std::memcpy(perm_out, h->perm.data(), sizeof(long long) * h->Nv);
  });
}

hb_status hb_proxy_rows(hb_handle h, long long t0, long long t1, const long long* seeds, int nseeds,
                        long long* out, long long* count) {
  return guarded(h, [&] {
    if (!h || !out || !count || (nseeds > 0 && !seeds)) throw hb::arg_error("null argument");
    if (t0 < 0 || t1 > h->Nv || t0 >= t1) throw hb::arg_error("bad range");
    for (int s = 0; s < nseeds; ++s)
      if (seeds[s] < 0 || seeds[s] >= h->Nv) throw hb::arg_error("seed out of range");
    std::vector<long long> rows;
    std::vector<int> stamp((size_t)h->Nv, -1);
    hb::proxy_rows(h, t0, t1, seeds, nseeds, rows, stamp, 1);
    std::memcpy(out, rows.data(), sizeof(long long) * rows.size());
    *count = (long long)rows.size();
  });
}

namespace {
// A context holding only what the host rules read (no device state).
void host_tree_ctx(hb_ctx& c, int nx, int ny, int leaf) {
  if (nx < 1 || ny < 1 || (long long)nx * ny > (1LL << 31)) throw hb::arg_error("bad grid");
  if (leaf < 1) throw hb::arg_error("leaf must be >= 1");
  c.nx = nx;
  c.ny = ny;
  c.Nv = (long long)nx * ny;
  c.opt.leaf = leaf;
  hb::tree_build(&c);
}
}  // namespace

hb_status hb_host_shard_rows(int nx, int ny, int leaf, int nranks, int rank, long long* lo, long long* hi) {
  return guarded(nullptr, [&] {
    if (!lo || !hi) throw hb::arg_error("null argument");
    hb_ctx c;
    host_tree_ctx(c, nx, ny, leaf);
    hb::shard_rows(&c, nranks, rank, lo, hi);
  });
}

hb_status hb_host_cluster_tree(int nx, int ny, int leaf, long long* perm_out, long long* bounds_out, int* levels) {
  return guarded(nullptr, [&] {
    if (!levels) throw hb::arg_error("null argument");
    hb_ctx c;
    host_tree_ctx(c, nx, ny, leaf);
    *levels = c.Lv;
    if (perm_out) std::memcpy(perm_out, c.perm.data(), sizeof(long long) * (size_t)c.Nv);
    if (bounds_out)
      for (int l = 0; l <= c.Lv; ++l) {
        std::memcpy(bounds_out, c.bounds[(size_t)l].data(), sizeof(long long) * c.bounds[(size_t)l].size());
        bounds_out += c.bounds[(size_t)l].size();
      }
  });
}

hb_status hb_host_segment_tree(const double* centers, long long ns, int leaf, long long* perm_out,
                               long long* bounds_out, int* levels) {
  return guarded(nullptr, [&] {
    if (!centers || !levels) throw hb::arg_error("null argument");
    if (ns < 1 || ns > (1LL << 31)) throw hb::arg_error("segments outside [1, 2^31]");
    if (leaf < 1) throw hb::arg_error("leaf must be >= 1");
    std::vector<double> cx((size_t)ns), cz((size_t)ns);
    for (long long i = 0; i < ns; ++i) {
      cx[(size_t)i] = centers[2 * i];
      cz[(size_t)i] = centers[2 * i + 1];
      if (!std::isfinite(cx[(size_t)i]) || !std::isfinite(cz[(size_t)i]))
        throw hb::arg_error("segment %lld: centre not finite", i);
    }
    std::vector<long long> perm;
    std::vector<std::vector<long long>> bounds;
    hb::segment_tree_build(cx.data(), cz.data(), ns, leaf, perm, bounds);
    *levels = (int)bounds.size() - 1;
    if (perm_out) std::memcpy(perm_out, perm.data(), sizeof(long long) * perm.size());
    if (bounds_out)
      for (const std::vector<long long>& b : bounds) {
        std::memcpy(bounds_out, b.data(), sizeof(long long) * b.size());
        bounds_out += b.size();
      }
  });
}

hb_status hb_host_point_proxy_rows(const double* rows_xz, long long nrows, long long t0, long long t1,
                                   const double* seeds_xz, int nseeds, double chi, double radius, long long* out,
                                   long long* count) {
  return guarded(nullptr, [&] {
    if (!rows_xz || !out || !count || nseeds < 0 || (nseeds > 0 && !seeds_xz)) throw hb::arg_error("null argument");
    if (t0 < 0 || t1 > nrows || t0 >= t1) throw hb::arg_error("bad range");
    if (!(chi > 0) || !(radius >= 0)) throw hb::arg_error("bad options (chi > 0, radius >= 0)");
    std::vector<long long> rows;
    hb::point_proxy_rows(rows_xz, t0, t1, seeds_xz, nseeds, chi, radius, rows);
    std::memcpy(out, rows.data(), sizeof(long long) * rows.size());
    *count = (long long)rows.size();
  });
}

hb_status hb_host_proxy_rows(int nx, int ny, int leaf, double chi, double nbr_radius_h, long long t0, long long t1,
                             const long long* seeds, int nseeds, long long* out, long long* count) {
  return guarded(nullptr, [&] {
    if (!out || !count || nseeds < 0 || (nseeds > 0 && !seeds)) throw hb::arg_error("null argument");
    if (!(chi > 0) || !(nbr_radius_h >= 0)) throw hb::arg_error("bad options (chi > 0, radius >= 0)");
    hb_ctx c;
    c.opt.chi = chi;
    c.opt.nbr_radius_h = nbr_radius_h;
    host_tree_ctx(c, nx, ny, leaf);
    if (t0 < 0 || t1 > c.Nv || t0 >= t1) throw hb::arg_error("bad range");
    for (int s = 0; s < nseeds; ++s)
      if (seeds[s] < 0 || seeds[s] >= c.Nv) throw hb::arg_error("seed out of range");
    std::vector<long long> rows;
    std::vector<int> stamp((size_t)c.Nv, -1);
    hb::proxy_rows(&c, t0, t1, seeds, nseeds, rows, stamp, 1);
    std::memcpy(out, rows.data(), sizeof(long long) * rows.size());
    *count = (long long)rows.size();
  });
}

hb_status hb_info(hb_handle h, hb_stats* stats) {
  return guarded(h, [&] {
    if (!h || !stats) throw hb::arg_error("null argument");
    *stats = h->stats;
    stats->built = h->built ? 1 : 0;
  });
}

hb_status hb_set_kernel_timing(hb_handle h, int enable) {
  return guarded(h, [&] {
    if (!h) throw hb::arg_error("null handle");
    h->timing = enable != 0;
  });
}

hb_status hb_kernel_times(hb_handle h, int cap, char (*names)[32], double* total_ms, long long* launches,
                          int* ngroups) {
  return guarded(h, [&] {
    if (!h || !ngroups || (cap > 0 && (!names || !total_ms || !launches))) throw hb::arg_error("null argument");
    int n = (int)h->tnames.size();
    *ngroups = n;
    for (int i = 0; i < n && i < cap; ++i) {
      std::strncpy(names[i], h->tnames[i].c_str(), 31);
      names[i][31] = 0;
      total_ms[i] = h->tms[i];
      launches[i] = h->tcount[i];
    }
    for (auto& v : h->tms) v = 0;
    for (auto& v : h->tcount) v = 0;
  });
}

const char* hb_last_error(hb_handle h) { return h ? h->err.c_str() : g_err.c_str(); }

void hb_destroy(hb_handle h) {
  if (!h) return;
  free_all(h);
  delete h;
}

}  // extern "C"
