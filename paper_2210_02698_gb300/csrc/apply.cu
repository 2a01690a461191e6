// apply.cu - butterfly / HODBF apply and its adjoint on the device
// (Sec. 4.2.1, Eq. butterfly_mat, Eq. butterfly_factors; Sec. 4.2 HODBF).
//
//   x  = h^2 s, gathered into cluster-tree order            (Eq. m_v2v)
//   steps of small dense products over all butterflies      (build.cu plans)
//   u  = y scattered back to natural order
//
// FP64 path: complex128 factors and vectors, one CTA per task, plain FP64
// FMAs (the baseline).  Mixed path (HB_MIXED_BF16X3): split-BF16 factors and
// vectors in the MMA-fragment layout of bf_mma.cu, up to 32 right-hand
// sides per pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <tuple>
#include <vector>

#include "hb_internal.cuh"

namespace hb {

__global__ void f64_to_f32_kernel(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

void convert_f64_f32(const double2* a, float2* b, long long n, cudaStream_t st) {
  if (n <= 0) return;
  f64_to_f32_kernel<<<1216, 256, 0, st>>>(a, b, n);
  HB_CHECK_LAUNCH();
}

template <class C>
struct Real;
template <>
struct Real<double2> {
  using T = double;
  static __device__ __forceinline__ double2 make(double x, double y) { return make_double2(x, y); }
};
template <>
struct Real<float2> {
  using T = float;
  static __device__ __forceinline__ float2 make(float x, float y) { return make_float2(x, y); }
};

// x[p][r] = scale * s[r*Nv + perm[p]]   (column-major natural -> row-major tree order)
// for tree positions p in [lo, hi); 0 elsewhere (a shard's share of the input)
template <class C>
__global__ void gather_kernel(const double2* __restrict__ s, const long long* __restrict__ perm, C* __restrict__ x,
                              long long Nv, int R, double scale, long long lo, long long hi) {
  long long total = Nv * R;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long p = idx / R;
    int r = (int)(idx % R);
    const double2 v = (p >= lo && p < hi) ? s[(size_t)r * Nv + perm[p]] : make_double2(0.0, 0.0);
    x[idx] = Real<C>::make((typename Real<C>::T)(v.x * scale), (typename Real<C>::T)(v.y * scale));
  }
}

// u[r*Nv + perm[p]] = y[p][r] for tree positions p in [lo, hi)
template <class C>
__global__ void scatter_kernel(const C* __restrict__ y, const long long* __restrict__ perm, double2* __restrict__ u,
                               long long Nv, int R, long long lo, long long hi) {
  long long total = (hi - lo) * R;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    long long p = lo + idx / R;
    int r = (int)(idx % R);
    C v = y[(size_t)p * R + r];
    u[(size_t)r * Nv + perm[p]] = make_double2((double)v.x, (double)v.y);
  }
}

// One CTA per task; thread -> (output row, right-hand side), rows fastest.
template <class C>
__global__ void __launch_bounds__(128) step_kernel(const Task* __restrict__ tasks, const C* __restrict__ F,
                                                   C* __restrict__ x, C* __restrict__ y, C* __restrict__ xh,
                                                   int R) {
  using T = typename Real<C>::T;
  const Task tk = tasks[blockIdx.x];
  C* bufs[3] = {x, y, xh};
  C* out = bufs[tk.y_buf] + (size_t)tk.y_off * R;
  const int total = tk.r_out * R;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int row = idx % tk.r_out, rr = idx / tk.r_out;
    T ar = 0, ai = 0;
    for (int t = 0; t < tk.nterm; ++t) {
      const C* f = F + tk.f_off[t];
      const C* xin = bufs[tk.x_buf] + (size_t)tk.x_off[t] * R + rr;
      const int rin = tk.r_in[t];
      if (!tk.conj_t) {
        for (int k = 0; k < rin; ++k) {
          const C a = f[(size_t)k * tk.r_out + row];
          const C v = xin[(size_t)k * R];
          ar = fma(a.x, v.x, fma(-a.y, v.y, ar));
          ai = fma(a.x, v.y, fma(a.y, v.x, ai));
        }
      } else {
        const C* fr = f + (size_t)row * rin;
        for (int k = 0; k < rin; ++k) {
          const C a = fr[k];
          const C v = xin[(size_t)k * R];
          ar = fma(a.x, v.x, fma(a.y, v.y, ar));     // conj(a) v
          ai = fma(a.x, v.y, fma(-a.y, v.x, ai));
        }
      }
    }
    C* o = out + (size_t)row * R + rr;
    if (tk.accumulate) {
      C prev = *o;
      ar += prev.x;
      ai += prev.y;
    }
    *o = Real<C>::make(ar, ai);
  }
}

namespace {

struct TimerScope {
  hb_ctx* c;
  cudaStream_t st;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
  int group(const char* name) {
    for (size_t i = 0; i < c->tnames.size(); ++i)
      if (c->tnames[i] == name) return (int)i;
    c->tnames.push_back(name);
    c->tms.push_back(0);
    c->tcount.push_back(0);
    return (int)c->tnames.size() - 1;
  }
  void begin(const char* name) {
    nvtxRangePushA(name);   // host-side phase marker (matched in end())
    if (!c->timing) return;
    cudaEvent_t a, b;
    HB_CUDA(cudaEventCreate(&a));
    HB_CUDA(cudaEventCreate(&b));
    HB_CUDA(cudaEventRecord(a, st));
    ev.push_back({group(name), {a, b}});
  }
  void end() {
    nvtxRangePop();
    if (!c->timing) return;
    HB_CUDA(cudaEventRecord(ev.back().second.second, st));
  }
  void finish() {
    if (!c->timing) return;
    HB_CUDA(cudaStreamSynchronize(st));
    for (auto& e : ev) {
      float ms = 0;
      HB_CUDA(cudaEventElapsedTime(&ms, e.second.first, e.second.second));
      c->tms[e.first] += ms;
      c->tcount[e.first] += 1;
      cudaEventDestroy(e.second.first);
      cudaEventDestroy(e.second.second);
    }
    ev.clear();
  }
};

// Scratch of the precision in use (allocated on first use, kept); the device
// is synchronised only after an allocation, so applies stay asynchronous.
void ensure_scratch(hb_ctx* c, int nrhs, bool fp64) {
  bool fresh = false;
  if (fp64 && c->cap_rhs < nrhs) {
    fresh = true;
    dev_free(c->d_x);
    dev_free(c->d_y);
    dev_free(c->d_xh);
    c->d_x = c->d_y = c->d_xh = nullptr;
    c->cap_rhs = 0;
    c->d_x = dev_alloc<double2>((size_t)(c->Nv + 1) * nrhs);
    c->d_y = dev_alloc<double2>((size_t)(c->Nv + 1) * nrhs);
    c->d_xh = dev_alloc<double2>((size_t)(std::max<long long>(c->xh_rows, 1) + 1) * nrhs);
    c->cap_rhs = nrhs;
  }
  if (!c->d_perm) {
    fresh = true;
    c->d_perm = upload(c->perm);
  }
  if (!fp64 && (!c->d_mx || !c->d_mxh || !c->d_flags || !c->d_mx_tc)) {
    // native vectors for two m-tiles: 2 KB per row tile, x again in the
    // tensor-core operand layout, and the dataflow launch's flags (all or
    // none: an allocation that failed half way is redone whole on the next
    // call)
    fresh = true;
    for (void* p : {(void*)c->d_mx, (void*)c->d_mxh, (void*)c->d_flags, (void*)c->d_mx_tc}) dev_free(p);
    c->d_mx = c->d_mxh = c->d_mx_tc = nullptr;
    c->d_flags = c->d_epoch = nullptr;
    c->d_mx = dev_alloc<uint4>((size_t)std::max<long long>(c->nv_tiles, 1) * 128);
    c->d_mx_tc = dev_alloc<uint4>((size_t)std::max<long long>(c->nv_tiles, 1) * 128);
    c->d_mxh = dev_alloc<uint4>((size_t)std::max<long long>(c->xh_tiles, 1) * 128);
    // + the dataflow launch's epoch and finish count, the grid barriers' arrival and finish counts
    const size_t nflags = (size_t)(c->nv_tiles + c->xh_tiles) + 4;
    c->d_flags = dev_alloc<unsigned>(nflags);
    HB_CUDA(cudaMemset(c->d_flags, 0, sizeof(unsigned) * nflags));
    c->d_epoch = c->d_flags + (c->nv_tiles + c->xh_tiles);
  }
  if (!c->h_err) {
    fresh = true;
    HB_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&c->h_err), sizeof(int), cudaHostAllocMapped));
    *c->h_err = 0;
    HB_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&c->d_err), c->h_err, 0));
  }
  if (fresh) HB_CUDA(cudaDeviceSynchronize());
}

}  // namespace

// One launch of FP64 step tasks (one CTA each), for other operators'
// butterflies (curve_bf.cu).
void run_tasks_fp64(const Task* d_tasks, int n, const double2* F, double2* x, double2* y, double2* xh, int R,
                    cudaStream_t st) {
  if (n <= 0) return;
  step_kernel<double2><<<n, 128, 0, st>>>(d_tasks, F, x, y, xh, R);
  HB_CHECK_LAUNCH();
}

namespace {

template <class C>
void run_steps(hb_ctx* c, const C* F, int nrhs, int dir, cudaStream_t st, TimerScope& ts) {
  const std::vector<int>& sb = c->step_begin[dir];
  for (size_t s = 0; s + 1 < sb.size(); ++s) {
    int n = sb[s + 1] - sb[s];
    if (n == 0) continue;
    ts.begin(dir ? "bf_step_adjoint" : "bf_step");
    step_kernel<C><<<n, 128, 0, st>>>(c->d_tasks[dir] + sb[s], F, (C*)c->d_x, (C*)c->d_y, (C*)c->d_xh, nrhs);
    HB_CHECK_LAUNCH();
    ts.end();
  }
}

}  // namespace

void apply_bf(hb_ctx* c, const double2* s, double2* u, int nrhs, int adjoint, int precision, cudaStream_t st) {
  NvtxRange nr(adjoint ? "hb_apply_adjoint" : "hb_apply");
  if (c->h_err && *reinterpret_cast<volatile int*>(c->h_err)) {
    *reinterpret_cast<volatile int*>(c->h_err) = 0;
    throw Error{HB_ERR_TIMEOUT, "a bounded device wait of an earlier apply gave up"};
  }
  // right-hand sides per pass: the scratch vectors (skeleton rows x pass x 16
  // bytes for FP64) stay bounded for any nrhs
  const int chunk = std::min(nrhs, precision == HB_FP64 ? 16 : 32);
  ensure_scratch(c, chunk, precision == HB_FP64);
  TimerScope ts{c, st, {}};
  const double scale = c->h * c->h;
  for (int r0 = 0; r0 < nrhs; r0 += chunk) {
    const int R = std::min(chunk, nrhs - r0);
    const double2* sc = s + (size_t)r0 * c->Nv;
    double2* uc = u + (size_t)r0 * c->Nv;
    const long long total = c->Nv * R;
    const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    if (precision == HB_FP64) {
      ts.begin("gather");
      gather_kernel<double2><<<grid, 256, 0, st>>>(sc, c->d_perm, (double2*)c->d_x, c->Nv, R, scale, 0, c->Nv);
      HB_CHECK_LAUNCH();
      ts.end();
      run_steps<double2>(c, c->d_f64, R, adjoint, st, ts);
      ts.begin("scatter");
      scatter_kernel<double2><<<grid, 256, 0, st>>>((double2*)c->d_y, c->d_perm, uc, c->Nv, R, 0, c->Nv);
      HB_CHECK_LAUNCH();
      ts.end();
    } else {
      // the gather and every depth (the last one writes u): one persistent
      // launch, or a gather and one launch per depth; the timer brackets the
      // step launches (with the gather inside them in the first form)
      flow_launch(c->flow_plan[adjoint], c->tc_plan[adjoint], c->d_tc[adjoint], c->d_nat[adjoint], sc, scale,
                  c->d_mx, c->d_mx_tc, c->d_mxh, uc, c->d_pperm, c->Nv, c->nv_tiles, R, c->d_flags, c->d_epoch,
                  c->d_err,
                  c->opt.barrier_cycles > 0 ? c->opt.barrier_cycles : (1LL << 31), c->wait_selftest,
                  c->opt.autotune, st, [&](int, bool begin) {
                    if (begin) ts.begin(adjoint ? "bf_tc_adjoint" : "bf_tc");
                    else ts.end();
                  });
    }
  }
  ts.finish();
}

// ------------------------------------------------------------- shards ----
// Rank `rank` of `nranks` (a power of two, at most 2^L_v) owns node `rank`
// of level log2(nranks) of the cluster tree: the tree positions [lo, hi).
void shard_rows(const hb_ctx* c, int nranks, int rank, long long* lo, long long* hi) {
  if (nranks < 1 || (nranks & (nranks - 1)) || rank < 0 || rank >= nranks)
    throw arg_error("nranks must be a power of two and 0 <= rank < nranks (got %d, %d)", nranks, rank);
  int k = 0;
  while ((1 << k) < nranks) ++k;
  if (k > c->Lv) throw arg_error("nranks=%d exceeds the %lld leaves of the cluster tree", nranks, 1LL << c->Lv);
  *lo = c->bounds[k][rank];
  *hi = c->bounds[k][rank + 1];
}

namespace {
struct ShardSteps {
  std::vector<int> begin;
  Task* d_tasks = nullptr;
};
}  // namespace

// The FP64 step lists of one shard: the tasks whose rows meet [lo, hi).
static ShardSteps& shard_steps(hb_ctx* c, int dir, long long lo, long long hi) {
  static_assert(sizeof(void*) == 8, "");
  auto key = std::make_tuple(dir, lo, hi);
  auto it = c->shard_cache.find(key);
  if (it != c->shard_cache.end()) return *static_cast<ShardSteps*>(it->second);
  ShardSteps* S = new ShardSteps();
  std::vector<Task> keep;
  const std::vector<int>& sb = c->step_begin[dir];
  for (size_t q = 0; q + 1 < sb.size(); ++q) {
    S->begin.push_back((int)keep.size());
    for (int t = sb[q]; t < sb[q + 1]; ++t) {
      const auto& rr = c->task_rows[dir][(size_t)t];
      if (rr.first < hi && rr.second > lo) keep.push_back(c->tasks_h[dir][(size_t)t]);
    }
  }
  S->begin.push_back((int)keep.size());
  try {
    S->d_tasks = upload(keep);
  } catch (...) {
    delete S;
    throw;
  }
  c->shard_cache[key] = S;
  return *S;
}

void shard_cache_free(hb_ctx* c) {
  for (auto& kv : c->shard_cache) {
    ShardSteps* S = static_cast<ShardSteps*>(kv.second);
    dev_free(S->d_tasks);
    delete S;
  }
  c->shard_cache.clear();
}

// The padded row (mixed path) where the leaf starting at tree position pos
// starts (pos = N_v: the end).
static long long padded_row_of(const hb_ctx* c, long long pos) {
  const std::vector<long long>& b = c->bounds[(size_t)c->Lv];
  const auto it = std::lower_bound(b.begin(), b.end(), pos);
  if (it == b.end() || *it != pos) throw Error{HB_ERR_STATE, "shard boundary is not a leaf boundary"};
  return 8 * c->leaf_tile[(size_t)(it - b.begin())];
}

// One rank's share of the apply.  Forward (u = A s): s is the whole input
// (natural order, every rank's cells); the rank computes every task whose
// rows meet its own and writes u on its cells only.  Adjoint (s = A^H u):
// u holds the rank's cells (the rest is ignored, read as zero); the rank
// computes the tasks whose rows meet its own with the skeleton vectors of
// the others zero, and writes its share of s on every cell; the shares of
// all ranks add up to the adjoint.
void apply_bf_shard(hb_ctx* c, const double2* s, double2* u, int nrhs, int adjoint, int precision, int nranks,
                    int rank, cudaStream_t st) {
  NvtxRange nr(adjoint ? "hb_apply_shard_adjoint" : "hb_apply_shard");
  if (c->h_err && *reinterpret_cast<volatile int*>(c->h_err)) {
    *reinterpret_cast<volatile int*>(c->h_err) = 0;
    throw Error{HB_ERR_TIMEOUT, "a bounded device wait of an earlier apply gave up"};
  }
  long long lo = 0, hi = 0;
  shard_rows(c, nranks, rank, &lo, &hi);
  const int chunk = std::min(nrhs, precision == HB_FP64 ? 16 : 32);
  ensure_scratch(c, chunk, precision == HB_FP64);
  const double scale = c->h * c->h;
  const long long glo = adjoint ? lo : 0, ghi = adjoint ? hi : c->Nv;    // input rows
  const long long slo = adjoint ? 0 : lo, shi = adjoint ? c->Nv : hi;   // output rows
  for (int r0 = 0; r0 < nrhs; r0 += chunk) {
    const int R = std::min(chunk, nrhs - r0);
    const double2* sc = s + (size_t)r0 * c->Nv;
    double2* uc = u + (size_t)r0 * c->Nv;
    const long long total = c->Nv * R;
    const int grid = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    if (precision == HB_FP64) {
      gather_kernel<double2><<<grid, 256, 0, st>>>(sc, c->d_perm, (double2*)c->d_x, c->Nv, R, scale, glo, ghi);
      HB_CHECK_LAUNCH();
      if (adjoint) {
        HB_CUDA(cudaMemsetAsync(c->d_y, 0, sizeof(double2) * (size_t)c->Nv * R, st));
        HB_CUDA(cudaMemsetAsync(c->d_xh, 0, sizeof(double2) * (size_t)std::max<long long>(c->xh_rows, 1) * R, st));
      }
      ShardSteps& S = shard_steps(c, adjoint, lo, hi);
      for (size_t q = 0; q + 1 < S.begin.size(); ++q) {
        const int n = S.begin[q + 1] - S.begin[q];
        if (n == 0) continue;
        step_kernel<double2><<<n, 128, 0, st>>>(S.d_tasks + S.begin[q], c->d_f64, (double2*)c->d_x,
                                               (double2*)c->d_y, (double2*)c->d_xh, R);
        HB_CHECK_LAUNCH();
      }
      const int g2 = (int)std::max<long long>(1, std::min<long long>(((shi - slo) * R + 255) / 256, 152LL * 16));
      scatter_kernel<double2><<<g2, 256, 0, st>>>((double2*)c->d_y, c->d_perm, uc, c->Nv, R, slo, shi);
      HB_CHECK_LAUNCH();
    } else {
      flow_launch_shard(c->flow_plan[adjoint], c->d_nat[adjoint], sc, scale, c->d_mx, c->d_mxh, c->xh_tiles, uc,
                        c->d_pperm, c->Nv, c->nv_tiles, R, lo, hi, adjoint ? padded_row_of(c, lo) : 0,
                        adjoint ? padded_row_of(c, hi) : (long long)8 * c->nv_tiles, adjoint != 0, c->d_err,
                        c->opt.barrier_cycles > 0 ? c->opt.barrier_cycles : (1LL << 31), st);
    }
  }
}

}  // namespace hb
