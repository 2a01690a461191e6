// bf_mma.cu - mixed-precision butterfly apply: one persistent dataflow
// launch, TMA-streamed factor chunks and split-BF16 tensor-core products
// (Sec. 4.2.1, Eq. butterfly_mat: every factor level is a batch of small
// dense complex products Y = op(F) X).
//
// Data movement.  Every product is cut into "pieces": a contiguous chunk of
// the column-major factor block (forward: KC whole columns, i.e. all output
// rows for KC inputs; adjoint op = F^H: OC whole stored columns, i.e. OC
// outputs for all inputs) plus the matching contiguous rows of the input
// vectors.  A producer warp streams pieces through a shared-memory ring with
// cp.async.bulk (the 1D TMA copy) on mbarriers, so every factor byte is read
// from HBM once, by the copy engine, with whole pieces (up to 16 KB of
// factors each) in flight; see flow_kernel for the scheduling.
//
// Arithmetic.  Factors and vectors are FP32 complex.  Products run as real
// BF16 MMAs (mma.sync m16n8k16, FP32 accumulate) on a split of both
// operands, a = a_hi + a_lo, a_hi = bf16(a), a_lo = bf16(a - a_hi):
//     a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi          (split BF16 x 3)
// Complex -> real layout (k' = 2k + c interleaves real/imaginary parts):
//     D_r[m][n] = sum_k' A_r[m][k'] B[k'][n],   D_i[m][n] = sum_k' A_i[m][k'] B[k'][n]
//     A_r[m][(2k,2k+1)] = (Re X[k][m], -Im X[k][m]),  A_i[m][(2k,2k+1)] = (Im X[k][m], Re X[k][m])
//     B[(2k,2k+1)][n]   = (Re F[n][k], Im F[n][k])   (conj(F[k][n]) for op = ^H)
// M = right-hand sides (16 per m-tile), N = 8 output rows per n-tile, K = 8
// complex inputs per k16 step; Y[n][m] = D_r[m][n] + i D_i[m][n].  Ranks
// pad only to multiples of 8 in registers, never in memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "hb_internal.cuh"

namespace hb {

constexpr int TMA_WARPS = 4;
constexpr int TMA_MAX_NT = 4;          // n-tiles per warp: outputs per CTA <= 128
constexpr int TMA_MAX_ROWS = 8 * TMA_WARPS * TMA_MAX_NT;
constexpr int TMA_F_BYTES = 16384;     // factor bytes per piece (stage)

struct TPiece {
  long long f_off;   // element offset of the contiguous factor chunk
  long long x_off;   // first input row
  int f_rows;        // stored rows of the chunk (its leading dimension)
  int f_cols;        // stored columns of the chunk
  int x_rows;        // input rows = reduction length of the piece
  unsigned char x_buf, conj_t, pad0, pad1;
};

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// split (x, y) -> hi = bf16x2(x, y), lo = bf16x2(x - hi.x, y - hi.y)
__device__ __forceinline__ void split2(float x, float y, uint32_t& hi, uint32_t& lo) {
  hi = bf16x2(x, y);
  const float hx = __uint_as_float(hi << 16);
  const float hy = __uint_as_float(hi & 0xffff0000u);
  lo = bf16x2(x - hx, y - hy);
}

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// 1D bulk copy global -> shared, completion counted on the mbarrier.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ uint32_t piece_fbytes(const TPiece& pc) {
  return (uint32_t)((pc.f_rows * pc.f_cols * 8 + 15) & ~15);
}

// ------------------------------------------------------ dataflow kernel ----
// One persistent launch runs every factor level of every HODBF block.  CTA
// tasks are listed in dependency order and dealt round-robin to the CTAs
// (all co-resident: cooperative launch).  Warp 4 is the producer: it waits
// (bounded) until the tasks that wrote a task's inputs have published their
// release flags, then streams the task's pieces into a FLOW_STAGES-deep
// shared-memory ring with 1D TMA copies.  Warps 0-3 are consumers: split-BF16
// MMAs per piece, and at a task's last piece they store its outputs, fence
// (generic -> async proxy, then gpu scope) and publish the task's flag.
// Because every task only waits on tasks earlier in the list, the earliest
// unfinished task can always progress.  Every wait is bounded by one
// deadline per thread (kernel start + budget cycles); past it the mapped
// error word is set and waits are abandoned, so the launch always ends.
constexpr int FLOW_STAGES = 3;
constexpr int FLOW_CONSUMERS = TMA_WARPS;

struct FTask {
  long long y_off;
  int r_out;
  int piece_begin, npiece;
  int wait_begin, nwait;
  int y_buf;
};

struct StageMeta {
  TPiece pc;
  long long y_off;
  int r_out, task, y_buf, xpad;
  int first, last;
};

// Wait for an mbarrier phase until the kernel-wide deadline (clock64 of this
// SM); past it, the error word is set and the wait is abandoned.
__device__ __forceinline__ bool mbar_wait_until(uint64_t* bar, uint32_t parity, long long deadline, int* err) {
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() > deadline) {
      if (err) *reinterpret_cast<volatile int*>(err) = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct FlowArgs {
  const FTask* tasks;
  const TPiece* pieces;
  const int* waits;
  int* flags;
  int ntasks;
  int epoch;
  const float2* F;
  float2* x;
  float2* y;
  float2* xh;
  int R;
  int stage_bytes;
  long long budget;
  int* err;
};

template <int MT>
__global__ void __launch_bounds__((FLOW_CONSUMERS + 1) * 32, 1) flow_kernel(FlowArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t full[FLOW_STAGES], empty[FLOW_STAGES];
  __shared__ StageMeta meta[FLOW_STAGES];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int R = a.R;
  auto buf = [&](int id) { return id == 0 ? a.x : (id == 1 ? a.y : a.xh); };

  if (tid == 0) {
    for (int s = 0; s < FLOW_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], FLOW_CONSUMERS);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const long long deadline = clock64() + a.budget;
  if (warp == FLOW_CONSUMERS) {
    // ------------------------------------------------------------ producer
    if (lane != 0) return;
    long long i = 0;
    for (int q = blockIdx.x; q < a.ntasks; q += gridDim.x) {
      const FTask T = a.tasks[q];
      for (int w = 0; w < T.nwait; ++w) {
        const int* f = a.flags + a.waits[T.wait_begin + w];
        while (ld_acquire(f) != a.epoch) {
          if (clock64() > deadline) {
            *reinterpret_cast<volatile int*>(a.err) = 2;
            break;
          }
          __nanosleep(32);
        }
      }
      asm volatile("fence.proxy.async.global;" ::: "memory");
      for (int p = 0; p < T.npiece; ++p, ++i) {
        const int s = (int)(i % FLOW_STAGES);
        if (i >= FLOW_STAGES)
          mbar_wait_until(&empty[s], (uint32_t)(((i / FLOW_STAGES) - 1) & 1), deadline, a.err);
        const TPiece pc = a.pieces[T.piece_begin + p];
        unsigned char* st = smem + (size_t)s * a.stage_bytes;
        const uint32_t fbytes = piece_fbytes(pc);
        const char* xsrc = reinterpret_cast<const char*>(buf(pc.x_buf) + (size_t)pc.x_off * R);
        const uintptr_t xa = reinterpret_cast<uintptr_t>(xsrc) & ~(uintptr_t)15;
        const int pad = (int)(reinterpret_cast<uintptr_t>(xsrc) - xa);
        const uint32_t xbytes = (uint32_t)((pad + pc.x_rows * R * 8 + 15) & ~15);
        StageMeta& m = meta[s];
        m.pc = pc;
        m.y_off = T.y_off;
        m.r_out = T.r_out;
        m.task = q;
        m.y_buf = T.y_buf;
        m.xpad = pad;
        m.first = (p == 0);
        m.last = (p == T.npiece - 1);
        mbar_expect_tx(&full[s], fbytes + xbytes);
        tma_load_1d(st, a.F + pc.f_off, fbytes, &full[s]);
        tma_load_1d(st + ((fbytes + 127) & ~127u), reinterpret_cast<const void*>(xa), xbytes, &full[s]);
      }
    }
    return;
  }

  // -------------------------------------------------------------- consumers
  const int g = lane >> 2, t = lane & 3;
  long long npieces = 0;
  for (int q = blockIdx.x; q < a.ntasks; q += gridDim.x) npieces += a.tasks[q].npiece;
  float acc_r[TMA_MAX_NT][MT][4];
  float acc_i[TMA_MAX_NT][MT][4];
  for (long long i = 0; i < npieces; ++i) {
    const int s = (int)(i % FLOW_STAGES);
    const bool ok = mbar_wait_until(&full[s], (uint32_t)((i / FLOW_STAGES) & 1), deadline, a.err);
    const StageMeta& m = meta[s];
    const TPiece pc = m.pc;
    const int r_out = m.r_out;
    if (m.first) {
#pragma unroll
      for (int j = 0; j < TMA_MAX_NT; ++j)
#pragma unroll
        for (int aa = 0; aa < MT; ++aa)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc_r[j][aa][e] = acc_i[j][aa][e] = 0.f;
    }
    const unsigned char* st = smem + (size_t)s * a.stage_bytes;
    const float2* Fs = reinterpret_cast<const float2*>(st);
    const float2* Xs = reinterpret_cast<const float2*>(st + ((piece_fbytes(pc) + 127) & ~127u) + m.xpad);
    const int kr = ok ? pc.x_rows : 0;
    for (int kb = 0; kb < kr; kb += 8) {
      const int k0 = kb + t, k1 = kb + t + 4;
      uint32_t bh0[TMA_MAX_NT], bl0[TMA_MAX_NT], bh1[TMA_MAX_NT], bl1[TMA_MAX_NT];
#pragma unroll
      for (int j = 0; j < TMA_MAX_NT; ++j) {
        const int n = 8 * (warp + FLOW_CONSUMERS * j) + g;
        float2 v0 = make_float2(0.f, 0.f), v1 = v0;
        if (n < r_out) {
          if (!pc.conj_t) {
            if (k0 < kr) v0 = Fs[k0 * pc.f_rows + n];
            if (k1 < kr) v1 = Fs[k1 * pc.f_rows + n];
          } else {
            if (k0 < kr) { v0 = Fs[n * pc.f_rows + k0]; v0.y = -v0.y; }
            if (k1 < kr) { v1 = Fs[n * pc.f_rows + k1]; v1.y = -v1.y; }
          }
        }
        split2(v0.x, v0.y, bh0[j], bl0[j]);
        split2(v1.x, v1.y, bh1[j], bl1[j]);
      }
#pragma unroll
      for (int aa = 0; aa < MT; ++aa) {
        const int mA = aa * 16 + g, mB = mA + 8;
        float2 x00 = make_float2(0.f, 0.f), x01 = x00, x10 = x00, x11 = x00;
        if (k0 < kr) {
          if (mA < R) x00 = Xs[k0 * R + mA];
          if (mB < R) x01 = Xs[k0 * R + mB];
        }
        if (k1 < kr) {
          if (mA < R) x10 = Xs[k1 * R + mA];
          if (mB < R) x11 = Xs[k1 * R + mB];
        }
        uint32_t arh[4], arl[4], aih[4], ail[4];
        split2(x00.x, -x00.y, arh[0], arl[0]);
        split2(x01.x, -x01.y, arh[1], arl[1]);
        split2(x10.x, -x10.y, arh[2], arl[2]);
        split2(x11.x, -x11.y, arh[3], arl[3]);
        split2(x00.y, x00.x, aih[0], ail[0]);
        split2(x01.y, x01.x, aih[1], ail[1]);
        split2(x10.y, x10.x, aih[2], ail[2]);
        split2(x11.y, x11.x, aih[3], ail[3]);
#pragma unroll
        for (int j = 0; j < TMA_MAX_NT; ++j) {
          if (8 * (warp + FLOW_CONSUMERS * j) >= r_out) break;
          mma16816(acc_r[j][aa], arh, bh0[j], bh1[j]);
          mma16816(acc_r[j][aa], arh, bl0[j], bl1[j]);
          mma16816(acc_r[j][aa], arl, bh0[j], bh1[j]);
          mma16816(acc_i[j][aa], aih, bh0[j], bh1[j]);
          mma16816(acc_i[j][aa], aih, bl0[j], bl1[j]);
          mma16816(acc_i[j][aa], ail, bh0[j], bh1[j]);
        }
      }
    }
    const int last = m.last, task = m.task, y_buf = m.y_buf;
    const long long y_off = m.y_off;
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);   // this warp is done reading stage s
    if (last) {
      float2* out = buf(y_buf) + (size_t)y_off * R;
#pragma unroll
      for (int j = 0; j < TMA_MAX_NT; ++j) {
#pragma unroll
        for (int aa = 0; aa < MT; ++aa) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int mm = aa * 16 + g + ((e & 2) ? 8 : 0);
            const int n = 8 * (warp + FLOW_CONSUMERS * j) + 2 * t + (e & 1);
            if (mm < R && n < r_out) out[(size_t)n * R + mm] = make_float2(acc_r[j][aa][e], acc_i[j][aa][e]);
          }
        }
      }
      // outputs may be read by other CTAs' bulk copies: order them for the
      // async proxy, then publish after all consumer warps have written
      asm volatile("fence.proxy.async.global;" ::: "memory");
      asm volatile("bar.sync 1, %0;" ::"n"(FLOW_CONSUMERS * 32) : "memory");
      if (tid == 0) {
        __threadfence();
        st_release(a.flags + task, a.epoch);
      }
    }
  }
}

// ------------------------------------------------------------- planning ----
struct FlowPlan {
  std::vector<FTask> tasks;
  std::vector<TPiece> pieces;
  std::vector<int> waits;
  FTask* d_tasks = nullptr;
  TPiece* d_pieces = nullptr;
  int* d_waits = nullptr;
  int* d_flags = nullptr;
  int max_f_bytes = 16, max_x_rows = 1;
  int epoch = 0;
};

void flow_plan_build(const std::vector<FlowTask>& lt, void** plan_out) {
  FlowPlan* P = new FlowPlan();
  try {
    std::vector<int> first((size_t)lt.size()), count((size_t)lt.size());
    for (size_t q = 0; q < lt.size(); ++q) {
      const FlowTask& L = lt[q];
      bool conj = !L.terms.empty() && L.terms[0].conj_t;
      std::vector<int> wl;
      for (const FlowTerm& tm : L.terms)
        for (int k = 0; k < 2; ++k)
          if (tm.producer[k] >= 0)
            for (int c = 0; c < count[(size_t)tm.producer[k]]; ++c) wl.push_back(first[(size_t)tm.producer[k]] + c);
      std::sort(wl.begin(), wl.end());
      wl.erase(std::unique(wl.begin(), wl.end()), wl.end());
      first[q] = (int)P->tasks.size();
      auto push_task = [&](long long y_off, int r_out, int pb) {
        FTask ft{};
        ft.y_off = y_off;
        ft.r_out = r_out;
        ft.y_buf = L.y_buf;
        ft.piece_begin = pb;
        ft.npiece = (int)P->pieces.size() - pb;
        ft.wait_begin = (int)P->waits.size();
        ft.nwait = (int)wl.size();
        P->waits.insert(P->waits.end(), wl.begin(), wl.end());
        P->tasks.push_back(ft);
      };
      if (!conj) {
        if (L.r_out > TMA_MAX_ROWS) throw Error{HB_ERR_UNSUPPORTED, "a forward factor block has more than 128 rows"};
        const int pb = (int)P->pieces.size();
        int kc = std::min(64, std::max(2, (TMA_F_BYTES / (8 * std::max(1, L.r_out))) & ~1));
        for (const FlowTerm& tm : L.terms)
          for (int j0 = 0; j0 < tm.r_in; j0 += kc) {
            TPiece p{};
            p.f_off = tm.f_off + (long long)j0 * tm.f_rows;
            p.f_rows = tm.f_rows;
            p.f_cols = std::min(kc, tm.r_in - j0);
            p.x_off = tm.x_off + j0;
            p.x_rows = p.f_cols;
            p.x_buf = tm.x_buf;
            P->max_f_bytes = std::max(P->max_f_bytes, p.f_rows * p.f_cols * 8);
            P->max_x_rows = std::max(P->max_x_rows, p.x_rows);
            P->pieces.push_back(p);
          }
        push_task(L.y_off, L.r_out, pb);
      } else {
        int rmax = 1;
        for (const FlowTerm& tm : L.terms) rmax = std::max(rmax, tm.r_in);
        const int oc = std::min(TMA_MAX_ROWS, std::max(8, (TMA_F_BYTES / (8 * rmax)) & ~7));
        for (int n0 = 0; n0 < L.r_out; n0 += oc) {
          const int pb = (int)P->pieces.size();
          const int w = std::min(oc, L.r_out - n0);
          for (const FlowTerm& tm : L.terms) {
            TPiece p{};
            p.f_off = tm.f_off + (long long)n0 * tm.f_rows;
            p.f_rows = tm.f_rows;
            p.f_cols = w;
            p.x_off = tm.x_off;
            p.x_rows = tm.r_in;
            p.x_buf = tm.x_buf;
            p.conj_t = 1;
            P->max_f_bytes = std::max(P->max_f_bytes, p.f_rows * p.f_cols * 8);
            P->max_x_rows = std::max(P->max_x_rows, p.x_rows);
            P->pieces.push_back(p);
          }
          push_task(L.y_off + n0, w, pb);
        }
      }
      count[q] = (int)P->tasks.size() - first[q];
    }
    P->d_tasks = upload(P->tasks);
    P->d_pieces = upload(P->pieces);
    P->d_waits = upload(P->waits);
    P->d_flags = dev_alloc<int>(P->tasks.size());
    HB_CUDA(cudaMemset(P->d_flags, 0, sizeof(int) * std::max<size_t>(1, P->tasks.size())));
  } catch (...) {
    flow_plan_free(P);
    throw;
  }
  *plan_out = P;
}

void flow_plan_free(void* plan) {
  FlowPlan* P = static_cast<FlowPlan*>(plan);
  if (!P) return;
  dev_free(P->d_tasks);
  dev_free(P->d_pieces);
  dev_free(P->d_waits);
  dev_free(P->d_flags);
  delete P;
}

int flow_plan_ctas(const void* plan) { return (int)static_cast<const FlowPlan*>(plan)->tasks.size(); }

template <int MT>
static void launch_flow(FlowPlan* P, const float2* F, float2* x, float2* y, float2* xh, int R, int* err,
                        long long budget, cudaStream_t st) {
  const int fb = (P->max_f_bytes + 15 + 127) & ~127;
  const int xb = (P->max_x_rows * R * 8 + 32 + 127) & ~127;
  const int stage = fb + xb;
  const size_t smem = (size_t)FLOW_STAGES * stage;
  auto k = flow_kernel<MT>;
  HB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, nsm = 0, per_sm = 0;
  HB_CUDA(cudaGetDevice(&dev));
  HB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  HB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (FLOW_CONSUMERS + 1) * 32, smem));
  if (per_sm < 1) throw Error{HB_ERR_UNSUPPORTED, "flow kernel does not fit on an SM"};
  const int grid = std::min((int)P->tasks.size(), nsm * per_sm);
  FlowArgs args{P->d_tasks, P->d_pieces, P->d_waits, P->d_flags, (int)P->tasks.size(), ++P->epoch,
                F, x, y, xh, R, stage, budget, err};
  void* params[] = {&args};
  HB_CUDA(cudaLaunchCooperativeKernel((const void*)k, dim3(grid), dim3((FLOW_CONSUMERS + 1) * 32), params, smem, st));
}

void flow_launch(void* plan, const float2* F, float2* x, float2* y, float2* xh, int R, int* err,
                 long long budget_cycles, cudaStream_t st) {
  FlowPlan* P = static_cast<FlowPlan*>(plan);
  if (P->tasks.empty()) return;
  if (R <= 16) launch_flow<1>(P, F, x, y, xh, R, err, budget_cycles, st);
  else if (R <= 32) launch_flow<2>(P, F, x, y, xh, R, err, budget_cycles, st);
  else if (R <= 64) launch_flow<4>(P, F, x, y, xh, R, err, budget_cycles, st);
  else throw Error{HB_ERR_UNSUPPORTED, "the mixed apply takes at most 64 right-hand sides per pass"};
}

}  // namespace hb
