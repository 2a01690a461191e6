// bf_mma.cu - mixed-precision butterfly apply on the tensor cores
// (Sec. 4.2.1, Eq. butterfly_mat: every factor level is a batch of small
// dense complex products Y = op(F) X; Sec. 4.2 HODBF sum).
//
// Storage.  Factors and vectors are kept as split-BF16 pairs: every complex
// value a is 8 bytes {hi, lo}, hi = bf16x2(Re a, Im a), lo = bf16x2 of the
// remainders a - hi, so that hi + lo keeps ~16 significant bits.  The pairs
// feed the MMA fragments directly; products are
//     a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi          (split BF16 x 3)
// with FP32 accumulation (mma.sync m16n8k16), and results are split again
// when stored.
//
// Complex -> real layout (k' = 2k + c interleaves real/imaginary parts):
//     D_r[m][n] = sum_k' A_r[m][k'] B[k'][n],   D_i[m][n] = sum_k' A_i[m][k'] B[k'][n]
//     A_r[m][(2k,2k+1)] = (Re X[k][m], -Im X[k][m]),  A_i[m][(2k,2k+1)] = (Im X[k][m], Re X[k][m])
//     B[(2k,2k+1)][n]   = (Re F[n][k], Im F[n][k])   (conj(F[k][n]) for op = ^H)
// so a B register is a stored pair (im sign flipped for ^H), an A_r register
// the X pair with the im sign flipped, an A_i register the X pair with its
// halves swapped.  M = right-hand sides (16 per m-tile), N = 8 outputs per
// n-tile, K = 8 complex inputs per k16 step.  Ranks pad to multiples of 8 in
// registers only, never in memory.
//
// Scheduling.  The plan lists tasks by dependency depth (depth d only reads
// outputs of depths < d).  One persistent kernel per depth: CTA b runs the
// depth's tasks b, b + G, ...; its producer warp streams each task's pieces
// (a contiguous factor chunk plus the matching contiguous input rows) into a
// FLOW_STAGES-deep shared-memory ring with cp.async.bulk (1D TMA) on
// mbarriers; four consumer warps run the MMAs and store each task's outputs.
// Depth kernels are chained with programmatic dependent launch: a kernel's
// CTAs start as the previous depth drains, prefetch their first factor
// chunks (constant data), and only then wait (griddepcontrol.wait) before
// copying inputs written by the previous depth.  Every wait is bounded by a
// per-thread deadline; past it the mapped error word is set.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "hb_internal.cuh"

namespace hb {

constexpr int TMA_WARPS = 4;
constexpr int TMA_MAX_NT = 4;          // n-tiles per warp: outputs per task <= 128
constexpr int TMA_MAX_ROWS = 8 * TMA_WARPS * TMA_MAX_NT;
constexpr int TMA_F_BYTES = 16384;     // factor bytes per piece
constexpr int FLOW_STAGES = 3;
constexpr int FLOW_CONSUMERS = TMA_WARPS;
constexpr uint32_t IM_SIGN = 0x80000000u;   // sign bit of the imaginary (upper) bf16

struct TPiece {
  long long f_off;   // element offset of the contiguous factor chunk
  long long x_off;   // first input row
  int f_rows;        // stored rows of the chunk (its leading dimension)
  int f_cols;        // stored columns of the chunk
  int x_rows;        // input rows = reduction length of the piece
  unsigned char x_buf, conj_t, pad0, pad1;
};

// A piece as the producer sees it (each CTA reads its own contiguous stream).
struct SRec {
  TPiece pc;
  long long y_off;
  int r_out;
  int y_buf;
  int first_last;   // bit 0: first piece of its task, bit 1: last
  int pad;
};

struct StageMeta {
  TPiece pc;
  long long y_off;
  int r_out, y_buf, xpad, first_last;
};

// ------------------------------------------------------------ helpers ----
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// split-BF16 pair of the complex value (re, im)
__device__ __forceinline__ uint2 to_pair(float re, float im) {
  const uint32_t hi = bf16x2(re, im);
  const float hr = __uint_as_float(hi << 16), hm = __uint_as_float(hi & 0xffff0000u);
  return make_uint2(hi, bf16x2(re - hr, im - hm));
}

__device__ __forceinline__ float2 from_pair(uint2 p) {
  return make_float2(__uint_as_float(p.x << 16) + __uint_as_float(p.y << 16),
                     __uint_as_float(p.x & 0xffff0000u) + __uint_as_float(p.y & 0xffff0000u));
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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// Wait for an mbarrier phase until the deadline (clock64 of this SM); past
// it the mapped error word is set and the wait is abandoned.
__device__ __forceinline__ bool mbar_wait_until(uint64_t* bar, uint32_t parity, long long deadline, int* err) {
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() > deadline) {
      if (err) *reinterpret_cast<volatile int*>(err) = 1;
      return false;
    }
  }
  return true;
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

struct StepArgs {
  const SRec* recs;
  const long long* cta_off;   // stream of CTA b: [cta_off[b], cta_off[b+1])
  const uint2* F;
  uint2* x;
  uint2* y;
  uint2* xh;
  int R;
  int stage_bytes;
  long long budget;
  int* err;
};

// ------------------------------------------------------------- kernel ----
template <int MT>
__global__ void __launch_bounds__((FLOW_CONSUMERS + 1) * 32, 1) bf_step_kernel(StepArgs a) {
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
  const long long rb = a.cta_off[blockIdx.x], nrec = a.cta_off[blockIdx.x + 1] - rb;

  if (warp == FLOW_CONSUMERS) {
    // ------------------------------------------------------------ producer
    // Pieces 0..FLOW_STAGES-1 first get their factor chunk (constant data),
    // then the kernel waits for the previous depth, then their input rows.
    bool waited = false;
    for (long long r0 = 0; r0 < nrec; r0 += 32) {
      const int nb = (int)min(32LL, nrec - r0);
      SRec rec{};
      if (lane < nb) rec = a.recs[rb + r0 + lane];
      for (int j = 0; j < nb; ++j) {
        if (lane == j) {
          const long long i = r0 + j;
          const int s = (int)(i % FLOW_STAGES);
          if (i >= FLOW_STAGES)
            mbar_wait_until(&empty[s], (uint32_t)(((i / FLOW_STAGES) - 1) & 1), deadline, a.err);
          const TPiece pc = rec.pc;
          unsigned char* st = smem + (size_t)s * a.stage_bytes;
          const uint32_t fbytes = piece_fbytes(pc);
          const char* xsrc = reinterpret_cast<const char*>(buf(pc.x_buf) + (size_t)pc.x_off * R);
          const uintptr_t xa = reinterpret_cast<uintptr_t>(xsrc) & ~(uintptr_t)15;
          const int pad = (int)(reinterpret_cast<uintptr_t>(xsrc) - xa);
          const uint32_t xbytes = (uint32_t)((pad + pc.x_rows * R * 8 + 15) & ~15);
          StageMeta& m = meta[s];
          m.pc = pc;
          m.y_off = rec.y_off;
          m.r_out = rec.r_out;
          m.y_buf = rec.y_buf;
          m.xpad = pad;
          m.first_last = rec.first_last;
          mbar_expect_tx(&full[s], fbytes + xbytes);
          tma_load_1d(st, a.F + pc.f_off, fbytes, &full[s]);
          if (!waited) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            asm volatile("fence.proxy.async.global;" ::: "memory");
            waited = true;
          }
          tma_load_1d(st + ((fbytes + 127) & ~127u), reinterpret_cast<const void*>(xa), xbytes, &full[s]);
        }
        __syncwarp();
      }
    }
    if (lane == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    return;
  }

  // -------------------------------------------------------------- consumers
  // Work split per task: nt n-tiles over wn warp groups and the reduction
  // (k-tiles of every piece) over wk = 4 / wn groups, so each warp holds at
  // most TMA_MAX_NT n-tiles and no warp idles on small ranks; partial sums of
  // the wk groups meet in shared memory at the task's last piece.
  const int g = lane >> 2, t = lane & 3;
  float* red = reinterpret_cast<float*>(smem + (size_t)FLOW_STAGES * a.stage_bytes);
  float acc_r[TMA_MAX_NT][MT][4];
  float acc_i[TMA_MAX_NT][MT][4];
  for (long long i = 0; i < nrec; ++i) {
    const int s = (int)(i % FLOW_STAGES);
    const bool ok = mbar_wait_until(&full[s], (uint32_t)((i / FLOW_STAGES) & 1), deadline, a.err);
    const StageMeta& m = meta[s];
    const TPiece pc = m.pc;
    const int r_out = m.r_out, fl = m.first_last, y_buf = m.y_buf;
    const long long y_off = m.y_off;
    const int nt = (r_out + 7) >> 3;
    const int wn = nt <= TMA_MAX_NT ? 1 : (nt <= 2 * TMA_MAX_NT ? 2 : 4);
    const int wk = FLOW_CONSUMERS / wn;
    const int gn = warp % wn, gk = warp / wn;
    if (fl & 1) {
#pragma unroll
      for (int j = 0; j < TMA_MAX_NT; ++j)
#pragma unroll
        for (int aa = 0; aa < MT; ++aa)
#pragma unroll
          for (int e = 0; e < 4; ++e) acc_r[j][aa][e] = acc_i[j][aa][e] = 0.f;
    }
    const unsigned char* st = smem + (size_t)s * a.stage_bytes;
    const uint2* Fs = reinterpret_cast<const uint2*>(st);
    const uint2* Xs = reinterpret_cast<const uint2*>(st + ((piece_fbytes(pc) + 127) & ~127u) + m.xpad);
    const int kr = ok ? pc.x_rows : 0;
    const uint32_t cs = pc.conj_t ? IM_SIGN : 0u;
    for (int kb = 8 * gk; kb < kr; kb += 8 * wk) {
      const int k0 = kb + t, k1 = kb + t + 4;
      uint32_t bh0[TMA_MAX_NT], bl0[TMA_MAX_NT], bh1[TMA_MAX_NT], bl1[TMA_MAX_NT];
#pragma unroll
      for (int j = 0; j < TMA_MAX_NT; ++j) {
        const int tile = gn + wn * j;
        const int n = 8 * tile + g;
        uint2 v0 = make_uint2(0u, 0u), v1 = v0;
        if (tile < nt && n < r_out) {
          if (!pc.conj_t) {
            if (k0 < kr) v0 = Fs[k0 * pc.f_rows + n];
            if (k1 < kr) v1 = Fs[k1 * pc.f_rows + n];
          } else {
            if (k0 < kr) v0 = Fs[n * pc.f_rows + k0];
            if (k1 < kr) v1 = Fs[n * pc.f_rows + k1];
          }
        }
        bh0[j] = v0.x ^ cs;
        bl0[j] = v0.y ^ cs;
        bh1[j] = v1.x ^ cs;
        bl1[j] = v1.y ^ cs;
      }
#pragma unroll
      for (int aa = 0; aa < MT; ++aa) {
        const int mA = aa * 16 + g, mB = mA + 8;
        uint2 x00 = make_uint2(0u, 0u), x01 = x00, x10 = x00, x11 = x00;
        if (k0 < kr) {
          if (mA < R) x00 = Xs[k0 * R + mA];
          if (mB < R) x01 = Xs[k0 * R + mB];
        }
        if (k1 < kr) {
          if (mA < R) x10 = Xs[k1 * R + mA];
          if (mB < R) x11 = Xs[k1 * R + mB];
        }
        const uint32_t arh[4] = {x00.x ^ IM_SIGN, x01.x ^ IM_SIGN, x10.x ^ IM_SIGN, x11.x ^ IM_SIGN};
        const uint32_t arl[4] = {x00.y ^ IM_SIGN, x01.y ^ IM_SIGN, x10.y ^ IM_SIGN, x11.y ^ IM_SIGN};
        const uint32_t aih[4] = {__byte_perm(x00.x, 0, 0x1032), __byte_perm(x01.x, 0, 0x1032),
                                 __byte_perm(x10.x, 0, 0x1032), __byte_perm(x11.x, 0, 0x1032)};
        const uint32_t ail[4] = {__byte_perm(x00.y, 0, 0x1032), __byte_perm(x01.y, 0, 0x1032),
                                 __byte_perm(x10.y, 0, 0x1032), __byte_perm(x11.y, 0, 0x1032)};
#pragma unroll
        for (int j = 0; j < TMA_MAX_NT; ++j) {
          if (gn + wn * j >= nt) break;
          mma16816(acc_r[j][aa], arh, bh0[j], bh1[j]);
          mma16816(acc_r[j][aa], arh, bl0[j], bl1[j]);
          mma16816(acc_r[j][aa], arl, bh0[j], bh1[j]);
          mma16816(acc_i[j][aa], aih, bh0[j], bh1[j]);
          mma16816(acc_i[j][aa], aih, bl0[j], bl1[j]);
          mma16816(acc_i[j][aa], ail, bh0[j], bh1[j]);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);   // this warp is done reading stage s
    if (fl & 2) {
      // red[warp][j][aa][e][r|i][lane]
      const int per_warp = TMA_MAX_NT * MT * 4 * 2 * 32;
      if (wk > 1) {
        if (gk > 0) {
          float* rw = red + (size_t)warp * per_warp;
#pragma unroll
          for (int j = 0; j < TMA_MAX_NT; ++j)
#pragma unroll
            for (int aa = 0; aa < MT; ++aa)
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                rw[(((j * MT + aa) * 4 + e) * 2 + 0) * 32 + lane] = acc_r[j][aa][e];
                rw[(((j * MT + aa) * 4 + e) * 2 + 1) * 32 + lane] = acc_i[j][aa][e];
              }
        }
        asm volatile("bar.sync 1, %0;" ::"n"(FLOW_CONSUMERS * 32) : "memory");
        if (gk == 0) {
          for (int q = 1; q < wk; ++q) {
            const float* rw = red + (size_t)(gn + wn * q) * per_warp;
#pragma unroll
            for (int j = 0; j < TMA_MAX_NT; ++j)
#pragma unroll
              for (int aa = 0; aa < MT; ++aa)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  acc_r[j][aa][e] += rw[(((j * MT + aa) * 4 + e) * 2 + 0) * 32 + lane];
                  acc_i[j][aa][e] += rw[(((j * MT + aa) * 4 + e) * 2 + 1) * 32 + lane];
                }
          }
        }
      }
      if (gk == 0) {
        uint2* out = buf(y_buf) + (size_t)y_off * R;
#pragma unroll
        for (int j = 0; j < TMA_MAX_NT; ++j) {
          if (gn + wn * j >= nt) break;
#pragma unroll
          for (int aa = 0; aa < MT; ++aa) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int mm = aa * 16 + g + ((e & 2) ? 8 : 0);
              const int n = 8 * (gn + wn * j) + 2 * t + (e & 1);
              if (mm < R && n < r_out) out[(size_t)n * R + mm] = to_pair(acc_r[j][aa][e], acc_i[j][aa][e]);
            }
          }
        }
      }
      if (wk > 1) asm volatile("bar.sync 1, %0;" ::"n"(FLOW_CONSUMERS * 32) : "memory");   // red reusable
    }
  }
}

// --------------------------------------------------- conversions / I/O ----
__global__ void f64_to_pair_kernel(const double2* __restrict__ a, uint2* __restrict__ b, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    b[i] = to_pair((float)a[i].x, (float)a[i].y);
}

// x[p][r] = pair(scale * s[r*Nv + perm[p]])
__global__ void gather_pair_kernel(const double2* __restrict__ s, const long long* __restrict__ perm,
                                   uint2* __restrict__ x, long long Nv, int R, double scale) {
  const long long total = Nv * R;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long p = idx / R;
    const int r = (int)(idx % R);
    const double2 v = s[(size_t)r * Nv + perm[p]];
    x[idx] = to_pair((float)(v.x * scale), (float)(v.y * scale));
  }
}

__global__ void scatter_pair_kernel(const uint2* __restrict__ y, const long long* __restrict__ perm,
                                    double2* __restrict__ u, long long Nv, int R) {
  const long long total = Nv * R;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long p = idx / R;
    const int r = (int)(idx % R);
    const uint2 v = y[idx];
    const double re = (double)__uint_as_float(v.x << 16) + (double)__uint_as_float(v.y << 16);
    const double im = (double)__uint_as_float(v.x & 0xffff0000u) + (double)__uint_as_float(v.y & 0xffff0000u);
    u[(size_t)r * Nv + perm[p]] = make_double2(re, im);
  }
}

void convert_f64_pairs(const double2* a, uint2* b, long long n, cudaStream_t st) {
  if (n <= 0) return;
  f64_to_pair_kernel<<<1216, 256, 0, st>>>(a, b, n);
  HB_CHECK_LAUNCH();
}

void gather_pairs(const double2* s, const long long* perm, uint2* x, long long Nv, int R, double scale,
                  cudaStream_t st) {
  const int grid = (int)std::min<long long>((Nv * R + 255) / 256, 152LL * 16);
  gather_pair_kernel<<<grid, 256, 0, st>>>(s, perm, x, Nv, R, scale);
  HB_CHECK_LAUNCH();
}

void scatter_pairs(const uint2* y, const long long* perm, double2* u, long long Nv, int R, cudaStream_t st) {
  const int grid = (int)std::min<long long>((Nv * R + 255) / 256, 152LL * 16);
  scatter_pair_kernel<<<grid, 256, 0, st>>>(y, perm, u, Nv, R);
  HB_CHECK_LAUNCH();
}

// ------------------------------------------------------------- planning ----
struct CtaTask {
  long long y_off;
  int r_out;
  int piece_begin, npiece;
  int y_buf;
};

struct DepthStreams {
  int grid = 0;
  SRec* d_recs = nullptr;
  long long* d_off = nullptr;
};

struct FlowPlan {
  std::vector<CtaTask> tasks;
  std::vector<TPiece> pieces;
  std::vector<int> depth_begin;           // task ranges per depth
  int max_f_bytes = 16, max_x_rows = 1;
  int gmax = 0;                           // grid the streams were built for
  std::vector<DepthStreams> streams;      // per depth
};

// Cut logical tasks into CTA tasks and TMA pieces.  Factor blocks start at
// even element offsets (16-byte aligned pairs) and column chunks keep even
// offsets, so every piece starts 16-byte aligned.
void flow_plan_build(const std::vector<FlowTask>& lt, void** plan_out) {
  FlowPlan* P = new FlowPlan();
  try {
    int depth = -1;
    for (size_t q = 0; q < lt.size(); ++q) {
      const FlowTask& L = lt[q];
      if (L.depth < depth) throw Error{HB_ERR_STATE, "flow tasks are not sorted by depth"};
      while (depth < L.depth) {
        P->depth_begin.push_back((int)P->tasks.size());
        ++depth;
      }
      const bool conj = !L.terms.empty() && L.terms[0].conj_t;
      auto push_task = [&](long long y_off, int r_out, int pb) {
        CtaTask ct{};
        ct.y_off = y_off;
        ct.r_out = r_out;
        ct.y_buf = L.y_buf;
        ct.piece_begin = pb;
        ct.npiece = (int)P->pieces.size() - pb;
        P->tasks.push_back(ct);
      };
      if (!conj) {
        if (L.r_out > TMA_MAX_ROWS) throw Error{HB_ERR_UNSUPPORTED, "a forward factor block has more than 128 rows"};
        const int pb = (int)P->pieces.size();
        const int kc = std::min(64, std::max(2, (TMA_F_BYTES / (8 * std::max(1, L.r_out))) & ~1));
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
    }
    P->depth_begin.push_back((int)P->tasks.size());
  } catch (...) {
    delete P;
    throw;
  }
  *plan_out = P;
}

void flow_plan_free(void* plan) {
  FlowPlan* P = static_cast<FlowPlan*>(plan);
  if (!P) return;
  for (DepthStreams& d : P->streams) {
    dev_free(d.d_recs);
    dev_free(d.d_off);
  }
  delete P;
}

int flow_plan_depths(const void* plan) {
  return (int)static_cast<const FlowPlan*>(plan)->depth_begin.size() - 1;
}

// Per-CTA record streams of every depth for a maximum grid of gmax CTAs.
static void build_streams(FlowPlan* P, int gmax) {
  for (DepthStreams& d : P->streams) {
    dev_free(d.d_recs);
    dev_free(d.d_off);
  }
  P->streams.clear();
  const int nd = (int)P->depth_begin.size() - 1;
  for (int d = 0; d < nd; ++d) {
    const int t0 = P->depth_begin[d], t1 = P->depth_begin[d + 1];
    DepthStreams ds;
    ds.grid = std::min(gmax, t1 - t0);
    std::vector<SRec> recs;
    std::vector<long long> off;
    for (int b = 0; b < ds.grid; ++b) {
      off.push_back((long long)recs.size());
      for (int q = t0 + b; q < t1; q += ds.grid) {
        const CtaTask& T = P->tasks[(size_t)q];
        for (int p = 0; p < T.npiece; ++p) {
          SRec r{};
          r.pc = P->pieces[(size_t)T.piece_begin + p];
          r.y_off = T.y_off;
          r.r_out = T.r_out;
          r.y_buf = T.y_buf;
          r.first_last = (p == 0 ? 1 : 0) | (p == T.npiece - 1 ? 2 : 0);
          recs.push_back(r);
        }
      }
    }
    off.push_back((long long)recs.size());
    if (ds.grid > 0) {
      ds.d_recs = upload(recs);
      ds.d_off = upload(off);
    }
    P->streams.push_back(ds);
  }
  HB_CUDA(cudaDeviceSynchronize());
  P->gmax = gmax;
}

template <int MT>
static void launch_depths(FlowPlan* P, const uint2* F, uint2* x, uint2* y, uint2* xh, int R, int* err,
                          long long budget, cudaStream_t st, const std::function<void(int, bool)>& timer) {
  const int fb = (P->max_f_bytes + 15 + 127) & ~127;
  const int xb = (P->max_x_rows * R * 8 + 32 + 127) & ~127;
  const int stage = fb + xb;
  const size_t red_bytes = (size_t)FLOW_CONSUMERS * TMA_MAX_NT * MT * 4 * 2 * 32 * sizeof(float);
  const size_t smem = (size_t)FLOW_STAGES * stage + red_bytes;
  auto k = bf_step_kernel<MT>;
  HB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, nsm = 0, per_sm = 0;
  HB_CUDA(cudaGetDevice(&dev));
  HB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  HB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (FLOW_CONSUMERS + 1) * 32, smem));
  if (per_sm < 1) throw Error{HB_ERR_UNSUPPORTED, "step kernel does not fit on an SM"};
  if (P->gmax != nsm * per_sm) build_streams(P, nsm * per_sm);
  const int nd = (int)P->streams.size();
  for (int d = 0; d < nd; ++d) {
    const DepthStreams& ds = P->streams[(size_t)d];
    if (ds.grid == 0) continue;
    StepArgs args{ds.d_recs, ds.d_off, F, x, y, xh, R, stage, budget, err};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ds.grid);
    cfg.blockDim = dim3((FLOW_CONSUMERS + 1) * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    timer(d, true);
    HB_CUDA(cudaLaunchKernelEx(&cfg, k, args));
    timer(d, false);
  }
}

void flow_launch(void* plan, const uint2* F, uint2* x, uint2* y, uint2* xh, int R, int* err,
                 long long budget_cycles, cudaStream_t st, const std::function<void(int, bool)>& timer) {
  FlowPlan* P = static_cast<FlowPlan*>(plan);
  if (P->tasks.empty()) return;
  if (R <= 16) launch_depths<1>(P, F, x, y, xh, R, err, budget_cycles, st, timer);
  else if (R <= 32) launch_depths<2>(P, F, x, y, xh, R, err, budget_cycles, st, timer);
  else if (R <= 64) launch_depths<4>(P, F, x, y, xh, R, err, budget_cycles, st, timer);
  else throw Error{HB_ERR_UNSUPPORTED, "the mixed apply takes at most 64 right-hand sides per pass"};
}

}  // namespace hb
