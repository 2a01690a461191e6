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
// Work units.  A "piece" is what one shared-memory stage holds: up to
// PB_MAX factor chunks (each a contiguous run of a column-major block) and
// up to PX_MAX runs of input rows, all fetched with cp.async.bulk (1D TMA)
// on one mbarrier.  Mode 0: the chunks are independent products with their
// own outputs (e.g. the V^0 blocks of all butterflies that read the same
// leaf, or runs of neighbouring transfer blocks); mode 1: all chunks
// accumulate into one output (a leaf's dense block plus its K^L terms, or
// one large block cut into column chunks), possibly over several pieces.
//
// Scheduling.  Pieces are grouped by dependency depth (depth d only reads
// outputs of depths < d); one persistent kernel per depth, CTA b running its
// share of the depth's pieces (the pieces of one accumulating task stay on
// one CTA, in order); a producer warp streams pieces through a
// FLOW_STAGES-deep ring, NCW consumer warps compute.  Depth kernels are
// chained with programmatic dependent launch: a kernel's CTAs start as the
// previous depth drains, prefetch their first factor chunks (constant data)
// and only then wait (griddepcontrol.wait) before copying inputs the
// previous depth wrote.  Every wait is bounded by a per-thread deadline;
// past it the mapped error word is set.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "hb_internal.cuh"

namespace hb {

constexpr int NCW = 8;                  // consumer warps
constexpr int TMA_MAX_NT = 4;           // n-tiles per work item (outputs per item <= 32)
constexpr int PB_MAX = 8;               // factor chunks per piece
constexpr int PX_MAX = 8;               // input runs per piece
constexpr int FLOW_STAGES = 3;
constexpr int F_CAP = 32768;            // factor bytes per piece
constexpr int X_CAP_ROWS = 160;         // input rows per piece
constexpr int MAX_OUT = 8 * TMA_MAX_NT * NCW;   // outputs of one block / accumulating task
constexpr uint32_t IM_SIGN = 0x80000000u;       // sign bit of the imaginary (upper) bf16

struct PBlk {            // one factor chunk of a piece (32 bytes)
  long long f_off;       // element offset of the contiguous chunk
  long long y_off;       // mode 0: first output row
  int f_rows;            // stored rows (leading dimension)
  int f_cols;            // stored columns
  short xc;              // input run of this chunk
  short x_row;           // first row inside that run
  short r_out;           // mode 0: outputs
  unsigned char conj_t;  // op = ^H
  unsigned char y_buf;   // mode 0: output buffer
};

struct PXc {             // one run of input rows (16 bytes)
  long long x_off;
  int rows;
  int buf;
};

struct PRec {            // one piece, 512 bytes
  int nb, nx, mode, first_last;
  long long y_off;       // mode 1 output
  int r_out, y_buf;
  PBlk blk[PB_MAX];
  PXc xc[PX_MAX];
  unsigned char pad[512 - 32 - PB_MAX * 32 - PX_MAX * 16];
};
static_assert(sizeof(PBlk) == 32, "PBlk layout");
static_assert(sizeof(PRec) == 512, "PRec layout");

struct StageMeta {
  PRec rec;
  int f_soff[PB_MAX];    // byte offset of each chunk in the stage
  int x_soff[PX_MAX];    // byte offset of each run's first row in the stage
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

struct StepArgs {
  const PRec* recs;
  const long long* cta_off;   // pieces of CTA b: [cta_off[b], cta_off[b+1])
  const uint2* F;
  uint2* x;
  uint2* y;
  uint2* xh;
  int R;
  int stage_bytes;
  long long budget;
  int* err;
};

// One warp's share of one factor chunk: n-tiles [t0, t0 + ntl), accumulated
// into acc (MT m-tiles of 16 right-hand sides).
template <int MT>
__device__ __forceinline__ void chunk_mma(const uint2* Fs, const uint2* Xs, int f_rows, int kr, int r_out,
                                          int conj, int t0, int ntl, int R, int g, int t,
                                          float (&acc_r)[TMA_MAX_NT][MT][4], float (&acc_i)[TMA_MAX_NT][MT][4]) {
  const uint32_t cs = conj ? IM_SIGN : 0u;
  for (int kb = 0; kb < kr; kb += 8) {
    const int k0 = kb + t, k1 = kb + t + 4;
    uint32_t bh0[TMA_MAX_NT], bl0[TMA_MAX_NT], bh1[TMA_MAX_NT], bl1[TMA_MAX_NT];
#pragma unroll
    for (int j = 0; j < TMA_MAX_NT; ++j) {
      const int n = 8 * (t0 + j) + g;
      uint2 v0 = make_uint2(0u, 0u), v1 = v0;
      if (j < ntl && n < r_out) {
        if (!conj) {
          if (k0 < kr) v0 = Fs[k0 * f_rows + n];
          if (k1 < kr) v1 = Fs[k1 * f_rows + n];
        } else {
          if (k0 < kr) v0 = Fs[n * f_rows + k0];
          if (k1 < kr) v1 = Fs[n * f_rows + k1];
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
        if (j >= ntl) break;
        mma16816(acc_r[j][aa], arh, bh0[j], bh1[j]);
        mma16816(acc_r[j][aa], arh, bl0[j], bl1[j]);
        mma16816(acc_r[j][aa], arl, bh0[j], bh1[j]);
        mma16816(acc_i[j][aa], aih, bh0[j], bh1[j]);
        mma16816(acc_i[j][aa], aih, bl0[j], bl1[j]);
        mma16816(acc_i[j][aa], ail, bh0[j], bh1[j]);
      }
    }
  }
}

template <int MT>
__device__ __forceinline__ void store_tiles(uint2* out, int t0, int ntl, int r_out, int R, int g, int t,
                                            const float (&acc_r)[TMA_MAX_NT][MT][4],
                                            const float (&acc_i)[TMA_MAX_NT][MT][4]) {
#pragma unroll
  for (int j = 0; j < TMA_MAX_NT; ++j) {
    if (j >= ntl) break;
#pragma unroll
    for (int aa = 0; aa < MT; ++aa) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int mm = aa * 16 + g + ((e & 2) ? 8 : 0);
        const int n = 8 * (t0 + j) + 2 * t + (e & 1);
        if (mm < R && n < r_out) out[(size_t)n * R + mm] = to_pair(acc_r[j][aa][e], acc_i[j][aa][e]);
      }
    }
  }
}

template <int MT>
__device__ __forceinline__ void zero_acc(float (&acc_r)[TMA_MAX_NT][MT][4], float (&acc_i)[TMA_MAX_NT][MT][4]) {
#pragma unroll
  for (int j = 0; j < TMA_MAX_NT; ++j)
#pragma unroll
    for (int aa = 0; aa < MT; ++aa)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc_r[j][aa][e] = acc_i[j][aa][e] = 0.f;
}

// ------------------------------------------------------------- kernel ----
template <int MT>
__global__ void __launch_bounds__((NCW + 1) * 32, 1) bf_step_kernel(StepArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t full[FLOW_STAGES], empty[FLOW_STAGES];
  __shared__ __align__(16) StageMeta meta[FLOW_STAGES];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int R = a.R;
  auto buf = [&](int id) { return id == 0 ? a.x : (id == 1 ? a.y : a.xh); };

  if (tid == 0) {
    for (int s = 0; s < FLOW_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], NCW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const long long deadline = clock64() + a.budget;
  const long long rb = a.cta_off[blockIdx.x], npc = a.cta_off[blockIdx.x + 1] - rb;

  if (warp == NCW) {
    // ------------------------------------------------------------ producer
    // Each record (512 bytes) is read by the warp in one coalesced load; the
    // first pieces get their factor chunks (constant data) before the wait
    // for the previous depth and their input runs after it.
    bool waited = false;
    const int4* src = reinterpret_cast<const int4*>(a.recs + rb);
    int4 nxt = (npc > 0) ? src[lane] : make_int4(0, 0, 0, 0);
    for (long long i = 0; i < npc; ++i) {
      const int s = (int)(i % FLOW_STAGES);
      const int4 cur = nxt;
      if (i + 1 < npc) nxt = src[(i + 1) * 32 + lane];   // prefetch the next record
      if (i >= FLOW_STAGES) mbar_wait_until(&empty[s], (uint32_t)(((i / FLOW_STAGES) - 1) & 1), deadline, a.err);
      reinterpret_cast<int4*>(&meta[s].rec)[lane] = cur;
      __syncwarp();
      if (lane == 0) {
        StageMeta& m = meta[s];
        const PRec& r = m.rec;
        unsigned char* st = smem + (size_t)s * a.stage_bytes;
        uint32_t off = 0, total = 0;
        uint32_t fb[PB_MAX];
        for (int b = 0; b < r.nb; ++b) {
          fb[b] = (uint32_t)((r.blk[b].f_rows * r.blk[b].f_cols * 8 + 15) & ~15);
          m.f_soff[b] = (int)off;
          off += (fb[b] + 127) & ~127u;
          total += fb[b];
        }
        uint32_t xb[PX_MAX], xdst[PX_MAX];
        const char* xsrc[PX_MAX];
        for (int c = 0; c < r.nx; ++c) {
          const char* xs = reinterpret_cast<const char*>(buf(r.xc[c].buf) + (size_t)r.xc[c].x_off * R);
          const uintptr_t al = reinterpret_cast<uintptr_t>(xs) & ~(uintptr_t)15;
          const int pad = (int)(reinterpret_cast<uintptr_t>(xs) - al);
          xb[c] = (uint32_t)((pad + r.xc[c].rows * R * 8 + 15) & ~15);
          xsrc[c] = reinterpret_cast<const char*>(al);
          xdst[c] = off;
          m.x_soff[c] = (int)off + pad;
          off += (xb[c] + 127) & ~127u;
          total += xb[c];
        }
        mbar_expect_tx(&full[s], total);
        for (int b = 0; b < r.nb; ++b) tma_load_1d(st + m.f_soff[b], a.F + r.blk[b].f_off, fb[b], &full[s]);
        if (!waited) {
          asm volatile("griddepcontrol.wait;" ::: "memory");
          asm volatile("fence.proxy.async.global;" ::: "memory");
          waited = true;
        }
        for (int c = 0; c < r.nx; ++c) tma_load_1d(st + xdst[c], xsrc[c], xb[c], &full[s]);
      }
      __syncwarp();
    }
    if (lane == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    return;
  }

  // -------------------------------------------------------------- consumers
  const int g = lane >> 2, t = lane & 3;
  float acc_r[TMA_MAX_NT][MT][4];
  float acc_i[TMA_MAX_NT][MT][4];
  for (long long i = 0; i < npc; ++i) {
    const int s = (int)(i % FLOW_STAGES);
    const bool ok = mbar_wait_until(&full[s], (uint32_t)((i / FLOW_STAGES) & 1), deadline, a.err);
    const StageMeta& m = meta[s];
    const PRec& r = m.rec;
    const unsigned char* st = smem + (size_t)s * a.stage_bytes;
    const int nb = ok ? r.nb : 0;
    if (r.mode == 0) {
      // independent chunks: work items (chunk, up to ipt n-tiles) dealt to the warps
      int total_tiles = 0;
      for (int b = 0; b < nb; ++b) total_tiles += (r.blk[b].r_out + 7) >> 3;
      const int ipt = max(1, min(TMA_MAX_NT, (total_tiles + NCW - 1) / NCW));
      int item = 0;
      for (int b = 0; b < nb; ++b) {
        const PBlk& B = r.blk[b];
        const int nt = (B.r_out + 7) >> 3;
        for (int t0 = 0; t0 < nt; t0 += ipt, ++item) {
          if (item % NCW != warp) continue;
          const int ntl = min(ipt, nt - t0);
          zero_acc<MT>(acc_r, acc_i);
          const uint2* Fs = reinterpret_cast<const uint2*>(st + m.f_soff[b]);
          const uint2* Xs = reinterpret_cast<const uint2*>(st + m.x_soff[B.xc]) + (size_t)B.x_row * R;
          const int kr = B.conj_t ? B.f_rows : B.f_cols;
          chunk_mma<MT>(Fs, Xs, B.f_rows, kr, B.r_out, B.conj_t, t0, ntl, R, g, t, acc_r, acc_i);
          store_tiles<MT>(buf(B.y_buf) + (size_t)B.y_off * R, t0, ntl, B.r_out, R, g, t, acc_r, acc_i);
        }
      }
    } else {
      // every chunk accumulates into one output; warp w owns a contiguous tile range
      const int r_out = r.r_out, nt = (r_out + 7) >> 3;
      const int ipt = max(1, min(TMA_MAX_NT, (nt + NCW - 1) / NCW));
      const int t0 = warp * ipt, ntl = max(0, min(ipt, nt - t0));
      if (r.first_last & 1) zero_acc<MT>(acc_r, acc_i);
      if (ntl > 0) {
        for (int b = 0; b < nb; ++b) {
          const PBlk& B = r.blk[b];
          const uint2* Fs = reinterpret_cast<const uint2*>(st + m.f_soff[b]);
          const uint2* Xs = reinterpret_cast<const uint2*>(st + m.x_soff[B.xc]) + (size_t)B.x_row * R;
          const int kr = B.conj_t ? B.f_rows : B.f_cols;
          chunk_mma<MT>(Fs, Xs, B.f_rows, kr, r_out, B.conj_t, t0, ntl, R, g, t, acc_r, acc_i);
        }
        if (r.first_last & 2) store_tiles<MT>(buf(r.y_buf) + (size_t)r.y_off * R, t0, ntl, r_out, R, g, t, acc_r, acc_i);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);   // this warp is done with stage s
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
struct DepthStreams {
  int grid = 0;
  PRec* d_recs = nullptr;
  long long* d_off = nullptr;
};

struct FlowPlan {
  std::vector<std::vector<PRec>> depth_pieces;   // pieces per depth, in issue order
  int max_f_bytes = 16, max_x_rows = 1;
  int gmax = 0;
  std::vector<DepthStreams> streams;
};

// One chunk of a factor block (contiguous in the arena).
struct Chunk {
  long long f_off, x_off, y_off;
  int f_rows, f_cols, x_rows, r_out;
  int x_buf, y_buf, conj;
};

// Greedy piece builder for one depth.
class PieceBuilder {
 public:
  explicit PieceBuilder(std::vector<PRec>& out) : out_(out) { reset(); }

  // mode 0: an independent chunk with its own output
  void add_independent(const Chunk& c) {
    if (cur_.nb > 0 && (cur_.mode != 0 || !fits(c))) emit();
    cur_.mode = 0;
    place(c);
  }

  // mode 1: the chunks of one accumulating task (one output), possibly several pieces
  void add_task(const std::vector<Chunk>& cs, long long y_off, int r_out, int y_buf) {
    if (cur_.nb > 0) emit();
    bool first = true;
    for (const Chunk& c : cs) {
      if (cur_.nb > 0 && !fits(c)) {
        cur_.first_last = first ? 1 : 0;
        first = false;
        emit();
      }
      cur_.mode = 1;
      cur_.y_off = y_off;
      cur_.r_out = r_out;
      cur_.y_buf = y_buf;
      place(c);
    }
    cur_.first_last = (first ? 1 : 0) | 2;
    emit();
  }

  void flush() {
    if (cur_.nb > 0) emit();
  }

  int max_f = 16, max_x = 1;

 private:
  int find_run(const Chunk& c, bool& extend) const {
    for (int k = 0; k < cur_.nx; ++k) {
      const PXc& r = cur_.xc[k];
      if (r.buf != c.x_buf) continue;
      if (c.x_off >= r.x_off && c.x_off + c.x_rows <= r.x_off + r.rows) {
        extend = false;
        return k;
      }
      if (c.x_off == r.x_off + r.rows) {
        extend = true;
        return k;
      }
    }
    return -1;
  }

  bool fits(const Chunk& c) const {
    if (cur_.nb >= PB_MAX) return false;
    if (fbytes_ + c.f_rows * c.f_cols * 8 > F_CAP) return false;
    bool extend = false;
    const int k = find_run(c, extend);
    if (k < 0 && cur_.nx >= PX_MAX) return false;
    const int add = (k < 0 || extend) ? c.x_rows : 0;
    return xrows_ + add <= X_CAP_ROWS;
  }

  void place(const Chunk& c) {
    bool extend = false;
    int k = find_run(c, extend);
    if (k < 0) {
      k = cur_.nx++;
      cur_.xc[k].x_off = c.x_off;
      cur_.xc[k].rows = c.x_rows;
      cur_.xc[k].buf = c.x_buf;
      xrows_ += c.x_rows;
    } else if (extend) {
      cur_.xc[k].rows += c.x_rows;
      xrows_ += c.x_rows;
    }
    PBlk& b = cur_.blk[cur_.nb++];
    b.f_off = c.f_off;
    b.y_off = c.y_off;
    b.f_rows = c.f_rows;
    b.f_cols = c.f_cols;
    b.xc = (short)k;
    b.x_row = (short)(c.x_off - cur_.xc[k].x_off);
    b.r_out = (short)c.r_out;
    b.conj_t = (unsigned char)c.conj;
    b.y_buf = (unsigned char)c.y_buf;
    fbytes_ += c.f_rows * c.f_cols * 8;
  }

  void emit() {
    max_f = std::max(max_f, fbytes_);
    max_x = std::max(max_x, xrows_);
    out_.push_back(cur_);
    reset();
  }

  void reset() {
    std::memset(&cur_, 0, sizeof(cur_));
    fbytes_ = 0;
    xrows_ = 0;
  }

  std::vector<PRec>& out_;
  PRec cur_;
  int fbytes_ = 0, xrows_ = 0;
};

// Cut one logical task into chunks.  Forward: column chunks of <= kc inputs
// (one accumulating task unless it is a single chunk).  ^H: column chunks
// of <= oc outputs of the stored blocks; with one term every chunk is an
// independent product.
static void task_chunks(const FlowTask& L, std::vector<std::vector<Chunk>>& groups, bool& independent) {
  const bool conj = !L.terms.empty() && L.terms[0].conj_t;
  groups.clear();
  if (!conj) {
    if (L.r_out > MAX_OUT) throw Error{HB_ERR_UNSUPPORTED, "a factor block has more than 256 rows"};
    const int kc = std::max(2, std::min(X_CAP_ROWS / 2, (F_CAP / 2 / (8 * std::max(1, L.r_out))) & ~1));
    std::vector<Chunk> cs;
    for (const FlowTerm& tm : L.terms)
      for (int j0 = 0; j0 < tm.r_in; j0 += kc) {
        Chunk c{};
        c.f_off = tm.f_off + (long long)j0 * tm.f_rows;
        c.f_rows = tm.f_rows;
        c.f_cols = std::min(kc, tm.r_in - j0);
        c.x_off = tm.x_off + j0;
        c.x_rows = c.f_cols;
        c.x_buf = tm.x_buf;
        c.conj = 0;
        c.r_out = L.r_out;
        c.y_off = L.y_off;
        c.y_buf = L.y_buf;
        cs.push_back(c);
      }
    independent = (cs.size() == 1);
    groups.push_back(cs);
  } else {
    int rmax = 1;
    for (const FlowTerm& tm : L.terms) rmax = std::max(rmax, tm.r_in);
    if (rmax > X_CAP_ROWS) throw Error{HB_ERR_UNSUPPORTED, "an adjoint factor block has too many rows"};
    const int oc = std::min(MAX_OUT, std::max(8, (F_CAP / 2 / (8 * rmax)) & ~7));
    independent = (L.terms.size() == 1);
    for (int n0 = 0; n0 < L.r_out; n0 += oc) {
      std::vector<Chunk> cs;
      const int w = std::min(oc, L.r_out - n0);
      for (const FlowTerm& tm : L.terms) {
        Chunk c{};
        c.f_off = tm.f_off + (long long)n0 * tm.f_rows;
        c.f_rows = tm.f_rows;
        c.f_cols = w;
        c.x_off = tm.x_off;
        c.x_rows = tm.r_in;
        c.x_buf = tm.x_buf;
        c.conj = 1;
        c.r_out = w;
        c.y_off = L.y_off + n0;
        c.y_buf = L.y_buf;
        cs.push_back(c);
      }
      groups.push_back(cs);
    }
  }
}

void flow_plan_build(const std::vector<FlowTask>& lt, void** plan_out) {
  FlowPlan* P = new FlowPlan();
  try {
    int maxd = -1;
    for (const FlowTask& L : lt) maxd = std::max(maxd, L.depth);
    P->depth_pieces.assign((size_t)(maxd + 1), {});
    std::vector<std::vector<Chunk>> groups;
    for (int d = 0; d <= maxd; ++d) {
      std::vector<Chunk> indep;
      std::vector<std::vector<Chunk>> accum;
      for (const FlowTask& L : lt) {
        if (L.depth != d) continue;
        bool ind = false;
        task_chunks(L, groups, ind);
        for (auto& cs : groups) {
          if (ind && cs.size() == 1) indep.push_back(cs[0]);
          else accum.push_back(cs);
        }
      }
      // chunks that read the same or neighbouring input rows meet in one piece
      std::stable_sort(indep.begin(), indep.end(), [](const Chunk& a, const Chunk& b) {
        if (a.x_buf != b.x_buf) return a.x_buf < b.x_buf;
        return a.x_off < b.x_off;
      });
      PieceBuilder pb(P->depth_pieces[(size_t)d]);
      for (const Chunk& c : indep) pb.add_independent(c);
      pb.flush();
      for (const auto& cs : accum) pb.add_task(cs, cs[0].y_off, cs[0].r_out, cs[0].y_buf);
      P->max_f_bytes = std::max(P->max_f_bytes, pb.max_f);
      P->max_x_rows = std::max(P->max_x_rows, pb.max_x);
    }
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

int flow_plan_depths(const void* plan) { return (int)static_cast<const FlowPlan*>(plan)->depth_pieces.size(); }

// Per-CTA piece streams of every depth for a maximum grid of gmax CTAs; the
// pieces of one accumulating task stay together, in order, on one CTA.
static void build_streams(FlowPlan* P, int gmax) {
  for (DepthStreams& d : P->streams) {
    dev_free(d.d_recs);
    dev_free(d.d_off);
  }
  P->streams.clear();
  for (const std::vector<PRec>& pcs : P->depth_pieces) {
    std::vector<std::vector<size_t>> units;
    for (size_t q = 0; q < pcs.size(); ++q) {
      if (pcs[q].mode == 1 && !(pcs[q].first_last & 1) && !units.empty()) units.back().push_back(q);
      else units.push_back({q});
    }
    DepthStreams ds;
    ds.grid = std::min<int>(gmax, (int)units.size());
    std::vector<PRec> recs;
    std::vector<long long> off;
    for (int b = 0; b < ds.grid; ++b) {
      off.push_back((long long)recs.size());
      for (size_t u = (size_t)b; u < units.size(); u += (size_t)ds.grid)
        for (size_t q : units[u]) recs.push_back(pcs[q]);
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
  // stage: every factor chunk and input run rounded up to 16 and placed 128-byte
  // aligned (at most 143 bytes of slack each), runs with a head pad below 16 bytes
  const int stage = (P->max_f_bytes + P->max_x_rows * R * 8 + (PB_MAX + PX_MAX) * 160 + 127) & ~127;
  const size_t smem = (size_t)FLOW_STAGES * stage;
  auto k = bf_step_kernel<MT>;
  HB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, nsm = 0, per_sm = 0;
  HB_CUDA(cudaGetDevice(&dev));
  HB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  HB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (NCW + 1) * 32, smem));
  if (per_sm < 1) throw Error{HB_ERR_UNSUPPORTED, "step kernel does not fit on an SM"};
  if (P->gmax != nsm * per_sm) build_streams(P, nsm * per_sm);
  const int nd = (int)P->streams.size();
  for (int d = 0; d < nd; ++d) {
    const DepthStreams& ds = P->streams[(size_t)d];
    if (ds.grid == 0) continue;
    StepArgs args{ds.d_recs, ds.d_off, F, x, y, xh, R, stage, budget, err};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ds.grid);
    cfg.blockDim = dim3((NCW + 1) * 32);
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
  if (P->depth_pieces.empty()) return;
  if (R <= 16) launch_depths<1>(P, F, x, y, xh, R, err, budget_cycles, st, timer);
  else if (R <= 32) launch_depths<2>(P, F, x, y, xh, R, err, budget_cycles, st, timer);
  else if (R <= 64) launch_depths<4>(P, F, x, y, xh, R, err, budget_cycles, st, timer);
  else throw Error{HB_ERR_UNSUPPORTED, "the mixed apply takes at most 64 right-hand sides per pass"};
}

}  // namespace hb
