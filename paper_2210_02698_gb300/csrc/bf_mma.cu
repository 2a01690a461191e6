// bf_mma.cu - mixed-precision butterfly apply on the tensor cores
// (Sec. 4.2.1, Eq. butterfly_mat: every factor level is a batch of small
// dense complex products Y = op(F) X; Sec. 4.2 HODBF sum).
//
// Numbers.  Every complex value a is a split-BF16 pair {hi, lo} (8 bytes):
// hi = bf16x2(Re a, Im a), lo = bf16x2 of the remainders a - hi, so hi + lo
// keeps ~16 significant bits.  Products are
//     a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi          (split BF16 x 3)
// with FP32 accumulation (mma.sync m16n8k16), split again when stored.
//
// Complex -> real.  With k' = 2k + c interleaving real/imaginary parts,
//     D_r[m][n] = sum_k' A_r[m][k'] B[k'][n],   D_i[m][n] = sum_k' A_i[m][k'] B[k'][n]
//     A_r[m][(2k,2k+1)] = (Re X[k][m], -Im X[k][m]),  A_i[m][(2k,2k+1)] = (Im X[k][m], Re X[k][m])
//     B[(2k,2k+1)][n]   = (Re F[n][k], Im F[n][k])
// so a B register is a stored pair, an A_r register the X pair with the
// imaginary sign flipped, an A_i register the X pair with its halves
// swapped.  M = 16 right-hand sides (an m-tile), N = 8 outputs (an n-tile),
// K = 8 complex inputs (a k-step).
//
// Native layout.  Factors and vectors live in HBM in the order the MMA
// fragments want them, so that every fragment is one conflict-free 16-byte
// shared-memory load per lane and no index is ever checked:
//   * the k-slots t and t + 4 of lane (g, t) carry input rows 2t and 2t + 1
//     of the k-step (any fixed order of k works; this one makes the
//     accumulator of one step the A fragment of the next);
//   * factor tile (k-step, n-tile) = 32 lanes x uint4
//       {hi(F[n][2t]), hi(F[n][2t+1]), lo(F[n][2t]), lo(F[n][2t+1])},  n = g;
//     tiles of a block ordered [k-step][n-tile]; the adjoint has its own
//     arena holding F^H, so both directions run the same code;
//   * vector tile (8 rows x 16 right-hand sides) = 32 lanes x uint4 of hi
//     words, then 32 x uint4 of lo words, word j of lane (g, t) holding
//     (row 2t + (j >> 1), right-hand side g + 8 (j & 1)); a buffer is
//     [row tile][m-tile] of such tiles.
// Rows of every block part (a leaf, a skeleton) are padded to a multiple of
// 8 with zeros; padded rows of the vectors stay exactly zero.
//
// Work units.  A "piece" is what one shared-memory stage holds: up to
// PB_MAX factor chunks (a run of k-steps of one block, contiguous in the
// arena) and up to PX_MAX runs of input row tiles, fetched with
// cp.async.bulk (1D TMA) on one mbarrier.  Mode 0: the chunks are
// independent products with their own outputs (e.g. the V^0 blocks that
// read the same leaf); mode 1: all chunks accumulate into one output (a
// leaf's dense block plus its K^L terms, or one large block cut into
// k-chunks), possibly over several pieces.
//
// Scheduling.  Pieces are grouped by dependency depth (depth d only reads
// outputs of depths < d); one persistent kernel per depth, CTA b running its
// share of the depth's pieces (the pieces of one accumulating task stay on
// one CTA, in order); a producer warp streams pieces through a ring of
// stages, NCW consumer warps compute.  Depth kernels are chained with
// programmatic dependent launch: a kernel's CTAs prefetch their first factor
// chunks (constant data) and only then wait (griddepcontrol.wait) before
// copying inputs the previous depth wrote.  Every wait is bounded by a
// per-thread deadline; past it the mapped error word is set.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "hb_internal.cuh"

namespace hb {

// Ring geometry (compile-time; the defaults are the tuned values).
#ifndef HB_FLOW_NCW
#define HB_FLOW_NCW 8
#endif
#ifndef HB_FLOW_TILES_PER_WARP
#define HB_FLOW_TILES_PER_WARP 8
#endif
#ifndef HB_FLOW_F_CAP
#define HB_FLOW_F_CAP 96
#endif
#ifndef HB_FLOW_X_CAP
#define HB_FLOW_X_CAP 24
#endif
#ifndef HB_FLOW_MAX_STAGES
#define HB_FLOW_MAX_STAGES 4
#endif
#ifndef HB_FLOW_PIECES_PER_SM
#define HB_FLOW_PIECES_PER_SM 0
#endif
constexpr int NCW = HB_FLOW_NCW;                   // consumer warps
constexpr int PB_MAX = 8;                          // factor chunks per piece
constexpr int PX_MAX = 8;                          // input runs per piece
constexpr int MAX_STAGES = HB_FLOW_MAX_STAGES;
constexpr int F_CAP_TILES = HB_FLOW_F_CAP;         // factor tiles (512 bytes) per piece
constexpr int X_CAP_TILES = HB_FLOW_X_CAP;         // input row tiles per piece
constexpr int PIECES_PER_SM = HB_FLOW_PIECES_PER_SM;   // > 0: smaller pieces for small depths
constexpr int MAX_NT = 32;                         // n-tiles of one output (256 rows)
constexpr uint32_t IM_SIGN = 0x80000000u;   // sign bit of the imaginary (upper) bf16

// A piece record (1 KB); the host planner precomputes everything in it.
// copies: one cp.async.bulk each into the stage: a factor chunk (buf 3) to
// stage byte dst, an input run (buf 0..2 = x, y, xh) to the input region,
// row tile dst (the input region starts at f_bytes; an input row tile is
// MT KB).  items: consumer warp w runs items [wbeg[w], wbeg[w + 1]).
struct PCopy {           // 16 bytes
  long long src;         // first factor tile / first vector row tile
  int dst;
  int tiles_buf;         // tiles | buf << 28
};

struct PItem {           // 24 bytes: ks k-steps x ntl n-tiles of one block
  long long y_tile;      // first output row tile
  int f_soff;            // stage byte offset of the item's first factor tile
  int x_t;               // first input row tile in the input region
  short ks;
  short f_stride;        // n-tiles of the block (tiles between k-steps)
  unsigned char ntl;
  unsigned char y_buf;
  unsigned char flags;   // 1: zero the accumulators first, 2: store them after
  unsigned char pad;
};

constexpr int MAX_COPIES = 16, MAX_ITEMS = 30;
struct PRec {
  int ncopy;
  int f_bytes;           // factor region of the stage
  int x_tiles;           // input row tiles after it
  int pad0;
  unsigned char wbeg[32];
  PCopy cp[MAX_COPIES];
  PItem it[MAX_ITEMS];
};
static_assert(sizeof(PCopy) == 16 && sizeof(PItem) == 24 && sizeof(PRec) == 1024, "record layout");
static_assert(NCW < 32 && PB_MAX + PX_MAX <= MAX_COPIES, "record capacity");

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
  const uint4* F;
  uint4* x;
  uint4* y;
  uint4* xh;
  int stages;
  int stage_bytes;
  long long budget;
  int* err;
};

// n-tiles per warp item (the accumulators take 8 NTW MT registers)
template <int MT>
struct Tiles {
  static constexpr int NTW = HB_FLOW_TILES_PER_WARP / MT;
};
static_assert(NCW * HB_FLOW_TILES_PER_WARP / 2 >= MAX_NT, "an accumulating task must fit the consumer warps");

// Accumulate ks k-steps of a chunk into acc: n-tiles [t0, t0 + NTL) of a
// block with nt n-tiles (Fs: its first k-step), input tiles Xs.  NTL is a
// compile-time count so that no MMA slot is issued for an absent tile.
template <int MT, int NTL>
__device__ __forceinline__ void chunk_mma_n(const uint4* __restrict__ Fs, const uint4* __restrict__ Xs, int nt,
                                            int ks, int t0, int lane, float (&acc)[Tiles<MT>::NTW][MT][8]) {
  const uint4* fp = Fs + t0 * 32 + lane;
  const uint4* xp = Xs + lane;
  for (int k = 0; k < ks; ++k, fp += nt * 32, xp += MT * 64) {
    uint4 b[NTL];
#pragma unroll
    for (int j = 0; j < NTL; ++j) b[j] = fp[j * 32];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const uint4 h = xp[mt * 64], l = xp[mt * 64 + 32];
      const uint32_t arh[4] = {h.x ^ IM_SIGN, h.y ^ IM_SIGN, h.z ^ IM_SIGN, h.w ^ IM_SIGN};
      const uint32_t arl[4] = {l.x ^ IM_SIGN, l.y ^ IM_SIGN, l.z ^ IM_SIGN, l.w ^ IM_SIGN};
      const uint32_t aih[4] = {__byte_perm(h.x, 0, 0x1032), __byte_perm(h.y, 0, 0x1032),
                               __byte_perm(h.z, 0, 0x1032), __byte_perm(h.w, 0, 0x1032)};
      const uint32_t ail[4] = {__byte_perm(l.x, 0, 0x1032), __byte_perm(l.y, 0, 0x1032),
                               __byte_perm(l.z, 0, 0x1032), __byte_perm(l.w, 0, 0x1032)};
#pragma unroll
      for (int j = 0; j < NTL; ++j) {
        float* ar = acc[j][mt];
        float* ai = acc[j][mt] + 4;
        mma16816(ar, arh, b[j].x, b[j].y);
        mma16816(ar, arh, b[j].z, b[j].w);
        mma16816(ar, arl, b[j].x, b[j].y);
        mma16816(ai, aih, b[j].x, b[j].y);
        mma16816(ai, aih, b[j].z, b[j].w);
        mma16816(ai, ail, b[j].x, b[j].y);
      }
    }
  }
}

template <int MT>
__device__ __forceinline__ void chunk_mma(const uint4* __restrict__ Fs, const uint4* __restrict__ Xs, int nt,
                                          int ks, int t0, int ntl, int lane,
                                          float (&acc)[Tiles<MT>::NTW][MT][8]) {
  switch (ntl) {
    case 1: chunk_mma_n<MT, 1>(Fs, Xs, nt, ks, t0, lane, acc); break;
    case 2: chunk_mma_n<MT, 2>(Fs, Xs, nt, ks, t0, lane, acc); break;
    case 3: chunk_mma_n<MT, 3>(Fs, Xs, nt, ks, t0, lane, acc); break;
    case 4: chunk_mma_n<MT, 4>(Fs, Xs, nt, ks, t0, lane, acc); break;
    default:
      if constexpr (Tiles<MT>::NTW > 4) {
        switch (ntl) {
          case 5: chunk_mma_n<MT, 5>(Fs, Xs, nt, ks, t0, lane, acc); break;
          case 6: chunk_mma_n<MT, 6>(Fs, Xs, nt, ks, t0, lane, acc); break;
          case 7: chunk_mma_n<MT, 7>(Fs, Xs, nt, ks, t0, lane, acc); break;
          case 8: chunk_mma_n<MT, 8>(Fs, Xs, nt, ks, t0, lane, acc); break;
          default: break;
        }
      }
      break;
  }
}

// Store n-tiles [t0, t0 + ntl) of the accumulators as vector tiles at Y.
// Accumulator element e of lane (g, t) is (right-hand side g + 8 (e >> 1),
// output 2t + (e & 1)); vector word j holds (row 2t + (j >> 1), right-hand
// side g + 8 (j & 1)), so words (0, 1, 2, 3) = elements (0, 2, 1, 3).
template <int MT>
__device__ __forceinline__ void store_tiles(uint4* Y, int t0, int ntl, int lane,
                                            const float (&acc)[Tiles<MT>::NTW][MT][8]) {
  constexpr int NTW = Tiles<MT>::NTW;
#pragma unroll
  for (int j = 0; j < NTW; ++j) {
    if (j >= ntl) break;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const float* a = acc[j][mt];
      const uint2 p0 = to_pair(a[0], a[4]), p1 = to_pair(a[1], a[5]);
      const uint2 p2 = to_pair(a[2], a[6]), p3 = to_pair(a[3], a[7]);
      uint4* o = Y + ((size_t)(t0 + j) * MT + mt) * 64;
      o[lane] = make_uint4(p0.x, p2.x, p1.x, p3.x);
      o[32 + lane] = make_uint4(p0.y, p2.y, p1.y, p3.y);
    }
  }
}

template <int MT>
__device__ __forceinline__ void zero_acc(float (&acc)[Tiles<MT>::NTW][MT][8]) {
#pragma unroll
  for (int j = 0; j < Tiles<MT>::NTW; ++j)
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[j][mt][e] = 0.f;
}

// ------------------------------------------------------------- kernel ----
template <int MT>
__global__ void __launch_bounds__((NCW + 1) * 32, 1) bf_step_kernel(StepArgs a) {
  constexpr int NTW = Tiles<MT>::NTW;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t full[MAX_STAGES], empty[MAX_STAGES];
  __shared__ __align__(16) PRec meta[MAX_STAGES];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nst = a.stages;
  auto buf = [&](int id) { return id == 0 ? a.x : (id == 1 ? a.y : a.xh); };

  if (tid == 0) {
    for (int s = 0; s < nst; ++s) {
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
    // The warp loads each record (1 KB) with two coalesced loads, one lane
    // per copy issues the copies; factor chunks (constant data) of the first
    // piece go out before the wait for the previous depth, input runs after.
    bool waited = false;
    const int4* src = reinterpret_cast<const int4*>(a.recs + rb);
    int4 n0 = make_int4(0, 0, 0, 0), n1 = n0;
    if (npc > 0) {
      n0 = src[lane];
      n1 = src[32 + lane];
    }
    for (long long i = 0; i < npc; ++i) {
      const int s = (int)(i % nst);
      const int4 c0 = n0, c1 = n1;
      if (i + 1 < npc) {   // prefetch the next record
        n0 = src[(i + 1) * 64 + lane];
        n1 = src[(i + 1) * 64 + 32 + lane];
      }
      if (i >= nst) mbar_wait_until(&empty[s], (uint32_t)(((i / nst) - 1) & 1), deadline, a.err);
      int4* m = reinterpret_cast<int4*>(&meta[s]);
      m[lane] = c0;
      m[32 + lane] = c1;
      __syncwarp();
      const PRec& r = meta[s];
      const int f_bytes = r.f_bytes;
      if (lane == 0) mbar_expect_tx(&full[s], (uint32_t)f_bytes + (uint32_t)r.x_tiles * (uint32_t)(MT * 1024));
      __syncwarp();
      unsigned char* st = smem + (size_t)s * a.stage_bytes;
      const bool mine = lane < r.ncopy;
      PCopy c{};
      if (mine) c = r.cp[lane];
      const int bid = c.tiles_buf >> 28, tiles = c.tiles_buf & 0x0fffffff;
      if (mine && bid == 3) tma_load_1d(st + c.dst, a.F + c.src * 32, (uint32_t)tiles * 512u, &full[s]);
      if (!waited) {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        asm volatile("fence.proxy.async.global;" ::: "memory");
        waited = true;
      }
      if (mine && bid < 3)
        tma_load_1d(st + f_bytes + (size_t)c.dst * (MT * 1024), buf(bid) + c.src * (MT * 64),
                    (uint32_t)tiles * (uint32_t)(MT * 1024), &full[s]);
      __syncwarp();
    }
    if (lane == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    return;
  }

  // -------------------------------------------------------------- consumers
  float acc[NTW][MT][8];
  zero_acc<MT>(acc);
  for (long long i = 0; i < npc; ++i) {
    const int s = (int)(i % nst);
    const bool ok = mbar_wait_until(&full[s], (uint32_t)((i / nst) & 1), deadline, a.err);
    const PRec& r = meta[s];
    const unsigned char* st = smem + (size_t)s * a.stage_bytes;
    const uint4* xr = reinterpret_cast<const uint4*>(st + r.f_bytes);
    const int e1 = ok ? r.wbeg[warp + 1] : 0;
    for (int e = r.wbeg[warp]; e < e1; ++e) {
      const PItem& it = r.it[e];
      const int flags = it.flags, ntl = it.ntl, ks = it.ks;
      if (flags & 1) zero_acc<MT>(acc);
      if (ks > 0)
        chunk_mma<MT>(reinterpret_cast<const uint4*>(st + it.f_soff), xr + (size_t)it.x_t * (MT * 64), it.f_stride,
                      ks, 0, ntl, lane, acc);
      if (flags & 2) store_tiles<MT>(buf(it.y_buf) + (size_t)it.y_tile * (MT * 64), 0, ntl, lane, acc);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);   // this warp is done with stage s
  }
}

// --------------------------------------------------- conversions / I/O ----
__device__ __forceinline__ int part_index(int pos, int r1, int r2) {
  const int p1 = (r1 + 7) & ~7;
  if (pos < p1) return pos < r1 ? pos : -1;
  return (pos - p1 < r2) ? r1 + pos - p1 : -1;
}

// One CTA per native block: tile (k-step, n-tile), lane (g, t) ->
// {hi F[n][2t], hi F[n][2t+1], lo F[n][2t], lo F[n][2t+1]} with n = 8 n-tile + g.
__global__ void nat_convert_kernel(const double2* __restrict__ F, const NatBlock* __restrict__ blocks,
                                   uint4* __restrict__ out) {
  const NatBlock B = blocks[blockIdx.x];
  const int nt = (B.r1 + 7) / 8 + (B.r2 + 7) / 8, ks = (B.k1 + 7) / 8 + (B.k2 + 7) / 8;
  for (int idx = threadIdx.x; idx < nt * ks * 32; idx += blockDim.x) {
    const int tile = idx >> 5, lane = idx & 31, g = lane >> 2, t = lane & 3;
    const int kstep = tile / nt, ntile = tile % nt;
    const int n = part_index(8 * ntile + g, B.r1, B.r2);
    uint2 p[2];
    for (int h = 0; h < 2; ++h) {
      const int k = part_index(8 * kstep + 2 * t + h, B.k1, B.k2);
      double re = 0, im = 0;
      if (n >= 0 && k >= 0) {
        if (B.conj) {
          const double2 v = F[B.src_off + k + (long long)n * B.ld];
          re = v.x;
          im = -v.y;
        } else {
          const double2 v = F[B.src_off + n + (long long)k * B.ld];
          re = v.x;
          im = v.y;
        }
      }
      p[h] = to_pair((float)re, (float)im);
    }
    out[(B.tile0 + tile) * 32 + lane] = make_uint4(p[0].x, p[1].x, p[0].y, p[1].y);
  }
}

void nat_convert(const double2* F64, const std::vector<NatBlock>& blocks, uint4* out, cudaStream_t st) {
  if (blocks.empty()) return;
  NatBlock* d = upload(blocks, st);
  for (size_t b0 = 0; b0 < blocks.size(); b0 += (1u << 30)) {
    const unsigned n = (unsigned)std::min<size_t>(blocks.size() - b0, 1u << 30);
    nat_convert_kernel<<<n, 128, 0, st>>>(F64, d + b0, out);
    HB_CHECK_LAUNCH();
  }
  HB_CUDA(cudaStreamSynchronize(st));
  dev_free(d);
}

// Vector word w of tile (row tile rt, m-tile mt): lane = w >> 2, j = w & 3,
// row 8 rt + 2 (lane & 3) + (j >> 1), right-hand side 16 mt + (lane >> 2) + 8 (j & 1).
__device__ __forceinline__ void word_coords(long long q, int MT, long long& rt, int& mt, int& w, long long& row,
                                            int& rhs) {
  w = (int)(q & 127);
  const long long tm = q >> 7;
  rt = tm / MT;
  mt = (int)(tm - rt * MT);
  const int ln = w >> 2, j = w & 3;
  row = 8 * rt + 2 * (ln & 3) + (j >> 1);
  rhs = 16 * mt + (ln >> 2) + 8 * (j & 1);
}

// x (native) = pair(scale * s[rhs * Nv + natural index of the padded row])
__global__ void gather_native_kernel(const double2* __restrict__ s, const long long* __restrict__ pperm,
                                     uint32_t* __restrict__ x, long long nv_tiles, long long Nv, int R, int MT,
                                     double scale) {
  const long long total = nv_tiles * MT * 128;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    long long rt, row;
    int mt, w, rhs;
    word_coords(q, MT, rt, mt, w, row, rhs);
    const long long nat = pperm[row];
    double2 v = make_double2(0.0, 0.0);
    if (nat >= 0 && rhs < R) v = s[(size_t)rhs * Nv + nat];
    const uint2 p = to_pair((float)(v.x * scale), (float)(v.y * scale));
    uint32_t* tile = x + (rt * MT + mt) * 256;
    tile[w] = p.x;
    tile[128 + w] = p.y;
  }
}

__global__ void scatter_native_kernel(const uint32_t* __restrict__ y, const long long* __restrict__ pperm,
                                      double2* __restrict__ u, long long nv_tiles, long long Nv, int R, int MT) {
  const long long total = nv_tiles * MT * 128;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    long long rt, row;
    int mt, w, rhs;
    word_coords(q, MT, rt, mt, w, row, rhs);
    const long long nat = pperm[row];
    if (nat < 0 || rhs >= R) continue;
    const uint32_t* tile = y + (rt * MT + mt) * 256;
    const uint32_t hi = tile[w], lo = tile[128 + w];
    const double re = (double)__uint_as_float(hi << 16) + (double)__uint_as_float(lo << 16);
    const double im = (double)__uint_as_float(hi & 0xffff0000u) + (double)__uint_as_float(lo & 0xffff0000u);
    u[(size_t)rhs * Nv + nat] = make_double2(re, im);
  }
}

void gather_native(const double2* s, const long long* pperm, uint4* x, long long nv_tiles, long long Nv, int R,
                   int MT, double scale, cudaStream_t st) {
  const long long total = nv_tiles * MT * 128;
  const int grid = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 152LL * 16));
  gather_native_kernel<<<grid, 256, 0, st>>>(s, pperm, reinterpret_cast<uint32_t*>(x), nv_tiles, Nv, R, MT, scale);
  HB_CHECK_LAUNCH();
}

void scatter_native(const uint4* y, const long long* pperm, double2* u, long long nv_tiles, long long Nv, int R,
                    int MT, cudaStream_t st) {
  const long long total = nv_tiles * MT * 128;
  const int grid = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 152LL * 16));
  scatter_native_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const uint32_t*>(y), pperm, u, nv_tiles, Nv, R,
                                              MT);
  HB_CHECK_LAUNCH();
}

// ------------------------------------------------------------- planning ----
// One chunk: ks k-steps of a block (contiguous tiles), its input row tiles.
struct Chunk {
  long long f_tile, x_tile, y_tile;
  int nt, ks, x_buf, y_buf;
};

struct Run {
  long long x_tile;
  int tiles, buf;
};

// A piece as the builder forms it; encoded into a PRec for a given MT when
// the launch streams are set up.
struct HostPiece {
  int mode = 0, first_last = 0;
  std::vector<Chunk> ch;
  std::vector<int> ch_run, ch_xt;   // input run of each chunk (-1: none), first tile inside it
  std::vector<Run> runs;
  int ftiles = 0, xtiles = 0;
};

struct DepthStreams {
  int grid = 0;
  PRec* d_recs = nullptr;
  long long* d_off = nullptr;
};

struct FlowPlan {
  std::vector<std::vector<HostPiece>> depth_pieces;   // pieces per depth, in issue order
  int max_f_tiles = 1, max_x_tiles = 1;
  int gmax[3] = {0, 0, 0};                            // per MT
  std::vector<DepthStreams> streams[3];
};

constexpr int NTW_MIN = HB_FLOW_TILES_PER_WARP / 2;   // n-tiles per item at MT = 2

// n-tiles per item: mode 0 spreads the piece's n-tiles over the warps,
// mode 1 gives warp g the n-tiles [g ipt, (g + 1) ipt) of the one output.
static int mode0_ipt(const std::vector<Chunk>& ch, int ntw) {
  int total = 0;
  for (const Chunk& c : ch) total += c.nt;
  return std::max(1, std::min(ntw, (total + NCW - 1) / NCW));
}
static int mode1_ipt(int nt) { return std::max(1, (nt + NCW - 1) / NCW); }

static int count_items(const std::vector<Chunk>& ch, int mode, int ntw) {
  if (ch.empty()) return 0;
  if (mode == 0) {
    const int ipt = mode0_ipt(ch, ntw);
    int n = 0;
    for (const Chunk& c : ch) n += (c.nt + ipt - 1) / ipt;
    return n;
  }
  const int ipt = mode1_ipt(ch[0].nt);
  return (int)ch.size() * ((ch[0].nt + ipt - 1) / ipt);
}

// Greedy piece builder for one depth.
class PieceBuilder {
 public:
  PieceBuilder(std::vector<HostPiece>& out, int f_cap) : out_(out), f_cap_(f_cap) {}

  // mode 0: an independent chunk with its own output
  void add_independent(const Chunk& c) {
    if (!cur_.ch.empty() && (cur_.mode != 0 || !fits(c, 0))) emit();
    cur_.mode = 0;
    place(c);
  }

  // mode 1: the chunks of one accumulating task (one output), possibly several pieces
  void add_task(const std::vector<Chunk>& cs) {
    if (!cur_.ch.empty()) emit();
    bool first = true;
    for (const Chunk& c : cs) {
      if (!cur_.ch.empty() && !fits(c, 1)) {
        cur_.first_last = first ? 1 : 0;
        first = false;
        emit();
      }
      cur_.mode = 1;
      place(c);
    }
    cur_.first_last = (first ? 1 : 0) | 2;
    emit();
  }

  void flush() {
    if (!cur_.ch.empty()) emit();
  }

  int max_f = 1, max_x = 1;

 private:
  int find_run(const Chunk& c, bool& extend) const {
    for (size_t k = 0; k < cur_.runs.size(); ++k) {
      const Run& r = cur_.runs[k];
      if (r.buf != c.x_buf) continue;
      if (c.x_tile >= r.x_tile && c.x_tile + c.ks <= r.x_tile + r.tiles) {
        extend = false;
        return (int)k;
      }
      if (c.x_tile == r.x_tile + r.tiles) {
        extend = true;
        return (int)k;
      }
    }
    return -1;
  }

  bool fits(const Chunk& c, int mode) const {
    if ((int)cur_.ch.size() >= PB_MAX) return false;
    if (cur_.ftiles + c.nt * c.ks > f_cap_) return false;
    std::vector<Chunk> t = cur_.ch;
    t.push_back(c);
    if (count_items(t, mode, NTW_MIN) > MAX_ITEMS) return false;
    if (c.ks == 0) return true;
    bool extend = false;
    const int k = find_run(c, extend);
    if (k < 0 && (int)cur_.runs.size() >= PX_MAX) return false;
    const int add = (k < 0 || extend) ? c.ks : 0;
    return cur_.xtiles + add <= X_CAP_TILES;
  }

  void place(const Chunk& c) {
    int k = -1, xt = 0;
    if (c.ks > 0) {
      bool extend = false;
      k = find_run(c, extend);
      if (k < 0) {
        k = (int)cur_.runs.size();
        cur_.runs.push_back(Run{c.x_tile, c.ks, c.x_buf});
        cur_.xtiles += c.ks;
      } else if (extend) {
        cur_.runs[(size_t)k].tiles += c.ks;
        cur_.xtiles += c.ks;
      }
      xt = (int)(c.x_tile - cur_.runs[(size_t)k].x_tile);
    }
    cur_.ch.push_back(c);
    cur_.ch_run.push_back(k);
    cur_.ch_xt.push_back(xt);
    cur_.ftiles += c.nt * c.ks;
  }

  void emit() {
    max_f = std::max(max_f, cur_.ftiles);
    max_x = std::max(max_x, cur_.xtiles);
    out_.push_back(std::move(cur_));
    cur_ = HostPiece();
  }

  std::vector<HostPiece>& out_;
  int f_cap_;
  HostPiece cur_;
};

// The record of a piece for MT m-tiles: stage layout, copies, and the items
// of every consumer warp (mode 0: largest item first to the least-loaded
// warp; mode 1: warp g owns n-tile group g across all pieces of the task).
static void encode(const HostPiece& p, int MT, PRec& r) {
  std::memset(&r, 0, sizeof r);
  const int ntw = HB_FLOW_TILES_PER_WARP / MT;
  std::vector<int> f_soff(p.ch.size()), run_off(p.runs.size());
  int off = 0, nc = 0;
  for (size_t b = 0; b < p.ch.size(); ++b) {
    f_soff[b] = off;
    const int tiles = p.ch[b].nt * p.ch[b].ks;
    if (tiles) r.cp[nc++] = PCopy{p.ch[b].f_tile, off, tiles | (3 << 28)};
    off += tiles * 512;
  }
  r.f_bytes = off;
  int xo = 0;
  for (size_t k = 0; k < p.runs.size(); ++k) {
    run_off[k] = xo;
    r.cp[nc++] = PCopy{p.runs[k].x_tile, xo, p.runs[k].tiles | (p.runs[k].buf << 28)};
    xo += p.runs[k].tiles;
  }
  r.x_tiles = xo;
  r.ncopy = nc;
  auto mk = [&](size_t b, int t0, int ntl, int flags) {
    const Chunk& c = p.ch[b];
    PItem it{};
    it.y_tile = c.y_tile + t0;
    it.f_soff = f_soff[b] + t0 * 512;
    it.x_t = p.ch_run[b] >= 0 ? run_off[(size_t)p.ch_run[b]] + p.ch_xt[b] : 0;
    it.ks = (short)c.ks;
    it.f_stride = (short)c.nt;
    it.ntl = (unsigned char)ntl;
    it.y_buf = (unsigned char)c.y_buf;
    it.flags = (unsigned char)flags;
    return it;
  };
  std::vector<std::vector<PItem>> per((size_t)NCW);
  if (p.mode == 0) {
    const int ipt = mode0_ipt(p.ch, ntw);
    std::vector<std::pair<long long, PItem>> items;
    for (size_t b = 0; b < p.ch.size(); ++b)
      for (int t0 = 0; t0 < p.ch[b].nt; t0 += ipt) {
        const int ntl = std::min(ipt, p.ch[b].nt - t0);
        items.push_back({(long long)ntl * std::max(1, p.ch[b].ks), mk(b, t0, ntl, 3)});
      }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<long long, PItem>& a, const std::pair<long long, PItem>& b) {
                       return a.first > b.first;
                     });
    std::vector<long long> load((size_t)NCW, 0);
    for (const auto& w : items) {
      const size_t m = (size_t)(std::min_element(load.begin(), load.end()) - load.begin());
      per[m].push_back(w.second);
      load[m] += w.first;
    }
  } else {
    const int nt = p.ch[0].nt, ipt = mode1_ipt(nt);
    for (int g = 0; g * ipt < nt; ++g)
      for (size_t b = 0; b < p.ch.size(); ++b) {
        int flags = 0;
        if ((p.first_last & 1) && b == 0) flags |= 1;
        if ((p.first_last & 2) && b + 1 == p.ch.size()) flags |= 2;
        per[(size_t)g].push_back(mk(b, g * ipt, std::min(ipt, nt - g * ipt), flags));
      }
  }
  int e = 0;
  for (int w = 0; w < NCW; ++w) {
    r.wbeg[w] = (unsigned char)e;
    for (const PItem& it : per[(size_t)w]) {
      if (e >= MAX_ITEMS) throw Error{HB_ERR_UNSUPPORTED, "piece record overflow"};
      r.it[e++] = it;
    }
  }
  r.wbeg[NCW] = (unsigned char)e;
}

// Cut one task into chunks of at most kc k-steps (kc nt tiles fit a piece
// of f_cap tiles).  A task that is one chunk is an independent product.
static void task_chunks(const NatTask& L, int f_cap, std::vector<Chunk>& cs) {
  if (L.nt > MAX_NT) throw Error{HB_ERR_UNSUPPORTED, "a factor block has more than 256 rows"};
  const int kc = std::max(1, std::min(X_CAP_TILES, f_cap / L.nt));
  cs.clear();
  for (const NatTerm& tm : L.terms)
    for (int k0 = 0; k0 < tm.ks; k0 += kc) {
      Chunk c{};
      c.f_tile = tm.f_tile + (long long)k0 * L.nt;
      c.x_tile = tm.x_tile + k0;
      c.y_tile = L.y_tile;
      c.nt = L.nt;
      c.ks = std::min(kc, tm.ks - k0);
      c.x_buf = tm.x_buf;
      c.y_buf = L.y_buf;
      cs.push_back(c);
    }
  if (cs.empty()) {   // every input is empty: the output is zero
    Chunk c{};
    c.y_tile = L.y_tile;
    c.nt = L.nt;
    c.y_buf = L.y_buf;
    cs.push_back(c);
  }
}

void flow_plan_build(const std::vector<NatTask>& lt, void** plan_out) {
  FlowPlan* P = new FlowPlan();
  try {
    int maxd = -1;
    for (const NatTask& L : lt) maxd = std::max(maxd, L.depth);
    P->depth_pieces.assign((size_t)(maxd + 1), {});
    std::vector<long long> dtiles((size_t)(maxd + 1), 0);
    for (const NatTask& L : lt)
      for (const NatTerm& tm : L.terms) dtiles[(size_t)L.depth] += (long long)L.nt * tm.ks;
    int dev = 0, nsm = 1;
    HB_CUDA(cudaGetDevice(&dev));
    HB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    std::vector<Chunk> cs;
    for (int d = 0; d <= maxd; ++d) {
      // optionally, small depths get smaller pieces: about PIECES_PER_SM per SM
      const int f_cap =
          PIECES_PER_SM <= 0
              ? F_CAP_TILES
              : (int)std::max<long long>(MAX_NT, std::min<long long>(F_CAP_TILES, dtiles[(size_t)d] /
                                                                                     ((long long)PIECES_PER_SM * nsm) /
                                                                                     8 * 8));
      std::vector<Chunk> indep;
      std::vector<std::vector<Chunk>> accum;
      for (const NatTask& L : lt) {
        if (L.depth != d || L.nt == 0) continue;
        task_chunks(L, f_cap, cs);
        if (cs.size() == 1) indep.push_back(cs[0]);
        else accum.push_back(cs);
      }
      // chunks that read the same or neighbouring input tiles meet in one piece
      std::stable_sort(indep.begin(), indep.end(), [](const Chunk& a, const Chunk& b) {
        if (a.x_buf != b.x_buf) return a.x_buf < b.x_buf;
        return a.x_tile < b.x_tile;
      });
      PieceBuilder pb(P->depth_pieces[(size_t)d], f_cap);
      for (const Chunk& c : indep) pb.add_independent(c);
      pb.flush();
      for (const auto& ch : accum) pb.add_task(ch);
      P->max_f_tiles = std::max(P->max_f_tiles, pb.max_f);
      P->max_x_tiles = std::max(P->max_x_tiles, pb.max_x);
    }
  } catch (...) {
    delete P;
    throw;
  }
  *plan_out = P;
}

static void free_streams(std::vector<DepthStreams>& ss) {
  for (DepthStreams& d : ss) {
    dev_free(d.d_recs);
    dev_free(d.d_off);
  }
  ss.clear();
}

void flow_plan_free(void* plan) {
  FlowPlan* P = static_cast<FlowPlan*>(plan);
  if (!P) return;
  for (auto& ss : P->streams) free_streams(ss);
  delete P;
}

int flow_plan_depths(const void* plan) { return (int)static_cast<const FlowPlan*>(plan)->depth_pieces.size(); }

// Per-CTA record streams of every depth for a maximum grid of gmax CTAs and
// MT m-tiles; the pieces of one accumulating task stay together, in order,
// on one CTA.
static void build_streams(FlowPlan* P, int gmax, int MT) {
  std::vector<DepthStreams>& out = P->streams[MT];
  free_streams(out);
  for (const std::vector<HostPiece>& pcs : P->depth_pieces) {
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
        for (size_t q : units[u]) {
          recs.emplace_back();
          encode(pcs[q], MT, recs.back());
        }
    }
    off.push_back((long long)recs.size());
    if (ds.grid > 0) {
      ds.d_recs = upload(recs);
      ds.d_off = upload(off);
    }
    out.push_back(ds);
  }
  HB_CUDA(cudaDeviceSynchronize());
  P->gmax[MT] = gmax;
}

template <int MT>
static void launch_depths(FlowPlan* P, const uint4* F, uint4* x, uint4* y, uint4* xh, int* err, long long budget,
                          cudaStream_t st, const std::function<void(int, bool)>& timer) {
  auto k = bf_step_kernel<MT>;
  int dev = 0, nsm = 0, optin = 0;
  HB_CUDA(cudaGetDevice(&dev));
  HB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  HB_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa{};
  HB_CUDA(cudaFuncGetAttributes(&fa, k));
  const int stage = P->max_f_tiles * 512 + P->max_x_tiles * MT * 1024;
  const int avail = optin - (int)fa.sharedSizeBytes;
  const int stages = std::min(MAX_STAGES, avail / stage);
  if (stages < 2) throw Error{HB_ERR_UNSUPPORTED, "step kernel stages do not fit in shared memory"};
  const size_t smem = (size_t)stages * stage;
  HB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  HB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, (NCW + 1) * 32, smem));
  if (per_sm < 1) throw Error{HB_ERR_UNSUPPORTED, "step kernel does not fit on an SM"};
  if (P->gmax[MT] != nsm * per_sm) build_streams(P, nsm * per_sm, MT);
  const std::vector<DepthStreams>& ss = P->streams[MT];
  for (int d = 0; d < (int)ss.size(); ++d) {
    const DepthStreams& ds = ss[(size_t)d];
    if (ds.grid == 0) continue;
    StepArgs args{ds.d_recs, ds.d_off, F, x, y, xh, stages, stage, budget, err};
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

void flow_launch(void* plan, const uint4* F, uint4* x, uint4* y, uint4* xh, int MT, int* err,
                 long long budget_cycles, cudaStream_t st, const std::function<void(int, bool)>& timer) {
  FlowPlan* P = static_cast<FlowPlan*>(plan);
  if (P->depth_pieces.empty()) return;
  if (MT == 1) launch_depths<1>(P, F, x, y, xh, err, budget_cycles, st, timer);
  else if (MT == 2) launch_depths<2>(P, F, x, y, xh, err, budget_cycles, st, timer);
  else throw Error{HB_ERR_UNSUPPORTED, "the mixed apply takes 1 or 2 m-tiles of 16 right-hand sides per pass"};
}

}  // namespace hb
