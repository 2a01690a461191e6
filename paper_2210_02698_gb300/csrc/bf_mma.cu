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
//     the n-tiles of a block are cut into groups of ng and its tiles are
//     ordered [group][k-step][n-tile in group], so that any run of k-steps
//     of one group is contiguous; the adjoint has its own arena holding F^H,
//     so both directions run the same code;
//   * vector tile (8 rows x 16 right-hand sides) = 32 lanes x uint4 of hi
//     words, then 32 x uint4 of lo words, word j of lane (g, t) holding
//     (row 2t + (j >> 1), right-hand side g + 8 (j & 1)); a buffer is
//     [row tile][m-tile] of such tiles.
// Rows of every block part (a leaf, a skeleton) are padded to a multiple of
// 8 with zeros; padded rows of the vectors stay exactly zero.
//
// Work.  A chain is one n-tile group of one output: the sum over the task's
// terms of (group of op(F)) x (input rows), cut into items of at most
// ITEM_BYTES (a run of k-steps of one term).  The items of a chain
// accumulate in one warp's registers and the last one stores the group.
//
// Scheduling.  Every warp of the GPU runs its own stream of chains (the
// host deals chains largest first to the least-loaded stream) through its
// own ring of shared-memory stages: lane 0 fetches an item's factor run and
// input run with cp.async.bulk (1D TMA) on the stage's mbarrier, the warp
// computes from the stage, and lane 0 refills it with the item NST ahead.
// No warp waits for another.  Chains are grouped by dependency depth
// (depth d only reads outputs of depths < d), one launch per depth, chained
// by programmatic dependent launch: factor runs (constant data) of the
// first items go out before griddepcontrol.wait, input runs after it.
// Every wait is bounded by a per-thread deadline; past it the mapped error
// word is set, the warp waits (bounded) for its copies in flight and stops.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <queue>
#include <vector>

#include "hb_internal.cuh"

namespace hb {

// Stream geometry (compile-time; the defaults are the tuned values).
#ifndef HB_FLOW_WARPS
#define HB_FLOW_WARPS 8
#endif
#ifndef HB_FLOW_ITEM_BYTES
#define HB_FLOW_ITEM_BYTES 16384
#endif
#ifndef HB_FLOW_MAX_STAGES
#define HB_FLOW_MAX_STAGES 4
#endif
constexpr int NWARP = HB_FLOW_WARPS;               // warps (streams) per CTA
constexpr int ITEM_BYTES = HB_FLOW_ITEM_BYTES;     // stage bytes of one item at 2 m-tiles
constexpr int MAX_STAGES = HB_FLOW_MAX_STAGES;     // ring stages per warp
#ifndef HB_FLOW_NTW
#define HB_FLOW_NTW 8
#endif
constexpr int NTW = HB_FLOW_NTW;                   // largest n-tile group (accumulators: 8 NTW MT registers)
constexpr uint32_t IM_SIGN = 0x80000000u;          // sign bit of the imaginary (upper) bf16

// One item (32 bytes): ks k-steps of one n-tile group of one term.
struct WItem {
  long long f_tile;      // first factor tile (a contiguous run of ntl x ks tiles)
  long long x_tile;      // first input row tile (a contiguous run of ks tiles)
  long long y_tile;      // first output row tile of the group
  short ks;
  unsigned char ntl;     // n-tiles of the group
  unsigned char flags;   // 1: zero the accumulators first, 2: store them after
  unsigned char x_buf;   // 0 = x, 1 = y, 2 = xh
  unsigned char y_buf;
  short pad;
};
static_assert(sizeof(WItem) == 32, "item layout");

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

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for an mbarrier phase until the deadline (clock64 of this SM).
__device__ __forceinline__ bool mbar_wait_until(uint64_t* bar, uint32_t parity, long long deadline) {
  while (!mbar_try_wait(bar, parity))
    if (clock64() > deadline) return false;
  return true;
}

// 1D bulk copy global -> shared, completion counted on the mbarrier, with
// an L2 cache policy.  dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                            uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
      "%4;\n" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// L2 policies: factors stream through once per apply (evict first); the
// vectors are written by one depth and read by the next (evict last).
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}

__device__ __forceinline__ void st_global_hint(uint4* p, const uint4& v, uint64_t policy) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w), "l"(policy)
               : "memory");
}

struct StepArgs {
  const WItem* items;
  const long long* off;       // items of stream s (= CTA * NWARP + warp): [off[s], off[s + 1])
  const uint4* F;
  uint4* x;
  uint4* xh;
  double2* u;                 // outputs of buffer 1 go straight to u[rhs * Nv + natural index]
  const long long* pperm;     // padded tree row -> natural index (-1: padding)
  long long Nv;
  int R;
  int stages;                 // ring stages per warp
  int stage_bytes;
  long long budget;
  int* err;
  int selftest;               // the first warp also waits on a barrier nothing completes
};

// Accumulate ks k-steps of an item into acc: NTL n-tiles whose tiles are
// [k-step][n-tile] at Fs, input row tiles at Xs.  NTL is a compile-time
// count so that no MMA slot is issued for an absent tile.
template <int MT, int NTL>
__device__ __forceinline__ void item_mma_n(const uint4* __restrict__ Fs, const uint4* __restrict__ Xs, int ks,
                                           int lane, float (&acc)[NTW][MT][8]) {
  const uint4* fp = Fs + lane;
  const uint4* xp = Xs + lane;
  // two k-steps per trip: the second step's fragment loads overlap the
  // first step's MMAs
#pragma unroll 2
  for (int k = 0; k < ks; ++k, fp += NTL * 32, xp += MT * 64) {
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
      // each split product over every accumulator before the next: no
      // two consecutive MMAs of the warp depend on one another
#pragma unroll
      for (int j = 0; j < NTL; ++j) {
        mma16816(acc[j][mt], arh, b[j].x, b[j].y);
        mma16816(acc[j][mt] + 4, aih, b[j].x, b[j].y);
      }
#pragma unroll
      for (int j = 0; j < NTL; ++j) {
        mma16816(acc[j][mt], arh, b[j].z, b[j].w);
        mma16816(acc[j][mt] + 4, aih, b[j].z, b[j].w);
      }
#pragma unroll
      for (int j = 0; j < NTL; ++j) {
        mma16816(acc[j][mt], arl, b[j].x, b[j].y);
        mma16816(acc[j][mt] + 4, ail, b[j].x, b[j].y);
      }
    }
  }
}

template <int MT>
__device__ __forceinline__ void item_mma(const uint4* Fs, const uint4* Xs, int ks, int ntl, int lane,
                                         float (&acc)[NTW][MT][8]) {
  switch (ntl) {
    case 1: item_mma_n<MT, 1>(Fs, Xs, ks, lane, acc); break;
    case 2: item_mma_n<MT, 2>(Fs, Xs, ks, lane, acc); break;
    case 3: item_mma_n<MT, 3>(Fs, Xs, ks, lane, acc); break;
    case 4: item_mma_n<MT, 4>(Fs, Xs, ks, lane, acc); break;
    default:
      if constexpr (NTW > 4) {
        switch (ntl) {
          case 5: item_mma_n<MT, 5>(Fs, Xs, ks, lane, acc); break;
          case 6: item_mma_n<MT, 6>(Fs, Xs, ks, lane, acc); break;
          case 7: item_mma_n<MT, 7>(Fs, Xs, ks, lane, acc); break;
          case 8: item_mma_n<MT, 8>(Fs, Xs, ks, lane, acc); break;
          default: break;
        }
      }
      break;
  }
}

// Store ntl n-tiles of the accumulators as vector tiles at Y.  Accumulator
// element e of lane (g, t) is (right-hand side g + 8 (e >> 1), output
// 2t + (e & 1)); vector word j holds (row 2t + (j >> 1), right-hand side
// g + 8 (j & 1)), so words (0, 1, 2, 3) = elements (0, 2, 1, 3).
template <int MT>
__device__ __forceinline__ void store_tiles(uint4* Y, int ntl, int lane, const float (&acc)[NTW][MT][8],
                                            uint64_t policy) {
#pragma unroll
  for (int j = 0; j < NTW; ++j) {
    if (j >= ntl) break;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const float* a = acc[j][mt];
      const uint2 p0 = to_pair(a[0], a[4]), p1 = to_pair(a[1], a[5]);
      const uint2 p2 = to_pair(a[2], a[6]), p3 = to_pair(a[3], a[7]);
      uint4* o = Y + ((size_t)j * MT + mt) * 64;
      st_global_hint(o + lane, make_uint4(p0.x, p2.x, p1.x, p3.x), policy);
      st_global_hint(o + 32 + lane, make_uint4(p0.y, p2.y, p1.y, p3.y), policy);
    }
  }
}

// Store ntl n-tiles of the accumulators in natural order: element e of
// lane (g, t) in tile j is row 8 (y_tile + j) + 2t + (e & 1), right-hand
// side 16 mt + g + 8 (e >> 1); padded rows and right-hand sides >= R are
// dropped.
template <int MT>
__device__ __forceinline__ void store_natural(const StepArgs& a, long long y_tile, int ntl, int lane,
                                              const float (&acc)[NTW][MT][8]) {
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int j = 0; j < NTW; ++j) {
    if (j >= ntl) break;
    const long long row = 8 * (y_tile + j) + 2 * t;
    const long long nat0 = a.pperm[row], nat1 = a.pperm[row + 1];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const float* v = acc[j][mt];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const long long nat = (e & 1) ? nat1 : nat0;
        const int rhs = 16 * mt + g + 8 * (e >> 1);
        if (nat >= 0 && rhs < a.R) a.u[(size_t)rhs * a.Nv + nat] = make_double2((double)v[e], (double)v[e + 4]);
      }
    }
  }
}

template <int MT>
__device__ __forceinline__ void zero_acc(float (&acc)[NTW][MT][8]) {
#pragma unroll
  for (int j = 0; j < NTW; ++j)
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[j][mt][e] = 0.f;
}

// ------------------------------------------------------------- kernel ----
template <int MT>
__global__ void __launch_bounds__(NWARP * 32, 1) bf_step_kernel(StepArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t full[NWARP][MAX_STAGES];
  __shared__ __align__(16) WItem slot[NWARP][MAX_STAGES];
  __shared__ __align__(16) int4 recs[NWARP][32][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nst = a.stages;
  auto buf = [&](int id) { return id == 0 ? a.x : a.xh; };   // inputs come from x or xh
  const long long sid = (long long)blockIdx.x * NWARP + warp;
  const long long ib = a.off[sid], n = a.off[sid + 1] - ib;
  unsigned char* ring = smem + (size_t)warp * nst * a.stage_bytes;
  uint64_t* bar = full[warp];
  WItem* sl = slot[warp];

  __shared__ uint64_t never;   // failure-detection self-test: nothing arrives on it
  if (lane == 0) {
    for (int s = 0; s < nst; ++s) mbar_init(&bar[s], 1);
    if (warp == 0) mbar_init(&never, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const long long deadline = clock64() + a.budget;
  const uint64_t pol_f = policy_evict_first(), pol_v = policy_evict_last();
  if (a.selftest && blockIdx.x == 0 && warp == 0) {
    const bool ok = mbar_wait_until(&never, 0u, deadline);
    if (lane == 0 && !ok) *reinterpret_cast<volatile int*>(a.err) = 1;
    __syncwarp();
  }

  // Item records: the warp keeps two windows of 32 in registers (lane j
  // holds record 32 w + j of window w), loading window w + 1 when the first
  // item of window w is issued; at that point window w moves to shared
  // memory, where lane 0 reads the record of each item it issues.
  int4 w0lo = make_int4(0, 0, 0, 0), w0hi = w0lo, w1lo = w0lo, w1hi = w0lo;
  auto load_win = [&](long long w) {
    const long long q = 32 * w + lane;
    if (q < n) {
      const int4* r = reinterpret_cast<const int4*>(a.items + ib + q);
      if (w & 1) {
        w1lo = r[0];
        w1hi = r[1];
      } else {
        w0lo = r[0];
        w0hi = r[1];
      }
    }
  };
  load_win(0);
  load_win(1);
  auto f_bytes = [](const WItem& w) { return (uint32_t)w.ntl * (uint32_t)w.ks * 512u; };
  auto x_bytes = [](const WItem& w) { return (uint32_t)w.ks * (uint32_t)(MT * 1024); };
  // all lanes: stage s gets item q; lane 0 stores its record, arms the
  // barrier and fetches the factor run (and the input run when with_x)
  auto issue = [&](int s, long long q, bool with_x) {
    if ((q & 31) == 0) {
      // the window of item q goes to shared memory (its loads were issued 32
      // items ago), then the next window is fetched into the freed registers
      const bool odd = (q >> 5) & 1;
      recs[warp][lane][0] = odd ? w1lo : w0lo;
      recs[warp][lane][1] = odd ? w1hi : w0hi;
      __syncwarp();
      if (q >= 32) load_win((q >> 5) + 1);
    }
    if (lane == 0) {
      const int4 lo = recs[warp][q & 31][0], hi = recs[warp][q & 31][1];
      int4* d = reinterpret_cast<int4*>(&sl[s]);
      d[0] = lo;
      d[1] = hi;
      const WItem& w = sl[s];
      unsigned char* st = ring + (size_t)s * a.stage_bytes;
      mbar_expect_tx(&bar[s], f_bytes(w) + x_bytes(w));
      if (w.ks) {
        tma_load_1d(st, a.F + w.f_tile * 32, f_bytes(w), &bar[s], pol_f);
        if (with_x)
          tma_load_1d(st + f_bytes(w), buf(w.x_buf) + w.x_tile * (MT * 64), x_bytes(w), &bar[s], pol_v);
      }
    }
  };

  // prologue: factor runs first, input runs once the previous depth is visible
  const long long pro = n < nst ? n : nst;
  for (long long q = 0; q < pro; ++q) issue((int)q, q, false);
  if (lane == 0) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
    for (long long q = 0; q < pro; ++q) {
      const WItem& w = sl[q];
      if (w.ks)
        tma_load_1d(ring + (size_t)q * a.stage_bytes + f_bytes(w), buf(w.x_buf) + w.x_tile * (MT * 64), x_bytes(w),
                    &bar[q], pol_v);
    }
  }
  __syncwarp();

  float acc[NTW][MT][8];
  zero_acc<MT>(acc);
  long long i = 0;
  for (; i < n; ++i) {
    const int s = (int)(i % nst);
    const bool ok = mbar_wait_until(&bar[s], (uint32_t)((i / nst) & 1), deadline);
    if (!__all_sync(0xffffffffu, ok)) break;
    const WItem& w = sl[s];
    const int flags = w.flags, ntl = w.ntl, ks = w.ks;
    const uint4* st = reinterpret_cast<const uint4*>(ring + (size_t)s * a.stage_bytes);
    if (flags & 1) zero_acc<MT>(acc);
    if (ks > 0) item_mma<MT>(st, st + ntl * ks * 32, ks, ntl, lane, acc);
    if (flags & 2) {
      if (w.y_buf == 1) store_natural<MT>(a, w.y_tile, ntl, lane, acc);
      else store_tiles<MT>(a.xh + (size_t)w.y_tile * (MT * 64), ntl, lane, acc, pol_v);
    }
    // every lane's reads of stage s are done before lane 0 refills it
    __syncwarp();
    if (i + nst < n) issue(s, i + nst, true);
    __syncwarp();
  }
  if (i < n) {
    // a wait ran out: report it, let the copies in flight land, stop
    if (lane == 0) {
      *reinterpret_cast<volatile int*>(a.err) = 1;
      const long long last = (i + nst < n) ? i + nst : n;
      const long long drain = a.budget > (1LL << 31) ? a.budget : (1LL << 31);
      for (long long j = i; j < last; ++j)
        mbar_wait_until(&bar[j % nst], (uint32_t)((j / nst) & 1), clock64() + drain);
    }
    __syncwarp();
  }
  if (lane == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// --------------------------------------------------- conversions / I/O ----
__device__ __forceinline__ int part_index(int pos, int r1, int r2) {
  const int p1 = (r1 + 7) & ~7;
  if (pos < p1) return pos < r1 ? pos : -1;
  return (pos - p1 < r2) ? r1 + pos - p1 : -1;
}

// One CTA per native block.  Tile index -> (group, k-step, n-tile in group);
// lane (g, t) of the tile gets {hi F[n][2t], hi F[n][2t+1], lo F[n][2t],
// lo F[n][2t+1]} with n = 8 n-tile + g.
__global__ void nat_convert_kernel(const double2* __restrict__ F, const NatBlock* __restrict__ blocks,
                                   uint4* __restrict__ out) {
  const NatBlock B = blocks[blockIdx.x];
  const int nt = (B.r1 + 7) / 8 + (B.r2 + 7) / 8, ks = (B.k1 + 7) / 8 + (B.k2 + 7) / 8;
  const int ngr = (nt + B.ng - 1) / B.ng;
  for (int idx = threadIdx.x; idx < nt * ks * 32; idx += blockDim.x) {
    const int tile = idx >> 5, lane = idx & 31, g = lane >> 2, t = lane & 3;
    const int grp = min(tile / (B.ng * ks), ngr - 1);
    const int within = tile - grp * B.ng * ks;
    const int gsz = (grp < ngr - 1) ? B.ng : nt - B.ng * (ngr - 1);
    const int kstep = within / gsz, ntile = grp * B.ng + within % gsz;
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

// x (native) = pair(scale * s[rhs * Nv + natural index of the padded row]).
// One warp per (row tile, m-tile): lane l reads rows l & 7, right-hand sides
// 16 mt + 4 (l >> 3) + c (c < 4) - for each c, eight lanes read one 128-byte
// run of a column when a leaf row is contiguous in natural order - and the
// pairs are transposed through shared memory into fragment order.
__global__ void __launch_bounds__(256) gather_native_kernel(const double2* __restrict__ s,
                                                            const long long* __restrict__ pperm,
                                                            uint4* __restrict__ x, long long nv_tiles, long long Nv,
                                                            int R, int MT, double scale) {
  __shared__ __align__(16) uint32_t tile[8][256];
  // the first depth launch may start now and stream its factor runs; it
  // reads x only after griddepcontrol.wait, i.e. after this grid completes
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const long long wid = (long long)blockIdx.x * 8 + wb;
  if (wid >= nv_tiles * MT) return;
  const long long rt = wid / MT;
  const int mt = (int)(wid - rt * MT);
  const int r = lane & 7, c0 = 4 * (lane >> 3);
  const long long nat = pperm[8 * rt + r];
  double2 v[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int rhs = 16 * mt + c0 + c;
    v[c] = (nat >= 0 && rhs < R) ? s[(size_t)rhs * Nv + nat] : make_double2(0.0, 0.0);
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int q = c0 + c;                               // right-hand side within the m-tile
    const int dl = (q & 7) * 4 + (r >> 1);              // destination lane (g, t) = (q & 7, r >> 1)
    const int dj = (r & 1) * 2 + (q >> 3);              // destination word
    const uint2 p = to_pair((float)(v[c].x * scale), (float)(v[c].y * scale));
    tile[wb][dl * 4 + dj] = p.x;
    tile[wb][128 + dl * 4 + dj] = p.y;
  }
  __syncwarp();
  uint4* out = x + (size_t)wid * 64;   // tile (rt, mt) = rt * MT + mt = wid
  out[lane] = reinterpret_cast<const uint4*>(tile[wb])[lane];
  out[32 + lane] = reinterpret_cast<const uint4*>(tile[wb])[32 + lane];
}

void gather_native(const double2* s, const long long* pperm, uint4* x, long long nv_tiles, long long Nv, int R,
                   int MT, double scale, cudaStream_t st) {
  const long long warps = nv_tiles * MT;
  if (warps == 0) return;
  gather_native_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(s, pperm, x, nv_tiles, Nv, R, MT, scale);
  HB_CHECK_LAUNCH();
}

// ------------------------------------------------------------- planning ----
struct DepthStreams {
  int grid = 0;
  WItem* d_items = nullptr;
  long long* d_off = nullptr;
};

struct LaunchShape {   // per m-tile count, set on first use
  bool ready = false;
  int stage = 0, stages = 0, grid = 0;
  size_t smem = 0;
};

// Everything below is kept per m-tile count MT (index 1 or 2): the items are
// cut so that NWARP warps x 2 stages of the largest item fit in shared memory.
struct FlowPlan {
  // chains of every depth: the items of one chain, in order
  std::vector<std::vector<std::vector<WItem>>> chains[3];
  int stage_bytes[3] = {0, 512, 512};     // largest item (factor run + input run)
  int grid[3] = {0, 0, 0};                // CTAs the streams were dealt for
  LaunchShape shape[3];
  std::vector<DepthStreams> streams[3];
};

// k-steps per item for groups of ntl n-tiles: at one m-tile, ITEM_BYTES
// bounds the factor run plus the input run counted at two m-tiles (so an
// item is at most 12 KB); at two m-tiles the bound is 13 KB (an item is then
// at most 12.5 KB, and 8 warps x 2 stages fit in 227 KB beside the record
// windows).
static int item_ks(int ntl, int MT) {
  return std::max(1, (MT == 1 ? ITEM_BYTES : 13312) / (512 * ntl + 2048));
}

// The chains of one task for MT m-tiles: group g holds n-tiles
// [g ng, g ng + ntl); each term contributes its k-steps in runs of at most
// item_ks(ntl, MT).
static void task_chains(const NatTask& L, int MT, std::vector<std::vector<WItem>>& out, int& stage_bytes) {
  if (L.ng < 1 || L.ng > NTW) throw Error{HB_ERR_UNSUPPORTED, "n-tile group larger than the accumulators"};
  const int ngr = (L.nt + L.ng - 1) / L.ng;
  for (int g = 0; g < ngr; ++g) {
    const int ntl = std::min(L.ng, L.nt - g * L.ng);
    const int kc = item_ks(ntl, MT);
    std::vector<WItem> ch;
    for (const NatTerm& tm : L.terms)
      for (int k0 = 0; k0 < tm.ks; k0 += kc) {
        WItem w{};
        w.f_tile = tm.f_tile + (long long)g * L.ng * tm.ks + (long long)k0 * ntl;
        w.x_tile = tm.x_tile + k0;
        w.y_tile = L.y_tile + (long long)g * L.ng;
        w.ks = (short)std::min(kc, tm.ks - k0);
        w.ntl = (unsigned char)ntl;
        w.x_buf = (unsigned char)tm.x_buf;
        w.y_buf = (unsigned char)L.y_buf;
        ch.push_back(w);
        stage_bytes = std::max(stage_bytes, ntl * (int)w.ks * 512 + (int)w.ks * MT * 1024);
      }
    if (ch.empty()) {   // every input is empty: the group is zero
      WItem w{};
      w.y_tile = L.y_tile + (long long)g * L.ng;
      w.ntl = (unsigned char)ntl;
      w.y_buf = (unsigned char)L.y_buf;
      ch.push_back(w);
    }
    ch.front().flags |= 1;
    ch.back().flags |= 2;
    out.push_back(std::move(ch));
  }
}

void flow_plan_build(const std::vector<NatTask>& lt, void** plan_out) {
  FlowPlan* P = new FlowPlan();
  try {
    int maxd = -1;
    for (const NatTask& L : lt) maxd = std::max(maxd, L.depth);
    for (int mt = 1; mt <= 2; ++mt) {
      P->chains[mt].assign((size_t)(maxd + 1), {});
      for (const NatTask& L : lt)
        if (L.nt > 0) task_chains(L, mt, P->chains[mt][(size_t)L.depth], P->stage_bytes[mt]);
    }
  } catch (...) {
    delete P;
    throw;
  }
  *plan_out = P;
}

static void free_streams(std::vector<DepthStreams>& ss) {
  for (DepthStreams& d : ss) {
    dev_free(d.d_items);
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

int flow_plan_depths(const void* plan) { return (int)static_cast<const FlowPlan*>(plan)->chains[1].size(); }

// Deal every depth's chains over grid x NWARP warp streams: longest chain
// (in factor tiles, plus a fixed cost per item) first, to the stream with
// the least work so far.
static void build_streams(FlowPlan* P, int grid, int MT) {
  std::vector<DepthStreams>& out = P->streams[MT];
  free_streams(out);
  const int ns = grid * NWARP;
  for (const auto& chains : P->chains[MT]) {
    DepthStreams ds;
    if (chains.empty()) {
      out.push_back(ds);
      continue;
    }
    std::vector<long long> cost(chains.size());
    for (size_t c = 0; c < chains.size(); ++c) {
      long long w = 0;
      for (const WItem& it : chains[c]) w += (long long)it.ntl * std::max<int>(1, it.ks) + 4;
      cost[c] = w;
    }
    std::vector<size_t> order(chains.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    using Load = std::pair<long long, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
    for (int s = 0; s < ns; ++s) pq.push({0, s});
    std::vector<std::vector<size_t>> per((size_t)ns);
    for (size_t c : order) {
      Load l = pq.top();
      pq.pop();
      per[(size_t)l.second].push_back(c);
      l.first += cost[c];
      pq.push(l);
    }
    std::vector<WItem> items;
    std::vector<long long> off;
    for (int s = 0; s < ns; ++s) {
      off.push_back((long long)items.size());
      for (size_t c : per[(size_t)s]) items.insert(items.end(), chains[c].begin(), chains[c].end());
    }
    off.push_back((long long)items.size());
    ds.grid = grid;
    ds.d_items = upload(items);
    ds.d_off = upload(off);
    out.push_back(ds);
  }
  HB_CUDA(cudaDeviceSynchronize());
  P->grid[MT] = grid;
}

template <int MT>
static void launch_depths(FlowPlan* P, const uint4* F, uint4* x, uint4* xh, double2* u, const long long* pperm,
                          long long Nv, int R, int* err, long long budget, bool selftest, cudaStream_t st,
                          const std::function<void(int, bool)>& timer) {
  auto k = bf_step_kernel<MT>;
  LaunchShape& L = P->shape[MT];
  if (!L.ready) {
    // once per plan and m-tile count: stages, shared memory, grid (then the streams)
    int dev = 0, nsm = 0, optin = 0;
    HB_CUDA(cudaGetDevice(&dev));
    HB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    HB_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa{};
    HB_CUDA(cudaFuncGetAttributes(&fa, k));
    L.stage = P->stage_bytes[MT];
    const int avail = optin - (int)fa.sharedSizeBytes;
    L.stages = std::min(MAX_STAGES, avail / (NWARP * L.stage));
    if (L.stages < 2) throw Error{HB_ERR_UNSUPPORTED, "step kernel stages do not fit in shared memory"};
    L.smem = (size_t)NWARP * L.stages * L.stage;
    // the kernel may take any size up to the opt-in limit (both directions' plans share it)
    HB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, avail));
    int per_sm = 0;
    HB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NWARP * 32, L.smem));
    if (per_sm < 1) throw Error{HB_ERR_UNSUPPORTED, "step kernel does not fit on an SM"};
    L.grid = nsm * per_sm;
    L.ready = true;
  }
  if (P->grid[MT] != L.grid) build_streams(P, L.grid, MT);
  bool first = true;   // the timer brackets all depth launches (PDL stays intact)
  for (int d = 0; d < (int)P->streams[MT].size(); ++d) {
    const DepthStreams& ds = P->streams[MT][(size_t)d];
    if (ds.grid == 0) continue;
    StepArgs args{ds.d_items, ds.d_off, F, x, xh, u, pperm, Nv, R, L.stages, L.stage, budget, err,
                  selftest ? 1 : 0};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ds.grid);
    cfg.blockDim = dim3(NWARP * 32);
    cfg.dynamicSmemBytes = L.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (first) timer(0, true);
    first = false;
    HB_CUDA(cudaLaunchKernelEx(&cfg, k, args));
  }
  if (!first) timer(0, false);
}

void flow_launch(void* plan, const uint4* F, uint4* x, uint4* xh, double2* u, const long long* pperm, long long Nv,
                 int R, int* err, long long budget_cycles, bool selftest, cudaStream_t st,
                 const std::function<void(int, bool)>& timer) {
  FlowPlan* P = static_cast<FlowPlan*>(plan);
  if (P->chains[1].empty()) return;
  const int MT = (R + 15) / 16;
  if (MT == 1) launch_depths<1>(P, F, x, xh, u, pperm, Nv, R, err, budget_cycles, selftest, st, timer);
  else if (MT == 2) launch_depths<2>(P, F, x, xh, u, pperm, Nv, R, err, budget_cycles, selftest, st, timer);
  else throw Error{HB_ERR_UNSUPPORTED, "the mixed apply takes 1 or 2 m-tiles of 16 right-hand sides per pass"};
}

}  // namespace hb
