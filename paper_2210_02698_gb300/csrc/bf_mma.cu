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
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <map>
#include <tuple>
#include <numeric>
#include <queue>
#include <vector>

#include "async_copy.cuh"
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
constexpr int PAIR_SLOTS = 1024;                   // fused level pairs: components per CTA and launch

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
// the kernels read records as two int4 (lo = bytes 0-15, hi = 16-31) and
// take x_tile = lo.z | lo.w << 32, ks = hi.z & 0xffff, flags = hi.z >> 24,
// x_buf = hi.w & 0xff, pad = hi.w >> 16 from them
static_assert(offsetof(WItem, x_tile) == 8 && offsetof(WItem, ks) == 24 && offsetof(WItem, flags) == 27 &&
                  offsetof(WItem, x_buf) == 28 && offsetof(WItem, pad) == 30,
              "item record fields");

// ------------------------------------------------------------ helpers ----
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
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
  const unsigned* need = nullptr;   // fused pairs: producer chains of each component slot, PAIR_SLOTS per CTA
  unsigned* gsync = nullptr;        // grid barriers: [0] arrivals, [1] CTAs finished (both 0 between launches)
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

// Store ntl n-tiles of the accumulators as row tiles in the operand layout
// of the tensor-core leaf kernel (leaf_tc.cu): in the 1 KB of row tile
// (y_tile + j, m-tile mt), the bf16 of (n = 16 c + rho, k) sits at
// (n / 8) 64 + (n % 8) 8 + k, c = 2 q + s for part q (Re, Im) of split half s
// (hi, lo) of right-hand side rho, k the row within the tile.  Lane (g, t)
// holds rows 2t, 2t + 1 of right-hand sides g and g + 8 (h = 0, 1), so each
// (c, h) is one 4-byte word per lane at word (2 c + h) 32 + lane.
template <int MT>
__device__ __forceinline__ void store_tiles_tc(uint4* Y, int ntl, int lane, const float (&acc)[NTW][MT][8]) {
#pragma unroll
  for (int j = 0; j < NTW; ++j) {
    if (j >= ntl) break;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) {
      const float* a = acc[j][mt];
      uint32_t* o = reinterpret_cast<uint32_t*>(Y + ((size_t)j * MT + mt) * 64);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint2 p0 = to_pair(a[2 * h], a[2 * h + 4]), p1 = to_pair(a[2 * h + 1], a[2 * h + 5]);
        o[(0 + h) * 32 + lane] = (p0.x & 0xffffu) | (p1.x << 16);
        o[(2 + h) * 32 + lane] = (p0.y & 0xffffu) | (p1.y << 16);
        o[(4 + h) * 32 + lane] = (p0.x >> 16) | (p1.x & 0xffff0000u);
        o[(6 + h) * 32 + lane] = (p0.y >> 16) | (p1.y & 0xffff0000u);
      }
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

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// ------------------------------------------------------------- kernel ----
// CONES: the launch runs cones of butterfly levels (a CTA takes whole cones;
// within a cone the level of every warp's items is separated by a barrier
// record, flags & 8).  At a barrier record every lane fences its stores for
// the async proxy, the warp arrives on the CTA's barrier and waits for the
// other warps (bounded); the input runs of items issued behind a barrier not
// yet passed go out once it is.
template <int MT, int VAR>
__global__ void __launch_bounds__(NWARP * 32, 1) bf_step_kernel(StepArgs a) {
  constexpr bool CONES = VAR == 1;   // barrier records between cone levels
  constexpr bool PAIRS = VAR == 2;   // fused level pairs: producer / consumer components within the CTA
  constexpr bool GRID = VAR == 3;    // every depth in one cooperative launch, grid barriers between depths
  constexpr bool BARS = CONES || GRID;   // barrier records in the streams
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
  __shared__ uint64_t cbar[2];   // level barriers of the CTA's warps (CONES, GRID), used alternately
  __shared__ uint64_t gbar[2];   // GRID: the grid barrier passed (warp 0 arrives), used alternately
  // PAIRS: producer chains still to finish, per component slot of this CTA
  __shared__ unsigned slot_left[PAIRS ? PAIR_SLOTS : 1];
  if constexpr (PAIRS)
    for (int t = threadIdx.x; t < PAIR_SLOTS; t += blockDim.x) slot_left[t] = a.need[(size_t)blockIdx.x * PAIR_SLOTS + t];
  if (lane == 0) {
    for (int s = 0; s < nst; ++s) mbar_init(&bar[s], 1);
    if (warp == 0) mbar_init(&never, 1);
    if (BARS && warp == 0) {
      mbar_init(&cbar[0], NWARP);
      mbar_init(&cbar[1], NWARP);
      mbar_init(&gbar[0], 1);
      mbar_init(&gbar[1], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if constexpr (BARS || PAIRS) __syncthreads();
  else __syncwarp();
  // barrier records issued / passed, and for each stage the barriers that
  // must be passed before its input run goes out (pending stages only)
  int bar_issued = 0, bar_passed = 0;
  unsigned pend = 0;
  int ep[MAX_STAGES];
#pragma unroll
  for (int s = 0; s < MAX_STAGES; ++s) ep[s] = 0;
  // PAIRS: cp.async groups committed so far, and the group of each stage
  long long gseq = 0;
  long long gs[MAX_STAGES];
#pragma unroll
  for (int s = 0; s < MAX_STAGES; ++s) gs[s] = -1;
  // the budget of the waits; counted again once the previous launch is
  // visible (a launch may start early and wait there for its predecessor)
  long long deadline = clock64() + a.budget;
  const uint64_t pol_f = policy_evict_first(), pol_v = policy_evict_last();
  // failure-detection self-test: the first warp also waits, through the
  // same bounded wait, on a barrier nothing completes (with cones and pairs
  // after its stream, since the other warps of its CTA may wait for it)
  if (!BARS && !PAIRS && a.selftest && blockIdx.x == 0 && warp == 0) {
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
  // PAIRS: a consumer item (flags & 16) reads the outputs of its component's
  // producer chains, which may run on other warps of the CTA; pad = the
  // component's slot.  Ready once no producer chain of the slot is left.
  auto slot_ready = [&](int pad) {
    const unsigned v = *reinterpret_cast<volatile unsigned*>(&slot_left[pad & (PAIR_SLOTS - 1)]);
    return __shfl_sync(0xffffffffu, (int)(v == 0u), 0) != 0;
  };
  // PAIRS, all lanes: the input run of the item in stage s (written by this
  // CTA's producers, in xh) copied into the stage with cp.async, one group
  auto own_copy = [&](int s, const WItem& w) {
    __threadfence_block();   // acquire side of the slot count just observed
    uint4* dst = reinterpret_cast<uint4*>(ring + (size_t)s * a.stage_bytes + f_bytes(w));
    const uint4* src = a.xh + w.x_tile * (MT * 64);
    const int chunks = w.ks * MT * 64;
    for (int c = lane; c < chunks; c += 32) cp_async16(dst + c, src + c);
    cp_async_commit();
    gs[s] = gseq++;
  };
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
    bool x_now = with_x;
    if constexpr (BARS) {
      // every lane tracks the barrier records (warp-uniform)
      const int4 hi = recs[warp][q & 31][1];
      if ((hi.z >> 24) & 8) {
        ++bar_issued;
      } else if (bar_issued > bar_passed) {
        x_now = false;
        const int ks = hi.z & 0xffff;
        if (ks) {
          pend |= 1u << s;
          ep[s] = bar_issued;
        }
      }
    }
    bool own = false;   // PAIRS: the input run is this warp's own output (copied by cp.async)
    if constexpr (PAIRS) {
      const int4 hi = recs[warp][q & 31][1];
      own = ((hi.z >> 24) & 16) != 0 && (hi.z & 0xffff) != 0;
      if (own) {
        x_now = false;
        const int pad = (int)((unsigned)hi.w >> 16);
        if (with_x && slot_ready(pad)) {
          const WItem& wq = *reinterpret_cast<const WItem*>(recs[warp][q & 31]);
          own_copy(s, wq);
        } else {
          pend |= 1u << s;
        }
      }
    }
    if (lane == 0) {
      const int4 lo = recs[warp][q & 31][0], hi = recs[warp][q & 31][1];
      int4* d = reinterpret_cast<int4*>(&sl[s]);
      d[0] = lo;
      d[1] = hi;
      const WItem& w = sl[s];
      unsigned char* st = ring + (size_t)s * a.stage_bytes;
      mbar_expect_tx(&bar[s], f_bytes(w) + (own ? 0u : x_bytes(w)));
      if (w.ks) {
        tma_load_1d(st, a.F + w.f_tile * 32, f_bytes(w), &bar[s], pol_f);
        if (x_now)
          tma_load_1d(st + f_bytes(w), buf(w.x_buf) + w.x_tile * (MT * 64), x_bytes(w), &bar[s], pol_v);
      }
    }
  };
  auto issue_x = [&](int s) {   // lane 0: the deferred input run of stage s
    const WItem& w = sl[s];
    tma_load_1d(ring + (size_t)s * a.stage_bytes + f_bytes(w), buf(w.x_buf) + w.x_tile * (MT * 64), x_bytes(w),
                &bar[s], pol_v);
  };

  // prologue: factor runs first, input runs once the previous depth is visible
  const long long pro = n < nst ? n : nst;
  for (long long q = 0; q < pro; ++q) issue((int)q, q, false);
  if (lane == 0) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
    for (long long q = 0; q < pro; ++q) {
      const WItem& w = sl[q];
      if (w.ks && !((pend >> q) & 1u)) issue_x((int)q);
    }
  }
  __syncwarp();
  deadline = clock64() + a.budget;

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
    if constexpr (BARS) {
      if (flags & 8) {
        // the warp's stores of this level reach the async proxy, then every
        // warp of the CTA has finished the level
        asm volatile("fence.proxy.async.global;" ::: "memory");
        __syncwarp();
        uint64_t* cb = &cbar[bar_passed & 1];
        const uint32_t par = (uint32_t)((bar_passed >> 1) & 1);
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(cb)) : "memory");
        bool okb = true;
        if (!GRID || warp == 0) okb = mbar_wait_until(cb, par, deadline);
        if constexpr (GRID) {
          // warp 0 publishes the CTA's level at gpu scope (the CTA barrier
          // made the other warps' stores visible to it), counts the CTA in
          // and waits (bounded) for every CTA; then it releases the CTA's
          // warps, which fetch the next level's inputs
          uint64_t* gb = &gbar[bar_passed & 1];
          if (warp == 0) {
            int okg = __all_sync(0xffffffffu, okb) ? 1 : 0;
            if (lane == 0) {
              __threadfence();
              atomicAdd(a.gsync, 1u);
              const unsigned target = (unsigned)(bar_passed + 1) * gridDim.x;
              while (okg && ld_acquire_gpu(a.gsync) < target)
                if (clock64() > deadline) okg = 0;
              asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(gb)) : "memory");
            }
            okb = __shfl_sync(0xffffffffu, okg, 0) != 0;
          }
          okb = mbar_wait_until(gb, par, deadline) && okb;
          if (lane == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
        }
        ++bar_passed;
        // deferred input runs now allowed (issued even after a timeout: in bounds)
        unsigned go = 0;
#pragma unroll
        for (int t = 0; t < MAX_STAGES; ++t)
          if (t < nst && ((pend >> t) & 1u) && ep[t] <= bar_passed) go |= 1u << t;
        if (lane == 0)
          for (int t = 0; t < nst; ++t)
            if ((go >> t) & 1u) issue_x(t);
        pend &= ~go;
        if (!__all_sync(0xffffffffu, okb)) break;
        __syncwarp();
        if (i + nst < n) issue(s, i + nst, true);
        __syncwarp();
        continue;
      }
    }
    if constexpr (PAIRS) {
      if ((flags & 16) && ks > 0) {
        if ((pend >> s) & 1u) {   // wait (bounded) for its producers, copy, then wait for the copy
          bool okp = true;
          while (!slot_ready(w.pad))
            if (clock64() > deadline) {
              okp = false;
              break;
            }
          own_copy(s, w);   // also after a timeout: in bounds
          pend &= ~(1u << s);
          if (!okp) break;
        }
        cp_async_wait_pending((int)(gseq - 1 - gs[s]));
        __syncwarp();
      }
    }
    if (flags & 1) zero_acc<MT>(acc);
    if (ks > 0) item_mma<MT>(st, st + ntl * ks * 32, ks, ntl, lane, acc);
    if (flags & 2) {
      if (w.y_buf == 1) store_natural<MT>(a, w.y_tile, ntl, lane, acc);
      else if (flags & 4) store_tiles_tc<MT>(a.xh + (size_t)w.y_tile * (MT * 64), ntl, lane, acc);
      else store_tiles<MT>(a.xh + (size_t)w.y_tile * (MT * 64), ntl, lane, acc, pol_v);
      if constexpr (PAIRS) {
        if (flags & 32) {   // a producer chain of the CTA's component `pad` is stored
          __threadfence_block();
          __syncwarp();
          if (lane == 0) atomicSub(&slot_left[w.pad & (PAIR_SLOTS - 1)], 1u);
        }
      }
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
      for (int t = 0; t < nst; ++t)
        if (!PAIRS && ((pend >> t) & 1u)) issue_x(t);   // in bounds: every stage completes
      const long long last = (i + nst < n) ? i + nst : n;
      const long long drain = a.budget > (1LL << 31) ? a.budget : (1LL << 31);
      for (long long j = i; j < last; ++j)
        mbar_wait_until(&bar[j % nst], (uint32_t)((j / nst) & 1), clock64() + drain);
    }
    __syncwarp();
  }
  if constexpr (PAIRS) asm volatile("cp.async.wait_all;" ::: "memory");   // no copy outlives the CTA
  if ((BARS || PAIRS) && a.selftest && blockIdx.x == 0 && warp == 0) {
    const bool ok = mbar_wait_until(&never, 0u, clock64() + a.budget);
    if (lane == 0 && !ok) *reinterpret_cast<volatile int*>(a.err) = 1;
    __syncwarp();
  }
  if constexpr (GRID) {
    // the last CTA to finish resets the barrier counters for the next
    // launch (every CTA has passed, or given up on, all its barriers)
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(a.gsync + 1, 1u) == gridDim.x - 1) {
        atomicExch(a.gsync, 0u);
        atomicExch(a.gsync + 1, 0u);
        __threadfence();
      }
    }
  }
  if (lane == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ------------------------------------------------ persistent dataflow ----
// One launch per apply: every warp runs its stream of chains of ALL depths,
// and a chain waits only for the row tiles it reads, not for a whole depth.
// Readiness is a per-row-tile flag (x tiles then xh tiles) holding the
// number of the launch that last wrote the tile; a launch writes
// target = (launches completed) + 1, so no flag is ever reset.
//
// Producers: the lanes of a warp store a chain's output tiles, fence, and
// set the tiles' flags (after pub_batch chains, or earlier when the warp is
// about to wait).  Consumers: the flags of an item's input tiles are read
// once when its record window is loaded (32 items ahead); an item found
// ready there, or at its refill, gets both copies at once; otherwise its
// factor run goes out and its input run is issued when the item is next to
// compute, after a bounded wait on the flags.
//
// Deadlock freedom.  The host places the chains by simulating the schedule
// (chains in order of their simulated ready time, each on the stream that
// frees first), so every stream runs its chains in increasing simulated
// start time and every producer starts before its consumers.  A warp waits
// on flags only for the item it must compute next, with all its earlier
// chains stored and published; the gather slices are published before any
// warp waits.  A waiting warp's producer therefore starts strictly earlier
// in the simulated order than the waiting chain, and the warp holding that
// producer is either running or waiting on a strictly earlier chain: no
// cycle.  The launch is cooperative, so all CTAs are resident together.
struct FlowArgs {
  StepArgs a;
  const double2* s;     // FP64 input in natural order (gathered here)
  double scale;
  long long nv_tiles;   // flags [0, nv_tiles): x row tiles; nv_tiles + t: xh row tile t
  unsigned* flags;
  unsigned* epoch;      // [0] launches completed, [1] CTAs finished in this launch
  int pub_batch;        // chains whose flags are set together
};

constexpr int PUB_MAX = 64;   // pending output tiles per warp

__device__ __forceinline__ unsigned ld_flag(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_flag(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// x (native) tile (rt, mt) = pairs of scale * s at the padded rows of row
// tile rt, one warp (as gather_native_kernel, through the warp's scratch)
template <int MT>
__device__ __forceinline__ void gather_tile(const FlowArgs& f, long long rt, int lane, uint32_t* tile) {
  const int r = lane & 7, c0 = 4 * (lane >> 3);
  const long long nat = f.a.pperm[8 * rt + r];
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) {
    double2 v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int rhs = 16 * mt + c0 + c;
      v[c] = (nat >= 0 && rhs < f.a.R) ? f.s[(size_t)rhs * f.a.Nv + nat] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int q = c0 + c;
      const int dl = (q & 7) * 4 + (r >> 1);
      const int dj = (r & 1) * 2 + (q >> 3);
      const uint2 p = to_pair((float)(v[c].x * f.scale), (float)(v[c].y * f.scale));
      tile[dl * 4 + dj] = p.x;
      tile[128 + dl * 4 + dj] = p.y;
    }
    __syncwarp();
    uint4* out = f.a.x + ((size_t)rt * MT + mt) * 64;
    out[lane] = reinterpret_cast<const uint4*>(tile)[lane];
    out[32 + lane] = reinterpret_cast<const uint4*>(tile)[32 + lane];
    __syncwarp();
  }
}

template <int MT>
__global__ void __launch_bounds__(NWARP * 32, 1) bf_flow_kernel(FlowArgs f) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ uint64_t full[NWARP][MAX_STAGES];
  __shared__ __align__(16) WItem slot[NWARP][MAX_STAGES];
  __shared__ __align__(16) int4 recs[NWARP][32][2];
  __shared__ __align__(16) uint32_t gtile[NWARP][256];
  __shared__ int pubs[NWARP][PUB_MAX];
  __shared__ unsigned s_target;
  __shared__ uint64_t never;   // failure-detection self-test: nothing arrives on it
  const StepArgs& a = f.a;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nst = a.stages;
  auto buf = [&](int id) { return id == 0 ? a.x : a.xh; };
  const long long sid = (long long)blockIdx.x * NWARP + warp;
  const long long nstreams = (long long)gridDim.x * NWARP;
  const long long ib = a.off[sid], n = a.off[sid + 1] - ib;
  unsigned char* ring = smem + (size_t)warp * nst * a.stage_bytes;
  uint64_t* bar = full[warp];
  WItem* sl = slot[warp];
  if (threadIdx.x == 0) s_target = *reinterpret_cast<volatile unsigned*>(f.epoch) + 1u;
  if (lane == 0) {
    for (int s = 0; s < nst; ++s) mbar_init(&bar[s], 1);
    if (warp == 0) mbar_init(&never, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const unsigned target = s_target;
  const long long deadline = clock64() + a.budget;
  const uint64_t pol_f = policy_evict_first(), pol_v = policy_evict_last();

  // flags of an item's input tiles: all lanes, warp-uniform result
  auto inputs_ready = [&](const WItem& w) {
    bool ok = true;
    const unsigned* fl = f.flags + (w.x_buf == 0 ? 0 : f.nv_tiles) + w.x_tile;
    for (int j = lane; j < w.ks; j += 32) ok = ok && ld_flag(fl + j) == target;
    return __all_sync(0xffffffffu, ok);
  };

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
  // move the window of item q to shared memory; each lane checks the flags
  // of its record's inputs there and marks the record ready (pad = 1)
  auto move_window = [&](long long q) {
    const bool odd = (q >> 5) & 1;
    int4 lo = odd ? w1lo : w0lo, hi = odd ? w1hi : w0hi;
    const int ks = hi.z & 0xffff, xb = hi.w & 0xff;
    const long long xt = (long long)(((unsigned long long)(unsigned)lo.w << 32) | (unsigned)lo.z);
    const unsigned* fl = f.flags + (xb == 0 ? 0 : f.nv_tiles) + xt;
    bool ok = true;
    for (int j0 = 0; j0 < ks; j0 += 8) {   // loads issued together, compared after
      unsigned v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = (j0 + j < ks) ? ld_flag(fl + j0 + j) : target;
#pragma unroll
      for (int j = 0; j < 8; ++j) ok = ok && v[j] == target;
    }
    hi.w = (hi.w & 0xffff) | (ok ? 0x10000 : 0);
    recs[warp][lane][0] = lo;
    recs[warp][lane][1] = hi;
    __syncwarp();
    if (q >= 32) load_win((q >> 5) + 1);
  };
  // stage s gets item q: lane 0 stores the record, arms the barrier for both
  // runs and fetches the factor run, and the input run when the record was
  // found ready (may_x); returns false (warp-uniform) when the input run is
  // left pending
  auto issue = [&](int s, long long q, bool may_x) {
    if ((q & 31) == 0) move_window(q);
    const int4 lo = recs[warp][q & 31][0], hi = recs[warp][q & 31][1];
    WItem w;
    reinterpret_cast<int4*>(&w)[0] = lo;
    reinterpret_cast<int4*>(&w)[1] = hi;
    const bool xok = w.ks == 0 || (may_x && w.pad != 0);
    if (lane == 0) {
      sl[s] = w;
      unsigned char* st = ring + (size_t)s * a.stage_bytes;
      mbar_expect_tx(&bar[s], f_bytes(w) + x_bytes(w));
      if (w.ks) {
        tma_load_1d(st, a.F + w.f_tile * 32, f_bytes(w), &bar[s], pol_f);
        if (xok) {
          asm volatile("fence.proxy.async.global;" ::: "memory");
          tma_load_1d(st + f_bytes(w), buf(w.x_buf) + w.x_tile * (MT * 64), x_bytes(w), &bar[s], pol_v);
        }
      }
    }
    return xok;
  };
  auto issue_x = [&](int s) {   // lane 0: the pending input run of stage s
    const WItem& w = sl[s];
    asm volatile("fence.proxy.async.global;" ::: "memory");
    tma_load_1d(ring + (size_t)s * a.stage_bytes + f_bytes(w), buf(w.x_buf) + w.x_tile * (MT * 64), x_bytes(w),
                &bar[s], pol_v);
  };

  // output tiles stored but not yet flagged
  int npub = 0, nchains = 0;
  auto publish = [&]() {
    if (npub == 0) return;
    __threadfence();
    __syncwarp();
    for (int j = lane; j < npub; j += 32) st_flag(f.flags + f.nv_tiles + pubs[warp][j], target);
    __syncwarp();
    npub = 0;
    nchains = 0;
  };

  // prologue: factor runs of the first items, then this warp's slice of the
  // gather (published at once), then the first input runs
  const long long pro = n < nst ? n : nst;
  unsigned pend = 0;
  for (long long q = 0; q < pro; ++q) issue((int)q, q, false);
  {
    const long long g0 = f.nv_tiles * sid / nstreams, g1 = f.nv_tiles * (sid + 1) / nstreams;
    for (long long rt = g0; rt < g1; ++rt) gather_tile<MT>(f, rt, lane, gtile[warp]);
    __threadfence();
    __syncwarp();
    for (long long rt = g0 + lane; rt < g1; rt += 32) st_flag(f.flags + rt, target);
    __syncwarp();
  }
  for (long long q = 0; q < pro; ++q)
    if (sl[q].ks) pend |= 1u << q;   // polled below like any pending stage
  __syncwarp();

  float acc[NTW][MT][8];
  zero_acc<MT>(acc);
  long long i = 0;
  bool timed_out = false;
  // Pending stages are polled without stalling: lane j reads the flag of
  // input tile j % 8 of stage j / 8 before the item's products and the
  // values are looked at after them (stages with more than 8 input tiles
  // wait until they are next).
  const int pst = lane >> 3, ptl = lane & 7;
  for (; i < n; ++i) {
    const int s = (int)(i % nst);
    unsigned pv = target;
    if (((pend >> pst) & 1u) && pst != s && pst < nst) {
      const WItem& w = sl[pst];
      if (w.ks <= 8 && ptl < w.ks) pv = ld_flag(f.flags + (w.x_buf == 0 ? 0 : f.nv_tiles) + w.x_tile + ptl);
    }
    if ((pend >> s) & 1u) {
      // next to compute: publish, then wait (bounded) for the input tiles
      publish();
      bool ok = false;
      while (!(ok = inputs_ready(sl[s])))
        if (clock64() > deadline) break;
      if (lane == 0) issue_x(s);   // also after a timeout: in bounds, so the stage completes
      pend &= ~(1u << s);
      if (!ok) {
        timed_out = true;
        break;
      }
    }
    const bool ok = mbar_wait_until(&bar[s], (uint32_t)((i / nst) & 1), deadline);
    if (!__all_sync(0xffffffffu, ok)) {
      timed_out = true;
      break;
    }
    const WItem& w = sl[s];
    const int flags = w.flags, ntl = w.ntl, ks = w.ks;
    const uint4* st = reinterpret_cast<const uint4*>(ring + (size_t)s * a.stage_bytes);
    if (flags & 1) zero_acc<MT>(acc);
    if (ks > 0) item_mma<MT>(st, st + ntl * ks * 32, ks, ntl, lane, acc);
    // pending stages whose tiles all showed ready get their input runs
    const unsigned bad = __ballot_sync(0xffffffffu, pv != target);
    unsigned go = 0;
    for (int t = 0; t < nst; ++t)
      if (((pend >> t) & 1u) && t != s && sl[t].ks <= 8 && ((bad >> (8 * t)) & 0xffu) == 0) go |= 1u << t;
    if (go) {
      if (lane == 0)
        for (int t = 0; t < nst; ++t)
          if ((go >> t) & 1u) issue_x(t);
      pend &= ~go;
    }
    // chains stored by earlier items: their stores have had this item's
    // products to land, so the fence before their flags is short
    if (nchains >= f.pub_batch) publish();
    if (flags & 2) {
      if (w.y_buf == 1) {
        store_natural<MT>(a, w.y_tile, ntl, lane, acc);
      } else {
        if (flags & 4) store_tiles_tc<MT>(a.xh + (size_t)w.y_tile * (MT * 64), ntl, lane, acc);
        else store_tiles<MT>(a.xh + (size_t)w.y_tile * (MT * 64), ntl, lane, acc, pol_v);
        if (npub + ntl > PUB_MAX) publish();
        if (lane < ntl) pubs[warp][npub + lane] = (int)(w.y_tile + lane);
        npub += ntl;
        ++nchains;
      }
    }
    __syncwarp();
    if (i + nst < n && !issue(s, i + nst, true)) pend |= 1u << s;
    __syncwarp();
  }
  publish();
  if (timed_out) {
    // report, issue every pending input run (in bounds) so that every stage
    // completes, let the copies in flight land, stop
    if (lane == 0) {
      *reinterpret_cast<volatile int*>(a.err) = 1;
      for (int t = 0; t < nst; ++t)
        if ((pend >> t) & 1u) issue_x(t);
      const long long last = (i + nst < n) ? i + nst : n;
      const long long drain = a.budget > (1LL << 31) ? a.budget : (1LL << 31);
      for (long long j = i; j < last; ++j)
        mbar_wait_until(&bar[j % nst], (uint32_t)((j / nst) & 1), clock64() + drain);
    }
    __syncwarp();
  }
  // failure-detection self-test: after its stream (so that no chain that
  // other warps wait for is held back), the first warp waits, through the
  // same bounded wait, on a barrier nothing completes
  if (a.selftest && blockIdx.x == 0 && warp == 0) {
    const bool ok = mbar_wait_until(&never, 0u, clock64() + a.budget);
    if (lane == 0 && !ok) *reinterpret_cast<volatile int*>(a.err) = 1;
    __syncwarp();
  }
  // the last CTA to finish counts the launch as completed
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(f.epoch + 1, 1u);
    if (done == gridDim.x - 1) {
      f.epoch[1] = 0;
      __threadfence();
      *reinterpret_cast<volatile unsigned*>(f.epoch) = target;
    }
  }
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
// pairs are transposed through shared memory into fragment order.  With
// x_tc, the tile is also written in the tensor-core operand layout (bf16 of
// (n = 16 c + rho, row k) at (n / 8) 64 + (n % 8) 8 + k, c = 2 q + s).
__global__ void __launch_bounds__(256) gather_native_kernel(const double2* __restrict__ s,
                                                            const long long* __restrict__ pperm,
                                                            uint4* __restrict__ x, uint4* __restrict__ x_tc,
                                                            long long nv_tiles, long long Nv, int R, int MT,
                                                            double scale, long long win_lo, long long win_hi) {
  __shared__ __align__(16) uint32_t tile[8][256];
  __shared__ __align__(16) uint16_t ttc[8][512];
  // the first depth launch may start now and stream its factor runs; it
  // reads x only after griddepcontrol.wait, i.e. after this grid completes
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const long long wid = (long long)blockIdx.x * 8 + wb;
  if (wid >= nv_tiles * MT) return;
  const long long rt = wid / MT;
  const int mt = (int)(wid - rt * MT);
  const int r = lane & 7, c0 = 4 * (lane >> 3);
  const long long prow = 8 * rt + r;                    // padded row; outside [win_lo, win_hi) it reads as 0
  const long long nat = (prow >= win_lo && prow < win_hi) ? pperm[prow] : -1;
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
    if (x_tc) {
      const uint16_t part[4] = {(uint16_t)(p.x & 0xffffu), (uint16_t)(p.y & 0xffffu), (uint16_t)(p.x >> 16),
                                (uint16_t)(p.y >> 16)};   // (Re, hi), (Re, lo), (Im, hi), (Im, lo)
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const int n = 16 * cc + q;
        ttc[wb][(n >> 3) * 64 + (n & 7) * 8 + r] = part[cc];
      }
    }
  }
  __syncwarp();
  uint4* out = x + (size_t)wid * 64;   // tile (rt, mt) = rt * MT + mt = wid
  out[lane] = reinterpret_cast<const uint4*>(tile[wb])[lane];
  out[32 + lane] = reinterpret_cast<const uint4*>(tile[wb])[32 + lane];
  if (x_tc) {
    uint4* ot = x_tc + (size_t)wid * 64;
    ot[lane] = reinterpret_cast<const uint4*>(ttc[wb])[lane];
    ot[32 + lane] = reinterpret_cast<const uint4*>(ttc[wb])[32 + lane];
  }
}

void gather_native(const double2* s, const long long* pperm, uint4* x, uint4* x_tc, long long nv_tiles, long long Nv,
                   int R, int MT, double scale, cudaStream_t st, long long win_lo, long long win_hi) {
  const long long warps = nv_tiles * MT;
  if (warps == 0) return;
  gather_native_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(s, pperm, x, x_tc, nv_tiles, Nv, R, MT, scale,
                                                                     win_lo, win_hi);
  HB_CHECK_LAUNCH();
}

// ------------------------------------------------------------- planning ----
struct DepthStreams {
  int grid = 0;
  WItem* d_items = nullptr;
  long long* d_off = nullptr;
  unsigned* d_need = nullptr;   // fused pairs: producer chains per component slot (PAIR_SLOTS per CTA)
};

// The launch shape of one m-tile count: the mode (one launch per depth, or
// one persistent dataflow launch), the item size the chains are cut to, the
// ring stages that fit, the grid, and how many chains a dataflow warp
// publishes together.  Chosen by the autotuner on the first apply (when
// hb_options.autotune is set) or set to the defaults.
struct LaunchShape {
  bool ready = false;
  int mode = 0;
  int item_bytes = ITEM_BYTES;
  int stage = 0, stages = 0, grid = 0;
  int pub = 2;
  int slack = 48;        // dataflow placement: cost units between a producer's finish and its consumer
  bool tc = false;       // mode 0: the leaf outputs on the tensor-core leaf kernel
  bool cones = false;    // mode 0: the first butterfly levels as cones in one launch
  bool pairs = false;    // mode 0: the transfer depths fused in pairs
  bool gridb = false;    // mode 0: every depth in one cooperative launch with grid barriers
  size_t smem = 0;
  double tuned_ms = 0;   // the chosen candidate's time (0: not tuned)
  int candidates = 0;    // candidates the autotuner timed
};

// Chains cut for one (m-tile count, item size) with their warp streams.
struct ChainSet {
  int stage_bytes = 512;                                   // largest item (factor run + input run)
  std::vector<std::vector<std::vector<WItem>>> by_depth;   // [depth][chain] -> items
  std::vector<std::vector<std::pair<long long, int>>> cone_of;   // [depth][chain] -> (cone, level)
  int depth_grid = 0;
  std::vector<DepthStreams> depth_streams;                 // mode 0: one stream set per depth
  int cone_grid = 0;
  DepthStreams cone_streams;                               // mode 0 with cones: the cone launch
  int depth_grid_c = 0;
  std::vector<DepthStreams> depth_streams_c;               // mode 0 with cones: the other chains per depth
  int pair_grid = 0;
  std::vector<DepthStreams> pair_streams;                  // mode 0 with fused level pairs: one per pair
  int gridb_grid = 0;
  DepthStreams gridb_streams;                              // mode 0 with grid barriers: all depths
  int flow_grid = 0;
  std::map<int, DepthStreams> flow_streams;                // mode 1: all depths in one stream set, per slack
};

// The terms of every task, uncut, kept per depth as "term chains": one
// WItem per term (ks = all of its k-steps) for each n-tile group; cut into
// items per (m-tile count, item size) on demand.
struct FlowPlan {
  std::vector<std::vector<std::vector<WItem>>> terms;   // [depth][group chain] -> uncut terms
  std::vector<std::vector<std::pair<long long, long long>>> rows;   // [depth][group chain] -> tree rows it serves
  std::vector<std::vector<std::pair<long long, int>>> cone;         // [depth][group chain] -> (cone, level)
  long long xh_tiles = 0;                               // row tiles the plan writes in xh
  std::map<std::tuple<int, int, int, long long, long long>, ChainSet> sets;   // (MT, item bytes, tc, rows) -> chains
  LaunchShape shape[3];
};

// k-steps per item for groups of ntl n-tiles: the factor run plus the input
// run counted at two m-tiles stays within item_bytes at one m-tile and
// within 13/16 of it at two (so that the largest items at two m-tiles, the
// 12.5 KB of the default 16 KB, still fit 8 warps x 2 stages in 227 KB).
static int item_ks(int ntl, int MT, int item_bytes) {
  const int budget = MT == 1 ? item_bytes : item_bytes * 13 / 16;
  return std::max(1, budget / (512 * ntl + 2048));
}

void flow_plan_build(const std::vector<NatTask>& lt, void** plan_out) {
  FlowPlan* P = new FlowPlan();
  try {
    int maxd = -1;
    for (const NatTask& L : lt) maxd = std::max(maxd, L.depth);
    P->terms.assign((size_t)(maxd + 1), {});
    P->rows.assign((size_t)(maxd + 1), {});
    P->cone.assign((size_t)(maxd + 1), {});
    for (const NatTask& L : lt) {
      if (L.nt <= 0) continue;
      if (L.ng < 1 || L.ng > NTW) throw Error{HB_ERR_UNSUPPORTED, "n-tile group larger than the accumulators"};
      if (L.y_buf == 2) P->xh_tiles = std::max(P->xh_tiles, L.y_tile + L.nt);
      const int ngr = (L.nt + L.ng - 1) / L.ng;
      for (int g = 0; g < ngr; ++g) {
        const int ntl = std::min(L.ng, L.nt - g * L.ng);
        std::vector<WItem> ch;
        for (const NatTerm& tm : L.terms) {
          if (tm.ks <= 0) continue;
          WItem w{};
          w.f_tile = tm.f_tile + (long long)g * L.ng * tm.ks;
          w.x_tile = tm.x_tile;
          w.y_tile = L.y_tile + (long long)g * L.ng;
          w.ks = (short)tm.ks;   // uncut: may exceed an item
          w.ntl = (unsigned char)ntl;
          w.x_buf = (unsigned char)tm.x_buf;
          w.y_buf = (unsigned char)L.y_buf;
          w.flags = L.tc_out ? 4 : 0;   // kept only in the chains of the tensor-core leaf shape
          ch.push_back(w);
        }
        if (ch.empty()) {   // every input is empty: the group is zero
          WItem w{};
          w.y_tile = L.y_tile + (long long)g * L.ng;
          w.ntl = (unsigned char)ntl;
          w.y_buf = (unsigned char)L.y_buf;
          w.flags = L.tc_out ? 4 : 0;
          ch.push_back(w);
        }
        P->terms[(size_t)L.depth].push_back(std::move(ch));
        P->rows[(size_t)L.depth].push_back({L.row_lo, L.row_hi});
        P->cone[(size_t)L.depth].push_back({L.cone, L.cone_level});
      }
    }
    for (const NatTask& L : lt)
      for (const NatTerm& tm : L.terms)
        if (tm.ks > 32767) throw Error{HB_ERR_UNSUPPORTED, "a factor block with more than 262136 inputs"};
  } catch (...) {
    delete P;
    throw;
  }
  *plan_out = P;
}

// The chains of one term chain cut for (MT, item bytes): each term's
// k-steps in runs of at most item_ks; the first item zeroes the
// accumulators, the last stores them.
static void cut_chain(const std::vector<WItem>& tc, int MT, int item_bytes, bool tc_layout, std::vector<WItem>& out,
                      int& stage_bytes) {
  const size_t first = out.size();
  const unsigned char keep = tc_layout ? 4 : 0;   // outputs in the tensor-core operand layout
  for (const WItem& t : tc) {
    if (t.ks == 0) {
      WItem w = t;
      w.flags = t.flags & keep;
      out.push_back(w);
      continue;
    }
    const int kc = item_ks(t.ntl, MT, item_bytes);
    for (int k0 = 0; k0 < t.ks; k0 += kc) {
      WItem w = t;
      w.f_tile = t.f_tile + (long long)k0 * t.ntl;
      w.x_tile = t.x_tile + k0;
      w.ks = (short)std::min(kc, (int)t.ks - k0);
      w.flags = t.flags & keep;
      out.push_back(w);
      stage_bytes = std::max(stage_bytes, (int)t.ntl * (int)w.ks * 512 + (int)w.ks * MT * 1024);
    }
  }
  out[first].flags |= 1;
  out.back().flags |= 2;
}

// The chains for one shape; with tc the last depth (the leaf outputs) is
// left to the tensor-core leaf kernel and the chains feeding it store their
// outputs in its operand layout.
static ChainSet& chain_set(FlowPlan* P, int MT, int item_bytes, bool tc, long long lo = 0, long long hi = -1) {
  auto key = std::make_tuple(MT, item_bytes, tc ? 1 : 0, lo, hi);
  auto it = P->sets.find(key);
  if (it != P->sets.end()) return it->second;
  ChainSet cs;
  const size_t nd = P->terms.size() - (tc ? 1 : 0);
  cs.by_depth.assign(nd, {});
  cs.cone_of.assign(nd, {});
  for (size_t d = 0; d < nd; ++d)
    for (size_t q = 0; q < P->terms[d].size(); ++q) {
      const auto& tch = P->terms[d][q];
      // a shard (hi >= 0) keeps the chains whose rows meet [lo, hi)
      if (hi >= 0 && !(P->rows[d][q].first < hi && P->rows[d][q].second > lo)) continue;
      std::vector<WItem> ch;
      cut_chain(tch, MT, item_bytes, tc, ch, cs.stage_bytes);
      cs.by_depth[d].push_back(std::move(ch));
      cs.cone_of[d].push_back(P->cone[d][q]);
    }
  return P->sets.emplace(key, std::move(cs)).first->second;
}

static void free_streams(DepthStreams& d) {
  dev_free(d.d_items);
  dev_free(d.d_off);
  dev_free(d.d_need);
  d = DepthStreams{};
}

static void free_set(ChainSet& cs) {
  for (DepthStreams& d : cs.depth_streams) free_streams(d);
  cs.depth_streams.clear();
  cs.depth_grid = 0;
  free_streams(cs.cone_streams);
  cs.cone_grid = 0;
  for (DepthStreams& d : cs.depth_streams_c) free_streams(d);
  cs.depth_streams_c.clear();
  cs.depth_grid_c = 0;
  for (DepthStreams& d : cs.pair_streams) free_streams(d);
  cs.pair_streams.clear();
  cs.pair_grid = 0;
  free_streams(cs.gridb_streams);
  cs.gridb_grid = 0;
  for (auto& kv : cs.flow_streams) free_streams(kv.second);
  cs.flow_streams.clear();
  cs.flow_grid = 0;
}

void flow_plan_free(void* plan) {
  FlowPlan* P = static_cast<FlowPlan*>(plan);
  if (!P) return;
  for (auto& kv : P->sets) free_set(kv.second);
  delete P;
}

int flow_plan_depths(const void* plan) { return (int)static_cast<const FlowPlan*>(plan)->terms.size(); }

static long long chain_cost(const std::vector<WItem>& ch) {
  long long w = 0;
  for (const WItem& it : ch) w += (long long)it.ntl * std::max<int>(1, it.ks) + 4;
  return w;
}

static DepthStreams upload_streams(const std::vector<std::vector<const std::vector<WItem>*>>& per, int grid) {
  std::vector<WItem> items;
  std::vector<long long> off;
  size_t total = 0;
  for (const auto& s : per)
    for (const auto* c : s) total += c->size();
  items.reserve(total);
  for (const auto& s : per) {
    off.push_back((long long)items.size());
    for (const auto* c : s) items.insert(items.end(), c->begin(), c->end());
  }
  off.push_back((long long)items.size());
  DepthStreams ds;
  ds.grid = grid;
  ds.d_items = upload(items);
  try {
    ds.d_off = upload(off);
  } catch (...) {
    dev_free(ds.d_items);
    throw;
  }
  HB_CUDA(cudaDeviceSynchronize());
  return ds;
}

// Mode 0: deal every depth's chains over grid x NWARP warp streams, longest
// chain (in factor tiles, plus a fixed cost per item) first, to the stream
// with the least work so far.
static void build_depth_streams(ChainSet& cs, int grid, bool skip_cones = false) {
  std::vector<DepthStreams>& out = skip_cones ? cs.depth_streams_c : cs.depth_streams;
  for (DepthStreams& d : out) free_streams(d);
  out.clear();
  const int ns = grid * NWARP;
  for (size_t dd = 0; dd < cs.by_depth.size(); ++dd) {
    const auto& chains = cs.by_depth[dd];
    std::vector<size_t> order;
    for (size_t c = 0; c < chains.size(); ++c)
      if (!skip_cones || cs.cone_of[dd][c].first < 0) order.push_back(c);
    if (order.empty()) {
      out.push_back(DepthStreams{});
      continue;
    }
    std::vector<long long> cost(chains.size());
    for (size_t c = 0; c < chains.size(); ++c) cost[c] = chain_cost(chains[c]);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    using Load = std::pair<long long, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
    for (int s = 0; s < ns; ++s) pq.push({0, s});
    std::vector<std::vector<const std::vector<WItem>*>> per((size_t)ns);
    for (size_t c : order) {
      Load l = pq.top();
      pq.pop();
      per[(size_t)l.second].push_back(&chains[c]);
      l.first += cost[c];
      pq.push(l);
    }
    out.push_back(upload_streams(per, grid));
  }
  (skip_cones ? cs.depth_grid_c : cs.depth_grid) = grid;
}

// Mode 0 with cones: the chains of every cone (the first butterfly levels,
// tasks with cone >= 0) in one launch.  Whole cones go to CTAs (largest
// first to the least-loaded CTA); within a CTA each cone's levels are dealt
// to its NWARP warps level by level (largest chain first to the warp with
// the least work in that level), and every warp gets a barrier record after
// each level but the cone's last, so all warps of the CTA hold the same
// barriers in the same order.
static void build_cone_streams(ChainSet& cs, int grid) {
  free_streams(cs.cone_streams);
  static const std::vector<WItem> barrier_rec = [] {
    WItem w{};
    w.flags = 8;
    return std::vector<WItem>{w};
  }();
  std::map<long long, std::vector<std::vector<const std::vector<WItem>*>>> cones;   // cone -> level -> chains
  std::map<long long, long long> cone_cost;
  for (size_t d = 0; d < cs.by_depth.size(); ++d)
    for (size_t q = 0; q < cs.by_depth[d].size(); ++q) {
      const auto& ci = cs.cone_of[d][q];
      if (ci.first < 0) continue;
      auto& lv = cones[ci.first];
      if ((int)lv.size() <= ci.second) lv.resize((size_t)ci.second + 1);
      lv[(size_t)ci.second].push_back(&cs.by_depth[d][q]);
      cone_cost[ci.first] += chain_cost(cs.by_depth[d][q]);
    }
  std::vector<long long> ids;
  for (const auto& kv : cones) ids.push_back(kv.first);
  std::stable_sort(ids.begin(), ids.end(), [&](long long x, long long y) { return cone_cost[x] > cone_cost[y]; });
  using Load = std::pair<long long, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
  for (int b = 0; b < grid; ++b) pq.push({0, b});
  std::vector<std::vector<long long>> of_cta((size_t)grid);
  for (long long id : ids) {
    Load l = pq.top();
    pq.pop();
    of_cta[(size_t)l.second].push_back(id);
    l.first += cone_cost[id];
    pq.push(l);
  }
  std::vector<std::vector<const std::vector<WItem>*>> per((size_t)grid * NWARP);
  for (int b = 0; b < grid; ++b)
    for (long long id : of_cta[(size_t)b]) {
      const auto& lv = cones[id];
      for (size_t k = 0; k < lv.size(); ++k) {
        std::vector<const std::vector<WItem>*> chs = lv[k];
        std::stable_sort(chs.begin(), chs.end(),
                         [](const std::vector<WItem>* x, const std::vector<WItem>* y) { return chain_cost(*x) > chain_cost(*y); });
        long long load[NWARP] = {};
        for (const auto* c : chs) {
          int wmin = 0;
          for (int w = 1; w < NWARP; ++w)
            if (load[w] < load[wmin]) wmin = w;
          per[(size_t)b * NWARP + wmin].push_back(c);
          load[wmin] += chain_cost(*c);
        }
        if (k + 1 < lv.size())
          for (int w = 0; w < NWARP; ++w) per[(size_t)b * NWARP + w].push_back(&barrier_rec);
      }
    }
  cs.cone_streams = upload_streams(per, grid);
  cs.cone_grid = grid;
}

// Mode 0 with grid barriers: every depth in one cooperative launch.  Each
// depth's chains are dealt to the grid x NWARP warps as in the per-depth
// launches (largest first to the least-loaded warp), and every warp gets a
// barrier record between consecutive non-empty depths, so all warps hold the
// same barriers in the same order; at a barrier the CTA's warps meet, one
// warp counts the CTA in at gpu scope and waits for the whole grid.
static void build_gridb_streams(ChainSet& cs, int grid) {
  free_streams(cs.gridb_streams);
  static const std::vector<WItem> barrier_rec = [] {
    WItem w{};
    w.flags = 8;
    return std::vector<WItem>{w};
  }();
  const int ns = grid * NWARP;
  std::vector<std::vector<const std::vector<WItem>*>> per((size_t)ns);
  bool any = false;
  for (size_t dd = 0; dd < cs.by_depth.size(); ++dd) {
    const auto& chains = cs.by_depth[dd];
    if (chains.empty()) continue;
    if (any)
      for (auto& p : per) p.push_back(&barrier_rec);
    any = true;
    std::vector<long long> cost(chains.size());
    std::vector<size_t> order(chains.size());
    for (size_t c = 0; c < chains.size(); ++c) {
      cost[c] = chain_cost(chains[c]);
      order[c] = c;
    }
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    using Load = std::pair<long long, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
    for (int st = 0; st < ns; ++st) pq.push({0, st});
    for (size_t c : order) {
      Load l = pq.top();
      pq.pop();
      per[(size_t)l.second].push_back(&chains[c]);
      l.first += cost[c];
      pq.push(l);
    }
  }
  cs.gridb_streams = upload_streams(per, grid);
  cs.gridb_grid = grid;
}

// Mode 0 with fused level pairs: the transfer depths (all but the leaf
// outputs) in pairs (2P, 2P + 1), one launch per pair.  A chain of depth
// 2P + 1 reads only skeleton tiles written at depth 2P.  Each connected
// component of that producer / consumer relation (a level k + 1 block reads
// two level k blocks, which feed one other block besides) goes to one CTA
// whole, largest first to the least-loaded CTA; there its chains are spread
// over the warps, each to the least-loaded one, every warp running all its
// producer chains before any consumer chain.  A component with consumers
// gets a slot of its CTA: the last item of each of its producer chains is
// flagged (flags & 32), every item of its consumers too (flags & 16), both
// carrying the slot in `pad`, and d_need holds the slot's producer count.
// The kernel counts a slot down in shared memory as the producers store,
// and a consumer's input run (other warps' outputs) goes out once the count
// is zero.  Producers wait for nothing of their own launch, and every warp
// runs its producers first, so every wait ends.  The last pair may hold one
// depth; the leaf outputs follow in their own launch.
static void build_pair_streams(ChainSet& cs, int grid, int ndepth) {
  for (DepthStreams& d : cs.pair_streams) free_streams(d);
  cs.pair_streams.clear();
  const int ns = grid * NWARP;
  for (int d0 = 0; d0 < ndepth; d0 += 2) {
    const auto& P = cs.by_depth[(size_t)d0];
    static const std::vector<std::vector<WItem>> none;
    const auto& C = (d0 + 1 < ndepth) ? cs.by_depth[(size_t)d0 + 1] : none;
    const size_t np = P.size(), nc = C.size(), nt = np + nc;
    // union-find over producers [0, np) and consumers [np, np + nc)
    std::vector<size_t> parent(nt);
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](size_t x) {
      while (parent[x] != x) x = parent[x] = parent[parent[x]];
      return x;
    };
    std::map<long long, size_t> prod;   // xh tile -> producer chain
    for (size_t c = 0; c < np; ++c) {
      const WItem& w = P[c].back();
      if (!(w.flags & 2)) throw Error{HB_ERR_STATE, "a producer chain does not end in a store"};
      if (w.y_buf == 2)
        for (int j = 0; j < w.ntl; ++j) prod[w.y_tile + j] = c;
    }
    for (size_t c = 0; c < nc; ++c)
      for (const WItem& w : C[c]) {
        if (w.ks == 0) continue;
        if (w.x_buf != 2) throw Error{HB_ERR_STATE, "a paired consumer reads the input vector"};
        for (int j = 0; j < w.ks; ++j) {
          const auto it = prod.find(w.x_tile + j);
          if (it == prod.end()) throw Error{HB_ERR_STATE, "a paired consumer reads a tile of another depth"};
          const size_t a = find(np + c), b = find(it->second);
          if (a != b) parent[a] = b;
        }
      }
    std::vector<long long> cost(nt);
    for (size_t t = 0; t < nt; ++t) cost[t] = chain_cost(t < np ? P[t] : C[t - np]);
    std::map<size_t, std::vector<size_t>> comp;   // root -> members
    for (size_t t = 0; t < nt; ++t) comp[find(t)].push_back(t);
    std::vector<std::pair<long long, size_t>> order;   // (cost, root)
    for (auto& kv : comp) {
      long long w = 0;
      for (size_t t : kv.second) w += cost[t];
      std::stable_sort(kv.second.begin(), kv.second.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
      order.push_back({w, kv.first});
    }
    std::stable_sort(order.begin(), order.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    using Load = std::pair<long long, int>;
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
    for (int b = 0; b < grid; ++b) pq.push({0, b});
    std::vector<std::vector<size_t>> of_cta((size_t)grid);   // component roots
    for (const auto& o : order) {
      Load l = pq.top();
      pq.pop();
      of_cta[(size_t)l.second].push_back(o.second);
      l.first += o.first;
      pq.push(l);
    }
    std::vector<std::vector<WItem>> sw((size_t)ns);
    std::vector<unsigned> need((size_t)grid * PAIR_SLOTS, 0u);
    for (int b = 0; b < grid; ++b) {
      long long load[NWARP] = {};
      auto least = [&]() {
        int m = 0;
        for (int w = 1; w < NWARP; ++w)
          if (load[w] < load[m]) m = w;
        return m;
      };
      std::vector<std::vector<WItem>> cons((size_t)NWARP);
      std::vector<int> slot_of(of_cta[(size_t)b].size(), -1);
      int slots = 0;
      for (size_t k = 0; k < of_cta[(size_t)b].size(); ++k) {
        const auto& mem = comp[of_cta[(size_t)b][k]];
        const bool has_cons = std::any_of(mem.begin(), mem.end(), [&](size_t t) { return t >= np; });
        if (!has_cons) continue;
        if (slots == PAIR_SLOTS) throw Error{HB_ERR_UNSUPPORTED, "more paired components on a CTA than slots"};
        slot_of[k] = slots++;
      }
      for (size_t k = 0; k < of_cta[(size_t)b].size(); ++k)
        for (size_t t : comp[of_cta[(size_t)b][k]]) {
          if (t >= np) continue;
          const int w = least();
          auto& out = sw[(size_t)b * NWARP + w];
          out.insert(out.end(), P[t].begin(), P[t].end());
          if (slot_of[k] >= 0) {
            out.back().flags |= 32;
            out.back().pad = (short)slot_of[k];
            ++need[(size_t)b * PAIR_SLOTS + slot_of[k]];
          }
          load[w] += cost[t];
        }
      for (size_t k = 0; k < of_cta[(size_t)b].size(); ++k)
        for (size_t t : comp[of_cta[(size_t)b][k]]) {
          if (t < np) continue;
          const int w = least();
          for (WItem it : C[t - np]) {
            it.flags |= 16;
            it.pad = (short)slot_of[k];
            cons[(size_t)w].push_back(it);
          }
          load[w] += cost[t];
        }
      for (int w = 0; w < NWARP; ++w) {
        auto& out = sw[(size_t)b * NWARP + w];
        out.insert(out.end(), cons[(size_t)w].begin(), cons[(size_t)w].end());
      }
    }
    std::vector<WItem> items;
    std::vector<long long> off;
    for (int st = 0; st < ns; ++st) {
      off.push_back((long long)items.size());
      items.insert(items.end(), sw[(size_t)st].begin(), sw[(size_t)st].end());
    }
    off.push_back((long long)items.size());
    DepthStreams ds;
    ds.grid = grid;
    try {
      ds.d_items = upload(items);
      ds.d_off = upload(off);
      ds.d_need = upload(need);
    } catch (...) {
      free_streams(ds);
      throw;
    }
    HB_CUDA(cudaDeviceSynchronize());
    cs.pair_streams.push_back(ds);
  }
  cs.pair_grid = grid;
}

// Mode 1: one stream set over all depths, placed by simulating the schedule.
// Chain costs as above; item k of a chain starts at (chain start + the cost
// of the chain's items before it), and must not start before every chain
// writing an xh row tile it reads has finished plus `slack` (time for the
// producer to publish and for this warp's prefetch to see it); the gather,
// which every warp runs first, counts as finished at a fixed time.  Chains
// are taken in order of their ready time and put on the stream that frees
// first; start = max(stream free, ready), finish = start + cost.  Each
// stream therefore runs its items in increasing simulated start time, and
// every producer's last item starts strictly before any item that reads
// its output - the order the kernel's deadlock freedom rests on.
static void build_flow_streams(ChainSet& cs, int grid, int slack, long long xh_tiles, long long nv_tiles, int MT) {
  auto old = cs.flow_streams.find(slack);
  if (old != cs.flow_streams.end()) {
    free_streams(old->second);
    cs.flow_streams.erase(old);
  }
  const int ns = grid * NWARP;
  std::vector<const std::vector<WItem>*> ch;
  for (const auto& chains : cs.by_depth)
    for (const auto& c : chains) ch.push_back(&c);
  const size_t nc = ch.size();
  std::vector<long long> cost(nc);
  for (size_t c = 0; c < nc; ++c) cost[c] = chain_cost(*ch[c]);
  // producer of every xh row tile
  std::vector<int> prod((size_t)std::max<long long>(xh_tiles, 1), -1);
  for (size_t c = 0; c < nc; ++c) {
    const WItem& w = ch[c]->back();
    if (w.y_buf == 2)
      for (int j = 0; j < w.ntl; ++j) prod[(size_t)(w.y_tile + j)] = (int)c;
  }
  // producers of every chain with the smallest prefix cost of an item that
  // reads them; consumers as CSR of (chain, prefix)
  std::vector<int> npend(nc, 0);
  std::vector<std::vector<std::pair<int, long long>>> prods(nc);
  for (size_t c = 0; c < nc; ++c) {
    auto& ps = prods[c];
    long long prefix = 0;
    for (const WItem& w : *ch[c]) {
      if (w.x_buf == 2)
        for (int j = 0; j < w.ks; ++j) {
          const int p = prod[(size_t)(w.x_tile + j)];
          if (p < 0) throw Error{HB_ERR_STATE, "a chain reads a skeleton row tile no chain writes"};
          ps.push_back({p, prefix});
        }
      prefix += (long long)w.ntl * std::max<int>(1, w.ks) + 4;
    }
    std::sort(ps.begin(), ps.end());   // by producer, smallest prefix first
    size_t m = 0;
    for (size_t q = 0; q < ps.size(); ++q)
      if (m == 0 || ps[q].first != ps[m - 1].first) ps[m++] = ps[q];
    ps.resize(m);
    npend[c] = (int)m;
  }
  std::vector<long long> cons_off(nc + 1, 0);
  for (size_t c = 0; c < nc; ++c)
    for (const auto& pp : prods[c]) ++cons_off[(size_t)pp.first + 1];
  for (size_t c = 0; c < nc; ++c) cons_off[c + 1] += cons_off[c];
  std::vector<std::pair<int, long long>> cons((size_t)cons_off[nc]);
  {
    std::vector<long long> fill(cons_off.begin(), cons_off.end() - 1);
    for (size_t c = 0; c < nc; ++c)
      for (const auto& pp : prods[c]) cons[(size_t)fill[(size_t)pp.first]++] = {(int)c, pp.second};
  }
  std::vector<std::vector<std::pair<int, long long>>>().swap(prods);
  const long long gather_done = 4LL * MT * ((nv_tiles + ns - 1) / ns);
  std::vector<long long> ready(nc, gather_done);
  using Ev = std::pair<long long, int>;   // (ready, chain)
  std::priority_queue<Ev, std::vector<Ev>, std::greater<Ev>> rq;
  for (size_t c = 0; c < nc; ++c)
    if (npend[c] == 0) rq.push({ready[c], (int)c});
  using Load = std::pair<long long, int>;   // (free at, stream)
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> sq;
  for (int s = 0; s < ns; ++s) sq.push({gather_done, s});
  std::vector<std::vector<const std::vector<WItem>*>> per((size_t)ns);
  size_t placed = 0;
  while (!rq.empty()) {
    const Ev e = rq.top();
    rq.pop();
    Load l = sq.top();
    sq.pop();
    const long long start = std::max(l.first, e.first);
    const long long fin = start + cost[(size_t)e.second];
    per[(size_t)l.second].push_back(ch[(size_t)e.second]);
    l.first = fin;
    sq.push(l);
    ++placed;
    for (long long q = cons_off[(size_t)e.second]; q < cons_off[(size_t)e.second + 1]; ++q) {
      const int c = cons[(size_t)q].first;
      ready[(size_t)c] = std::max(ready[(size_t)c], fin + slack - cons[(size_t)q].second);
      if (--npend[(size_t)c] == 0) rq.push({ready[(size_t)c], c});
    }
  }
  if (placed != nc) throw Error{HB_ERR_STATE, "the chain dependencies have a cycle"};
  cs.flow_streams[slack] = upload_streams(per, grid);
  cs.flow_grid = grid;
}

template <int MT>
static void set_shape(FlowPlan* P, LaunchShape& L, int mode, int item_bytes, int pub, int slack, bool tc,
                      bool cones = false, bool pairs = false, bool gridb = false) {
  int dev = 0, nsm = 0, optin = 0;
  HB_CUDA(cudaGetDevice(&dev));
  HB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  HB_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (tc && mode != 0) throw Error{HB_ERR_UNSUPPORTED, "the tensor-core leaf kernel runs with one launch per depth"};
  if (cones && mode != 0) throw Error{HB_ERR_UNSUPPORTED, "cones run with one launch per depth"};
  ChainSet& cs = chain_set(P, MT, item_bytes, tc);
  if (cones && pairs) throw Error{HB_ERR_UNSUPPORTED, "cones and fused pairs do not combine"};
  if (gridb && (mode != 0 || tc || cones || pairs))
    throw Error{HB_ERR_UNSUPPORTED, "grid barriers run every depth on the step kernel alone"};
  L.tc = tc;
  L.cones = cones;
  L.pairs = pairs;
  L.gridb = gridb;
  cudaFuncAttributes fa{};
  const void* k = mode == 0 ? (cones   ? (const void*)bf_step_kernel<MT, 1>
                              : gridb ? (const void*)bf_step_kernel<MT, 3>
                                      : (const void*)bf_step_kernel<MT, 0>)
                            : (const void*)bf_flow_kernel<MT>;
  HB_CUDA(cudaFuncGetAttributes(&fa, k));
  L.mode = mode;
  L.item_bytes = item_bytes;
  L.pub = pub;
  L.slack = slack;
  L.stage = cs.stage_bytes;
  size_t stat = fa.sharedSizeBytes;
  if (pairs) {   // the pair launches hold the component counters besides
    cudaFuncAttributes fp{};
    HB_CUDA(cudaFuncGetAttributes(&fp, (const void*)bf_step_kernel<MT, 2>));
    stat = std::max(stat, fp.sharedSizeBytes);
  }
  const int avail = optin - (int)stat;
  L.stages = std::min(MAX_STAGES, avail / (NWARP * L.stage));
  if (L.stages < 2) throw Error{HB_ERR_UNSUPPORTED, "step kernel stages do not fit in shared memory"};
  L.smem = (size_t)NWARP * L.stages * L.stage;
  // the kernel may take any size up to the opt-in limit (both directions' plans share it)
  HB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, avail));
  if (cones || pairs) {   // the other launches of the shape, each up to its own limit
    for (const void* o : {(const void*)bf_step_kernel<MT, 0>, (const void*)bf_step_kernel<MT, 2>}) {
      cudaFuncAttributes fo{};
      HB_CUDA(cudaFuncGetAttributes(&fo, o));
      HB_CUDA(cudaFuncSetAttribute(o, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fo.sharedSizeBytes));
    }
  }
  int per_sm = 0;
  HB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NWARP * 32, L.smem));
  if (per_sm < 1) throw Error{HB_ERR_UNSUPPORTED, "step kernel does not fit on an SM"};
  L.grid = nsm * per_sm;
  L.ready = true;
}

struct LaunchCtx {
  const uint4* F;
  const double2* s;
  double scale;
  uint4* x;
  uint4* x_tc;
  void* tc_plan;
  const void* F_tc;
  uint4* xh;
  double2* u;
  const long long* pperm;
  long long Nv, nv_tiles;
  int R;
  unsigned* flags;
  unsigned* epoch;
  int* err;
  long long budget;
  bool selftest;
  cudaStream_t st;
};

template <int MT>
static void launch_shape(FlowPlan* P, const LaunchShape& L, const LaunchCtx& c,
                         const std::function<void(int, bool)>& timer) {
  ChainSet& cs = chain_set(P, MT, L.item_bytes, L.tc);
  if (L.mode == 0) {
    gather_native(c.s, c.pperm, c.x, L.tc ? c.x_tc : nullptr, c.nv_tiles, c.Nv, c.R, MT, c.scale, c.st);
    bool first = true;   // the timer brackets all depth launches (PDL stays intact)
    auto launch = [&](const DepthStreams& ds, bool cone_kernel) {
      StepArgs args{ds.d_items, ds.d_off, c.F, c.x, c.xh, c.u, c.pperm, c.Nv, c.R, L.stages, L.stage, c.budget,
                    c.err, c.selftest ? 1 : 0};
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(ds.grid);
      cfg.blockDim = dim3(NWARP * 32);
      cfg.dynamicSmemBytes = L.smem;
      cfg.stream = c.st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (first) timer(0, true);
      first = false;
      if (cone_kernel) HB_CUDA(cudaLaunchKernelEx(&cfg, bf_step_kernel<MT, 1>, args));
      else HB_CUDA(cudaLaunchKernelEx(&cfg, bf_step_kernel<MT, 0>, args));
    };
    if (L.gridb) {
      // one cooperative launch (every CTA resident: the grid barriers)
      if (cs.gridb_grid != L.grid) build_gridb_streams(cs, L.grid);
      const DepthStreams& ds = cs.gridb_streams;
      StepArgs args{ds.d_items, ds.d_off, c.F, c.x, c.xh, c.u, c.pperm, c.Nv, c.R, L.stages, L.stage, c.budget,
                    c.err, c.selftest ? 1 : 0, nullptr, c.epoch + 2};
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(ds.grid);
      cfg.blockDim = dim3(NWARP * 32);
      cfg.dynamicSmemBytes = L.smem;
      cfg.stream = c.st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      timer(0, true);
      HB_CUDA(cudaLaunchKernelEx(&cfg, bf_step_kernel<MT, 3>, args));
      timer(0, false);
      return;
    }
    if (L.pairs) {
      const int ntransfer = (int)P->terms.size() - 1;   // every depth but the leaf outputs
      if (cs.pair_grid != L.grid) build_pair_streams(cs, L.grid, ntransfer);
      for (const DepthStreams& ds : cs.pair_streams) {
        StepArgs args{ds.d_items, ds.d_off, c.F, c.x, c.xh, c.u, c.pperm, c.Nv, c.R, L.stages, L.stage, c.budget,
                      c.err, c.selftest ? 1 : 0, ds.d_need};
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(ds.grid);
        cfg.blockDim = dim3(NWARP * 32);
        cfg.dynamicSmemBytes = L.smem;
        cfg.stream = c.st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (first) timer(0, true);
        first = false;
        HB_CUDA(cudaLaunchKernelEx(&cfg, bf_step_kernel<MT, 2>, args));
      }
      if (L.tc) {
        tc_leaf_launch(c.tc_plan, MT, c.F_tc, c.x_tc, c.xh, c.u, c.pperm, c.Nv, c.R, c.err, c.budget, c.st);
      } else {
        if (cs.depth_grid != L.grid) build_depth_streams(cs, L.grid);
        launch(cs.depth_streams.back(), false);   // the leaf outputs
      }
      timer(0, false);
      return;
    }
    if (L.cones) {
      if (cs.cone_grid != L.grid) build_cone_streams(cs, L.grid);
      if (cs.depth_grid_c != L.grid) build_depth_streams(cs, L.grid, true);
      launch(cs.cone_streams, true);
      for (const DepthStreams& ds : cs.depth_streams_c)
        if (ds.grid) launch(ds, false);
      if (L.tc) {
        tc_leaf_launch(c.tc_plan, MT, c.F_tc, c.x_tc, c.xh, c.u, c.pperm, c.Nv, c.R, c.err, c.budget, c.st);
      }
      timer(0, false);
      return;
    }
    if (cs.depth_grid != L.grid) build_depth_streams(cs, L.grid);
    for (const DepthStreams& ds : cs.depth_streams) {
      if (ds.grid == 0) continue;
      StepArgs args{ds.d_items, ds.d_off, c.F, c.x, c.xh, c.u, c.pperm, c.Nv, c.R, L.stages, L.stage, c.budget,
                    c.err, c.selftest ? 1 : 0};
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(ds.grid);
      cfg.blockDim = dim3(NWARP * 32);
      cfg.dynamicSmemBytes = L.smem;
      cfg.stream = c.st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (first) timer(0, true);
      first = false;
      HB_CUDA(cudaLaunchKernelEx(&cfg, bf_step_kernel<MT, 0>, args));
    }
    if (L.tc) {   // the leaf outputs (the last depth) on the tensor cores
      if (first) timer(0, true);
      first = false;
      tc_leaf_launch(c.tc_plan, MT, c.F_tc, c.x_tc, c.xh, c.u, c.pperm, c.Nv, c.R, c.err, c.budget, c.st);
    }
    if (!first) timer(0, false);
    return;
  }
  if (cs.flow_grid != L.grid) {
    for (auto& kv : cs.flow_streams) free_streams(kv.second);
    cs.flow_streams.clear();
  }
  if (!cs.flow_streams.count(L.slack)) build_flow_streams(cs, L.grid, L.slack, P->xh_tiles, c.nv_tiles, MT);
  const DepthStreams& fs = cs.flow_streams[L.slack];
  FlowArgs fa{};
  fa.a = StepArgs{fs.d_items, fs.d_off, c.F, c.x, c.xh, c.u, c.pperm, c.Nv, c.R,
                  L.stages, L.stage, c.budget, c.err, c.selftest ? 1 : 0};
  fa.s = c.s;
  fa.scale = c.scale;
  fa.nv_tiles = c.nv_tiles;
  fa.flags = c.flags;
  fa.epoch = c.epoch;
  fa.pub_batch = L.pub;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(L.grid);
  cfg.blockDim = dim3(NWARP * 32);
  cfg.dynamicSmemBytes = L.smem;
  cfg.stream = c.st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // every CTA resident: chains wait on one another
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  timer(0, true);
  HB_CUDA(cudaLaunchKernelEx(&cfg, bf_flow_kernel<MT>, fa));
  timer(0, false);
}

// The autotuner: time every candidate shape (each a full apply of these
// right-hand sides, one untimed run then the best of three, CUDA events on
// the caller's stream) and keep the fastest.  Candidates: one launch per
// depth, the cone launch, fused level pairs and grid barriers, each at 16 KB
// and 8 KB items and (but grid barriers) with the tensor-core leaf kernel;
// the dataflow launch at 16 KB and 8 KB items with 1 and 4 chains per
// publication and three placement slacks.  Only the winner's streams are
// kept.
template <int MT>
static void autotune(FlowPlan* P, LaunchShape& L, const LaunchCtx& c) {
  struct Cand {
    int mode, item_bytes, pub, slack, tc, cones;   // cones: 1 = cone launch, 2 = fused level pairs, 3 = grid barriers
  };
  const Cand cands[] = {{0, 16384, 1, 0, 0, 0},  {0, 8192, 1, 0, 0, 0},   {0, 16384, 1, 0, 1, 0},
                        {0, 8192, 1, 0, 1, 0},   {0, 16384, 1, 0, 0, 1},  {0, 8192, 1, 0, 0, 1},
                        {0, 16384, 1, 0, 1, 1},  {0, 16384, 1, 0, 0, 2},  {0, 16384, 1, 0, 1, 2},
                        {0, 8192, 1, 0, 0, 2},   {1, 16384, 1, 16, 0, 0}, {1, 16384, 1, 48, 0, 0},
                        {1, 16384, 1, 128, 0, 0}, {1, 16384, 4, 48, 0, 0}, {1, 8192, 1, 16, 0, 0},
                        {1, 8192, 1, 48, 0, 0},  {1, 8192, 1, 128, 0, 0}, {0, 16384, 1, 0, 0, 3},
                        {0, 8192, 1, 0, 0, 3}};
  cudaEvent_t e0, e1;
  HB_CUDA(cudaEventCreate(&e0));
  HB_CUDA(cudaEventCreate(&e1));
  auto none = [](int, bool) {};
  double best = 1e30;
  LaunchShape win;
  int timed = 0;
  try {
    for (const Cand& k : cands) {
      LaunchShape T;
      try {
        set_shape<MT>(P, T, k.mode, k.item_bytes, k.pub, k.slack, k.tc != 0, k.cones == 1, k.cones == 2,
                      k.cones == 3);
      } catch (const Error&) {
        continue;   // does not fit: not a candidate
      }
      launch_shape<MT>(P, T, c, none);
      float ms = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        HB_CUDA(cudaEventRecord(e0, c.st));
        launch_shape<MT>(P, T, c, none);
        HB_CUDA(cudaEventRecord(e1, c.st));
        HB_CUDA(cudaEventSynchronize(e1));
        float t = 0;
        HB_CUDA(cudaEventElapsedTime(&t, e0, e1));
        ms = std::min(ms, t);
      }
      ++timed;
      if (ms < best) {
        best = ms;
        win = T;
      }
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!timed) throw Error{HB_ERR_UNSUPPORTED, "no launch shape fits"};
  win.tuned_ms = best;
  win.candidates = timed;
  L = win;
  // keep only the winner's chains and streams
  for (auto it = P->sets.begin(); it != P->sets.end();) {
    if (std::get<0>(it->first) == MT && std::get<4>(it->first) < 0 &&
        (std::get<1>(it->first) != L.item_bytes || std::get<2>(it->first) != (L.tc ? 1 : 0))) {
      free_set(it->second);
      it = P->sets.erase(it);
    } else {
      ++it;
    }
  }
  ChainSet& cs = chain_set(P, MT, L.item_bytes, L.tc);
  for (auto it = cs.flow_streams.begin(); it != cs.flow_streams.end();) {
    if (L.mode == 0 || it->first != L.slack) {
      free_streams(it->second);
      it = cs.flow_streams.erase(it);
    } else {
      ++it;
    }
  }
  if (L.mode == 1) {
    for (DepthStreams& d : cs.depth_streams) free_streams(d);
    cs.depth_streams.clear();
    cs.depth_grid = 0;
  }
}

template <int MT>
static void run_mt(FlowPlan* P, const LaunchCtx& c, int tune, const std::function<void(int, bool)>& timer) {
  LaunchShape& L = P->shape[MT];
  if (!L.ready) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    HB_CUDA(cudaStreamIsCapturing(c.st, &cap));
    if (tune == 1 && cap == cudaStreamCaptureStatusNone) autotune<MT>(P, L, c);
    else if (tune == 2) set_shape<MT>(P, L, 1, ITEM_BYTES, 1, 48, false);
    else if (tune == 3) set_shape<MT>(P, L, 0, ITEM_BYTES, 1, 0, true);
    else if (tune == 4) set_shape<MT>(P, L, 0, ITEM_BYTES, 1, 0, false, true);
    else if (tune == 5) set_shape<MT>(P, L, 0, ITEM_BYTES, 1, 0, false, false, true);
    else if (tune == 6) set_shape<MT>(P, L, 0, ITEM_BYTES, 1, 0, false, false, false, true);
    else set_shape<MT>(P, L, 0, ITEM_BYTES, 1, 0, false);
  }
  launch_shape<MT>(P, L, c, timer);
}

void flow_launch(void* plan, void* tc_plan, const void* F_tc, const uint4* F, const double2* s, double scale,
                 uint4* x, uint4* x_tc, uint4* xh, double2* u, const long long* pperm, long long Nv,
                 long long nv_tiles, int R, unsigned* flags, unsigned* epoch, int* err, long long budget_cycles,
                 bool selftest, int autotune_on, cudaStream_t st, const std::function<void(int, bool)>& timer) {
  FlowPlan* P = static_cast<FlowPlan*>(plan);
  if (P->terms.empty()) return;
  const int MT = (R + 15) / 16;
  const LaunchCtx c{F,     s,      scale, x,    x_tc,          tc_plan,  F_tc, xh, u, pperm, Nv, nv_tiles, R,
                    flags, epoch, err,   budget_cycles, selftest, st};
  if (MT == 1) run_mt<1>(P, c, autotune_on, timer);
  else if (MT == 2) run_mt<2>(P, c, autotune_on, timer);
  else throw Error{HB_ERR_UNSUPPORTED, "the mixed apply takes 1 or 2 m-tiles of 16 right-hand sides per pass"};
}

template <int MT>
static void launch_shard_mt(FlowPlan* P, const LaunchCtx& c, long long lo, long long hi, long long pad_lo,
                            long long pad_hi, bool adjoint, long long xh_tiles) {
  // per-depth launches over the shard's chains, shaped like the default
  ChainSet& cs = chain_set(P, MT, ITEM_BYTES, false, lo, hi);
  LaunchShape L;
  set_shape<MT>(P, L, 0, ITEM_BYTES, 1, 0, false);
  L.stage = std::max(L.stage, cs.stage_bytes);
  gather_native(c.s, c.pperm, c.x, nullptr, c.nv_tiles, c.Nv, c.R, MT, c.scale, c.st, pad_lo, pad_hi);
  if (adjoint)   // the skeleton vectors of the other shards' rows read as zero
    HB_CUDA(cudaMemsetAsync(c.xh, 0, (size_t)std::max<long long>(xh_tiles, 1) * MT * 1024, c.st));
  if (cs.depth_grid != L.grid) build_depth_streams(cs, L.grid);
  for (const DepthStreams& ds : cs.depth_streams) {
    if (ds.grid == 0) continue;
    StepArgs args{ds.d_items, ds.d_off, c.F, c.x, c.xh, c.u, c.pperm, c.Nv, c.R, L.stages, L.stage, c.budget,
                  c.err, 0};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ds.grid);
    cfg.blockDim = dim3(NWARP * 32);
    cfg.dynamicSmemBytes = L.smem;
    cfg.stream = c.st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    HB_CUDA(cudaLaunchKernelEx(&cfg, bf_step_kernel<MT, 0>, args));
  }
}

void flow_launch_shard(void* plan, const uint4* F, const double2* s, double scale, uint4* x, uint4* xh,
                       long long xh_tiles, double2* u, const long long* pperm, long long Nv, long long nv_tiles,
                       int R, long long row_lo, long long row_hi, long long pad_lo, long long pad_hi, bool adjoint,
                       int* err, long long budget, cudaStream_t st) {
  FlowPlan* P = static_cast<FlowPlan*>(plan);
  if (P->terms.empty()) return;
  const int MT = (R + 15) / 16;
  const LaunchCtx c{F, s, scale, x, nullptr, nullptr, nullptr, xh, u, pperm, Nv, nv_tiles, R, nullptr, nullptr,
                    err, budget, false, st};
  if (MT == 1) launch_shard_mt<1>(P, c, row_lo, row_hi, pad_lo, pad_hi, adjoint, xh_tiles);
  else if (MT == 2) launch_shard_mt<2>(P, c, row_lo, row_hi, pad_lo, pad_hi, adjoint, xh_tiles);
  else throw Error{HB_ERR_UNSUPPORTED, "the mixed apply takes 1 or 2 m-tiles of 16 right-hand sides per pass"};
}

void flow_shape(const void* plan, int MT, int* mode, int* item_bytes, int* stages, int* pub, int* slack,
                double* tuned_ms, int* candidates) {
  const FlowPlan* P = static_cast<const FlowPlan*>(plan);
  const LaunchShape& L = P->shape[MT];
  *mode = !L.ready ? -1
          : L.mode == 1 ? 1
          : L.gridb     ? 7
          : L.cones     ? (L.tc ? 4 : 3)
          : L.pairs     ? (L.tc ? 6 : 5)
                        : (L.tc ? 2 : 0);
  *item_bytes = L.item_bytes;
  *stages = L.stages;
  *pub = L.pub;
  *slack = L.slack;
  *tuned_ms = L.tuned_ms;
  *candidates = L.candidates;
}

}  // namespace hb
