// leaf_tc.cu - the leaf outputs of the mixed apply on the 5th-generation
// tensor cores (tcgen05.mma, accumulators in tensor memory), Sec. 4.2 HODBF:
// for every leaf t of the cluster tree,
//     y(t) = D_t x(t) + sum over HODBF levels l of K^L_l(t) xhat_l(t)
// (forward; the adjoint sums D_t^H x(t) and V^0^H xhat), one accumulation
// chain of up to 64 outputs over all its terms.
//
// Complex -> real, planar.  A = the factor rows interleaved by part: row
// m = 2 o + p holds part p (0 = Re, 1 = Im) of output o (M = 128 rows = 64
// outputs), K = 16 inputs per MMA.  B = the input vector, N = 64 rows per 16
// right-hand sides: row n = 16 c + rho holds, for c = 2 q + s, part q of the
// split half s (0 = hi, 1 = lo) of right-hand side rho.  Then
//     D[(o,p)][(q,s,rho)] = sum_k part_p(F[o][k]) part_q(X_s[k][rho])
// and with F = F_hi + F_lo (two MMAs per 16 inputs, both accumulating)
//     Re Y[o][rho] = sum_s D[(o,Re)][(Re,s,rho)] - D[(o,Im)][(Im,s,rho)]
//     Im Y[o][rho] = sum_s D[(o,Re)][(Im,s,rho)] + D[(o,Im)][(Re,s,rho)];
// the Re and Im rows of an output sit in adjacent TMEM lanes, so the
// epilogue combines them with one shuffle.  All four products hi x hi,
// hi x lo, lo x hi, lo x lo are taken, accumulated in FP32.
//
// Operand layouts (K-major, no swizzle; a core matrix = 8 rows x 8
// elements, 128 contiguous bytes, row r at 16 r):
//  * factor k-group (8 inputs) = 4 KB: hi then lo, each 16 core matrices
//    (row group g at 128 g) - so LBO (next k-group) = 4096, SBO = 128;
//  * input row tile (8 inputs) = MT KB: 8 MT core matrices (row group at
//    128 g) - LBO = 1024 MT, SBO = 128.
//    The chains writing the skeleton vectors that only the leaf outputs
//    read store them in this layout (store_tiles_tc), and the gather writes
//    a copy of x in it.
// A term with an odd number of k-groups ends with an MMA whose second
// k-group is a zero block in shared memory (its LBO points there).
//
// Roles (one CTA of 6 warps per SM): warp 0 lane 0 streams the items
// (factor run + input run, 1D bulk copies) through a ring of stages; warp 1
// lane 0 issues the MMAs (two accumulator buffers in TMEM, 2 x 64 MT
// columns) and commits each stage back to the producer and each finished
// chain to the epilogue; warps 2-5 read the accumulators (each its quarter
// of the TMEM lanes), combine parts and halves, and store FP64 outputs in
// natural order.  Every wait is bounded; a wait that runs out sets the
// error word and the CTA winds down (waiting, bounded, for its copies and
// products in flight before it frees its tensor memory).
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <queue>
#include <vector>

#include "async_copy.cuh"
#include "hb_internal.cuh"

namespace hb {

#ifndef HB_TC_MAX_STAGES
#define HB_TC_MAX_STAGES 10
#endif
#ifndef HB_TC_ITEM_KG
#define HB_TC_ITEM_KG 4
#endif
constexpr int TC_WARPS = 6;
constexpr int TC_MAX_STAGES = HB_TC_MAX_STAGES;
constexpr int TC_FKG = 4096;             // bytes of one factor k-group (hi + lo, 128 rows x 8 inputs each)
constexpr int TC_ITEM_KG = HB_TC_ITEM_KG;   // k-groups per item (at most)
constexpr int TC_ZERO = 2048;    // zero block for odd k-group tails

struct TcItem {
  long long f_unit;      // first factor k-group (4 KB units of the tc arena)
  long long x_tile;      // first input row tile
  short nkg;             // k-groups (8 inputs each)
  unsigned char x_buf;   // 0: x (operand-layout copy), 2: xh
  unsigned char flags;   // 1: first item of its chain, 2: last
  int chain;             // index of its chain (global)
  long long pad;         // 32 bytes: records load as two 16-byte words
};
static_assert(sizeof(TcItem) == 32 && alignof(TcItem) == 8, "item layout");

struct TcOut {
  long long y_tile;      // first padded row tile of the outputs
  int nout;              // outputs (<= 64)
  int pad;
};

struct TcArgs {
  const TcItem* items;
  const long long* ioff;   // items of CTA b: [ioff[b], ioff[b + 1])
  const TcOut* chains;
  const long long* coff;   // chains of CTA b: [coff[b], coff[b + 1])
  const uint4* F;
  const uint4* x;
  const uint4* xh;
  double2* u;
  const long long* pperm;
  long long Nv;
  int R;
  int stages;
  int stage_bytes;
  long long budget;
  int* err;
};

// shared-memory matrix descriptor: start, leading byte offset (next core
// matrix along K), stride byte offset (next 8-row group), all >> 4;
// descriptor version 1; no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: D f32, A and B bf16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, bool acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d),
      "l"(a), "l"(b), "r"(idesc), "r"((int)acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// 32 lanes x 32 consecutive columns of tensor memory (one column per register)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// bounded wait that also gives up when another role has aborted
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, long long deadline, volatile int* abort_flag) {
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() > deadline) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

template <int MT>
__global__ void __launch_bounds__(TC_WARPS * 32, 1) bf_leaf_tc_kernel(TcArgs a) {
  constexpr int N = 64 * MT;          // accumulator columns of one buffer
  constexpr int XKG = 1024 * MT;      // bytes of one input row tile
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t full[TC_MAX_STAGES], empty[TC_MAX_STAGES], accf[2], acce[2], done;
  __shared__ __align__(16) TcItem slot[TC_MAX_STAGES];   // the record of the item in each stage
  __shared__ __align__(16) TcItem win[32];               // the producer's record window
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ long long issued, consumed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nst = a.stages;
  unsigned char* zero = smem + (size_t)nst * a.stage_bytes;
  for (int i = threadIdx.x; i < TC_ZERO / 16; i += blockDim.x) reinterpret_cast<uint4*>(zero)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 4);
    }
    mbar_init(&done, 1);
    abort_flag = 0;
    issued = consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(2 * N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the zero block, for the tensor cores
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  volatile int* abf = &abort_flag;
  const long long i0 = a.ioff[blockIdx.x], i1 = a.ioff[blockIdx.x + 1];
  const long long c0 = a.coff[blockIdx.x], c1 = a.coff[blockIdx.x + 1];
  const long long deadline = clock64() + a.budget;

  if (warp == 0) {
    // records: lane j holds record 32 w + j of the next window in registers;
    // a window moves to shared memory when its first item is issued
    const long long n = i1 - i0;
    const uint64_t pol_f = policy_evict_first(), pol_v = policy_evict_last();
    auto load_rec = [&](long long w, int4& r0, int4& r1) {
      const long long q = 32 * w + lane;
      if (q < n) {
        const int4* src = reinterpret_cast<const int4*>(a.items + i0 + q);   // 32-byte records
        r0 = src[0];
        r1 = src[1];
      }
    };
    int4 r0 = make_int4(0, 0, 0, 0), r1 = r0;
    load_rec(0, r0, r1);
    auto x_src = [&](const TcItem& it) { return (it.x_buf == 0 ? a.x : a.xh) + it.x_tile * (XKG / 16); };
    bool waited = false;
    for (long long k = 0; k < n; ++k) {
      const int s = (int)(k % nst);
      if ((k & 31) == 0) {
        int4* dst = reinterpret_cast<int4*>(&win[lane]);
        dst[0] = r0;
        dst[1] = r1;
        __syncwarp();
        load_rec((k >> 5) + 1, r0, r1);
      }
      bool stop = false;
      if (lane == 0) {
        if (k == nst && !waited) {
          // the first stages' factor runs went out before the previous
          // depth finished; their input runs follow once it has
          asm volatile("griddepcontrol.wait;" ::: "memory");
          asm volatile("fence.proxy.async.global;" ::: "memory");
          waited = true;
          for (int t = 0; t < nst; ++t)
            tma_load_1d(smem + (size_t)t * a.stage_bytes + (uint32_t)slot[t].nkg * TC_FKG, x_src(slot[t]),
                        (uint32_t)slot[t].nkg * XKG, &full[t], pol_v);
        }
        if (k >= nst && !tc_wait(&empty[s], (uint32_t)(((k / nst) - 1) & 1), deadline, abf)) {
          stop = true;
        } else {
          const TcItem it = win[k & 31];
          slot[s] = it;
          unsigned char* st = smem + (size_t)s * a.stage_bytes;
          const uint32_t fb = (uint32_t)it.nkg * TC_FKG, xb = (uint32_t)it.nkg * XKG;
          mbar_expect_tx(&full[s], fb + xb);
          tma_load_1d(st, a.F + it.f_unit * (TC_FKG / 16), fb, &full[s], pol_f);
          if (k >= nst) tma_load_1d(st + fb, x_src(it), xb, &full[s], pol_v);
          issued = k + 1;
        }
      }
      if (__shfl_sync(0xffffffffu, (int)stop, 0)) break;
    }
    if (lane == 0 && !waited) {
      // fewer items than stages: their input runs
      asm volatile("griddepcontrol.wait;" ::: "memory");
      asm volatile("fence.proxy.async.global;" ::: "memory");
      for (long long t = 0; t < issued; ++t)
        tma_load_1d(smem + (size_t)t * a.stage_bytes + (uint32_t)slot[t].nkg * TC_FKG, x_src(slot[t]),
                    (uint32_t)slot[t].nkg * XKG, &full[t], pol_v);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc_idesc(128, N);
      const uint32_t zaddr = smem_u32(zero);
      for (long long q = i0; q < i1; ++q) {
        const long long k = q - i0;
        const int s = (int)(k % nst);
        if (!tc_wait(&full[s], (uint32_t)((k / nst) & 1), deadline, abf)) break;
        const TcItem it = slot[s];
        const long long j = it.chain - c0;   // chain index within this CTA
        const int b = (int)(j & 1);
        if ((it.flags & 1) && j >= 2 && !tc_wait(&acce[b], (uint32_t)(((j / 2) - 1) & 1), deadline, abf)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t fs = smem_u32(smem + (size_t)s * a.stage_bytes);
        const uint32_t xs = fs + (uint32_t)it.nkg * TC_FKG;
        const uint32_t dt = tmem + (uint32_t)(b * N);
        for (int kk = 0; kk < it.nkg; kk += 2) {
          const uint32_t fa = fs + (uint32_t)kk * TC_FKG, xa = xs + (uint32_t)kk * XKG;
          const bool pair = kk + 1 < it.nkg;
          const uint32_t lhi = pair ? (uint32_t)TC_FKG : zaddr - fa;
          const uint32_t llo = pair ? (uint32_t)TC_FKG : zaddr - (fa + 2048);
          const uint32_t lx = pair ? (uint32_t)XKG : zaddr - xa;
          const uint64_t bd = tc_desc(xa, lx, 128);
          tc_mma(dt, tc_desc(fa, lhi, 128), bd, idesc, !((it.flags & 1) && kk == 0));
          tc_mma(dt, tc_desc(fa + 2048, llo, 128), bd, idesc, true);
        }
        tc_commit(&empty[s]);                 // the stage is free once these products are done
        if (it.flags & 2) tc_commit(&accf[b]);   // the chain's accumulator is complete
        consumed = k + 1;
      }
      tc_commit(&done);
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = rows m = 2 o + p
    const int q4 = warp & 3;
    const int m = 32 * q4 + lane, o = m >> 1, p = m & 1;
    // the output row of the next chain is looked up while this one computes
    auto nat_of = [&](long long cc) {
      const TcOut ch = a.chains[cc];
      return o < ch.nout ? a.pperm[8 * ch.y_tile + o] : -1LL;
    };
    long long nat_next = c0 < c1 ? nat_of(c0) : -1;
    for (long long cc = c0; cc < c1; ++cc) {
      const long long j = cc - c0;
      const int b = (int)(j & 1);
      const long long nat = nat_next;
      if (cc + 1 < c1) nat_next = nat_of(cc + 1);
      const bool ok = tc_wait(&accf[b], (uint32_t)((j / 2) & 1), deadline, abf);
      if (!__all_sync(0xffffffffu, ok)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      double* ud = reinterpret_cast<double*>(a.u);
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        uint32_t v[2][32];
        const uint32_t ta = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * N + 64 * mt);
        tmem_ld32(ta, v[0]);
        tmem_ld32(ta + 32, v[1]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (mt == MT - 1) {
          // the buffer may take the next chain's products
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&acce[b]);
        }
#pragma unroll
        for (int rl = 0; rl < 16; ++rl) {
          // columns 16 c + rl, c = 2 q + s: (Re, hi), (Re, lo), (Im, hi), (Im, lo)
          const float are = __uint_as_float(v[0][rl]) + __uint_as_float(v[0][16 + rl]);
          const float aim = __uint_as_float(v[1][rl]) + __uint_as_float(v[1][16 + rl]);
          const float recv = __shfl_xor_sync(0xffffffffu, aim, 1);
          const float out = p ? recv + are : are - recv;
          const int rhs = 16 * mt + rl;
          if (nat >= 0 && rhs < a.R) ud[2 * ((size_t)rhs * a.Nv + nat) + p] = (double)out;
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && abort_flag) {
    *reinterpret_cast<volatile int*>(a.err) = 1;
    // copies issued but not consumed: let them land before the CTA exits
    const long long drain = a.budget > (1LL << 31) ? a.budget : (1LL << 31);
    for (long long k = consumed; k < issued; ++k)
      mbar_wait_until(&full[k % nst], (uint32_t)((k / nst) & 1), clock64() + drain);
  }
  if (warp == 1) {
    // every product issued has completed before the tensor memory is freed
    const long long drain = a.budget > (1LL << 31) ? a.budget : (1LL << 31);
    if (lane == 0) mbar_wait_until(&done, 0u, clock64() + drain);
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * N) : "memory");
  }
}

// ------------------------------------------------------ operand layouts ----
// Factor block -> tc arena: k-group kg of the block (inputs 8 kg ..) is 4 KB
// at unit0 + kg: hi (2 KB) then lo; element (row m = 2 o + p, input k) at
// (m / 8) 128 + (m % 8) 16 + (k % 8) 2 bytes.  Outputs o0 .. o0 + nout of the
// block; rows past them and inputs past k are zero.
__global__ void tc_convert_kernel(const double2* __restrict__ F, const TcBlock* __restrict__ blocks,
                                  uint16_t* __restrict__ out) {
  const TcBlock B = blocks[blockIdx.x];
  const int nkg = (B.k + 7) / 8;
  for (int idx = threadIdx.x; idx < nkg * 1024; idx += blockDim.x) {
    const int kg = idx >> 10, e = idx & 1023, m = e >> 3, kk = e & 7;
    const int o = m >> 1, p = m & 1, k = 8 * kg + kk;
    double v = 0.0;
    if (o < B.nout && k < B.k) {
      const int n = B.o0 + o;
      if (B.conj) {
        const double2 f = F[B.src_off + k + (long long)n * B.ld];
        v = p ? -f.y : f.x;
      } else {
        const double2 f = F[B.src_off + n + (long long)k * B.ld];
        v = p ? f.y : f.x;
      }
    }
    const float hf = (float)v;
    const uint32_t hb = bf16x2(hf, 0.f) & 0xffffu;
    const float lo = hf - __uint_as_float(hb << 16);
    const uint32_t lb = bf16x2(lo, 0.f) & 0xffffu;
    const size_t base = (size_t)(B.unit0 + kg) * (TC_FKG / 2) + (size_t)(m >> 3) * 64 + (m & 7) * 8 + kk;
    out[base] = (uint16_t)hb;
    out[base + 1024] = (uint16_t)lb;
  }
}

void tc_convert(const double2* F64, const std::vector<TcBlock>& blocks, void* out, cudaStream_t st) {
  if (blocks.empty()) return;
  TcBlock* d = upload(blocks, st);
  for (size_t b0 = 0; b0 < blocks.size(); b0 += (1u << 30)) {
    const unsigned n = (unsigned)std::min<size_t>(blocks.size() - b0, 1u << 30);
    tc_convert_kernel<<<n, 256, 0, st>>>(F64, d + b0, static_cast<uint16_t*>(out));
    HB_CHECK_LAUNCH();
  }
  HB_CUDA(cudaStreamSynchronize(st));
  dev_free(d);
}

// ---------------------------------------------------------------- plan ----
struct TcPlan {
  std::vector<TcChainHost> chains;
  int grid[3] = {0, 0, 0};
  int stage_bytes[3] = {0, 0, 0};
  TcItem* d_items[3] = {nullptr, nullptr, nullptr};
  long long* d_ioff[3] = {nullptr, nullptr, nullptr};
  TcOut* d_chains[3] = {nullptr, nullptr, nullptr};
  long long* d_coff[3] = {nullptr, nullptr, nullptr};
};

void* tc_plan_build(std::vector<TcChainHost>&& chains) {
  TcPlan* P = new TcPlan();
  P->chains = std::move(chains);
  return P;
}

static void tc_free_lists(TcPlan* P, int MT) {
  dev_free(P->d_items[MT]);
  dev_free(P->d_ioff[MT]);
  dev_free(P->d_chains[MT]);
  dev_free(P->d_coff[MT]);
  P->d_items[MT] = nullptr;
  P->d_ioff[MT] = nullptr;
  P->d_chains[MT] = nullptr;
  P->d_coff[MT] = nullptr;
  P->grid[MT] = 0;
}

void tc_plan_free(void* plan) {
  TcPlan* P = static_cast<TcPlan*>(plan);
  if (!P) return;
  for (int mt = 1; mt <= 2; ++mt) tc_free_lists(P, mt);
  delete P;
}

// Deal the chains over the CTAs (largest first to the least-loaded CTA) and
// cut each chain's terms into items of at most TC_ITEM_KG k-groups (runs of
// an even count, so only a term's last MMA can have an odd tail).
static void tc_build_lists(TcPlan* P, int MT, int grid) {
  tc_free_lists(P, MT);
  const size_t nc = P->chains.size();
  std::vector<long long> cost(nc);
  for (size_t c = 0; c < nc; ++c) {
    long long w = 0;
    for (const TcTerm& t : P->chains[c].terms) w += t.nkg + 2;
    cost[c] = w;
  }
  std::vector<size_t> order(nc);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
  using Load = std::pair<long long, int>;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> pq;
  for (int b = 0; b < grid; ++b) pq.push({0, b});
  std::vector<std::vector<size_t>> per((size_t)grid);
  for (size_t c : order) {
    Load l = pq.top();
    pq.pop();
    per[(size_t)l.second].push_back(c);
    l.first += cost[c];
    pq.push(l);
  }
  std::vector<TcItem> items;
  std::vector<TcOut> outs;
  std::vector<long long> ioff, coff;
  int stage = 0;
  for (int b = 0; b < grid; ++b) {
    ioff.push_back((long long)items.size());
    coff.push_back((long long)outs.size());
    for (size_t c : per[(size_t)b]) {
      const TcChainHost& ch = P->chains[c];
      const int gidx = (int)outs.size();
      outs.push_back(TcOut{ch.y_tile, ch.nout, 0});
      const size_t first = items.size();
      for (const TcTerm& t : ch.terms)
        for (int k0 = 0; k0 < t.nkg; k0 += TC_ITEM_KG) {
          TcItem it{};
          it.f_unit = t.unit0 + k0;
          it.x_tile = t.x_tile + k0;
          it.nkg = (short)std::min(TC_ITEM_KG, t.nkg - k0);
          it.x_buf = (unsigned char)t.x_buf;
          it.chain = gidx;
          items.push_back(it);
          stage = std::max(stage, (int)it.nkg * (TC_FKG + 1024 * MT));
        }
      if (items.size() == first) throw Error{HB_ERR_STATE, "a leaf-output chain without terms"};
      items[first].flags |= 1;
      items.back().flags |= 2;
    }
  }
  ioff.push_back((long long)items.size());
  coff.push_back((long long)outs.size());
  P->d_items[MT] = upload(items);
  P->d_ioff[MT] = upload(ioff);
  P->d_chains[MT] = upload(outs);
  P->d_coff[MT] = upload(coff);
  HB_CUDA(cudaDeviceSynchronize());
  P->grid[MT] = grid;
  P->stage_bytes[MT] = stage;
}

template <int MT>
static void tc_launch_mt(TcPlan* P, const uint4* F, const uint4* x, const uint4* xh, double2* u,
                         const long long* pperm, long long Nv, int R, int* err, long long budget, cudaStream_t st) {
  auto k = bf_leaf_tc_kernel<MT>;
  if (!P->grid[MT]) {
    int dev = 0, nsm = 0;
    HB_CUDA(cudaGetDevice(&dev));
    HB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    tc_build_lists(P, MT, nsm);
  }
  int dev = 0, optin = 0;
  HB_CUDA(cudaGetDevice(&dev));
  HB_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa{};
  HB_CUDA(cudaFuncGetAttributes(&fa, k));
  const int avail = optin - (int)fa.sharedSizeBytes - TC_ZERO - 1024;
  const int stages = std::min(TC_MAX_STAGES, avail / std::max(1, P->stage_bytes[MT]));
  if (stages < 2) throw Error{HB_ERR_UNSUPPORTED, "tensor-core leaf stages do not fit in shared memory"};
  const size_t smem = (size_t)stages * P->stage_bytes[MT] + TC_ZERO;
  HB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  TcArgs args{P->d_items[MT], P->d_ioff[MT], P->d_chains[MT], P->d_coff[MT], F, x, xh, u, pperm, Nv, R,
              stages, P->stage_bytes[MT], budget, err};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(P->grid[MT]);
  cfg.blockDim = dim3(TC_WARPS * 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  HB_CUDA(cudaLaunchKernelEx(&cfg, k, args));
}

void tc_leaf_launch(void* plan, int MT, const void* F, const uint4* x, const uint4* xh, double2* u,
                    const long long* pperm, long long Nv, int R, int* err, long long budget, cudaStream_t st) {
  TcPlan* P = static_cast<TcPlan*>(plan);
  if (!P || P->chains.empty()) return;
  if (MT == 1)
    tc_launch_mt<1>(P, static_cast<const uint4*>(F), x, xh, u, pperm, Nv, R, err, budget, st);
  else if (MT == 2)
    tc_launch_mt<2>(P, static_cast<const uint4*>(F), x, xh, u, pperm, Nv, R, err, budget, st);
  else
    throw Error{HB_ERR_UNSUPPORTED, "the tensor-core leaf kernel takes 1 or 2 m-tiles"};
}

}  // namespace hb
