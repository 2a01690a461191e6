// bf_mma.cu - mixed-precision butterfly step kernel on the tensor cores
// (Sec. 4.2.1, Eq. butterfly_mat: every factor level is a batch of small
// dense complex products Y = op(F) X).
//
// Factors and vectors are FP32 complex in HBM.  Each product runs as real
// BF16 MMAs (mma.sync m16n8k16, FP32 accumulate) on a split of both
// operands, a = a_hi + a_lo with a_hi = bf16(a), a_lo = bf16(a - a_hi):
//     a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi          (split BF16 x 3)
// which keeps ~16 significant bits per product.
//
// Complex -> real layout (k' = 2k + c interleaves real/imaginary parts):
//     D_r[m][n] = sum_k' A_r[m][k'] B[k'][n],   D_i[m][n] = sum_k' A_i[m][k'] B[k'][n]
//     A_r[m][(2k,2k+1)] = (Re X[k][m], -Im X[k][m]),  A_i[m][(2k,2k+1)] = (Im X[k][m], Re X[k][m])
//     B[(2k,2k+1)][n]   = (Re F[n][k], Im F[n][k])   (or conj(F[k][n]) for op = ^H)
// so M = right-hand sides (16 per m-tile), N = output rows (8 per n-tile),
// K = 8 complex inputs per k16 step; Y[n][m] = D_r[m][n] + i D_i[m][n].
// Each factor entry is loaded from global memory exactly once, straight
// into the B fragment registers (8-byte loads, 64-byte runs per fragment
// row); X fragments are reused across the warp's n-tiles.
//
// Work unit = one warp: (task, first output row).  A unit covers NT n-tiles
// (8*NT output rows) and all right-hand sides.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "hb_internal.cuh"

namespace hb {

constexpr int MMA_NT = 4;        // n-tiles per warp unit

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

struct Unit {
  int task;
  int nb;     // first output row
};

// MT m-tiles (16 right-hand sides each) per pass; larger R loops over passes.
template <int MT>
__global__ void __launch_bounds__(256) mma_step_kernel(const Unit* __restrict__ units, int nunits,
                                                       const Task* __restrict__ tasks,
                                                       const float2* __restrict__ F, float2* __restrict__ x,
                                                       float2* __restrict__ y, float2* __restrict__ xh,
                                                       int R) {
  const int warp_global = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (warp_global >= nunits) return;
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const Unit u = units[warp_global];
  const Task tk = tasks[u.task];
  auto buf = [&](int id) { return id == 0 ? x : (id == 1 ? y : xh); };
  const int mtiles = (R + 15) >> 4;

  for (int m0 = 0; m0 < mtiles; m0 += MT) {
    const int mt_here = min(MT, mtiles - m0);
    float acc_r[MT][MMA_NT][4];
    float acc_i[MT][MMA_NT][4];
#pragma unroll
    for (int a = 0; a < MT; ++a)
#pragma unroll
      for (int j = 0; j < MMA_NT; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc_r[a][j][e] = acc_i[a][j][e] = 0.f;

    for (int term = 0; term < tk.nterm; ++term) {
      const float2* f = F + (term ? tk.f_off[1] : tk.f_off[0]);
      const float2* xin = buf(tk.x_buf) + (size_t)(term ? tk.x_off[1] : tk.x_off[0]) * R;
      const int rin = term ? tk.r_in[1] : tk.r_in[0];
      for (int kb = 0; kb < rin; kb += 8) {
        const int k0 = kb + t, k1 = kb + t + 4;
        // B fragments for the warp's n-tiles
        uint32_t bh0[MMA_NT], bl0[MMA_NT], bh1[MMA_NT], bl1[MMA_NT];
#pragma unroll
        for (int j = 0; j < MMA_NT; ++j) {
          const int n = u.nb + 8 * j + g;
          float2 v0 = make_float2(0.f, 0.f), v1 = v0;
          if (n < tk.r_out) {
            if (!tk.conj_t) {
              if (k0 < rin) v0 = f[(size_t)k0 * tk.r_out + n];
              if (k1 < rin) v1 = f[(size_t)k1 * tk.r_out + n];
            } else {
              if (k0 < rin) { v0 = f[(size_t)n * rin + k0]; v0.y = -v0.y; }
              if (k1 < rin) { v1 = f[(size_t)n * rin + k1]; v1.y = -v1.y; }
            }
          }
          split2(v0.x, v0.y, bh0[j], bl0[j]);
          split2(v1.x, v1.y, bh1[j], bl1[j]);
        }
#pragma unroll
        for (int a = 0; a < MT; ++a) {
          if (a >= mt_here) break;
          const int mA = (m0 + a) * 16 + g, mB = mA + 8;
          float2 x00 = make_float2(0.f, 0.f), x01 = x00, x10 = x00, x11 = x00;   // [k][m]
          if (k0 < rin) {
            if (mA < R) x00 = xin[(size_t)k0 * R + mA];
            if (mB < R) x01 = xin[(size_t)k0 * R + mB];
          }
          if (k1 < rin) {
            if (mA < R) x10 = xin[(size_t)k1 * R + mA];
            if (mB < R) x11 = xin[(size_t)k1 * R + mB];
          }
          uint32_t arh[4], arl[4], aih[4], ail[4];
          // a0: row g, k' pair (2t,2t+1) -> complex k0; a1: row g+8; a2: k1 row g; a3: k1 row g+8
          split2(x00.x, -x00.y, arh[0], arl[0]);
          split2(x01.x, -x01.y, arh[1], arl[1]);
          split2(x10.x, -x10.y, arh[2], arl[2]);
          split2(x11.x, -x11.y, arh[3], arl[3]);
          split2(x00.y, x00.x, aih[0], ail[0]);
          split2(x01.y, x01.x, aih[1], ail[1]);
          split2(x10.y, x10.x, aih[2], ail[2]);
          split2(x11.y, x11.x, aih[3], ail[3]);
#pragma unroll
          for (int j = 0; j < MMA_NT; ++j) {
            if (u.nb + 8 * j >= tk.r_out) break;
            mma16816(acc_r[a][j], arh, bh0[j], bh1[j]);
            mma16816(acc_r[a][j], arh, bl0[j], bl1[j]);
            mma16816(acc_r[a][j], arl, bh0[j], bh1[j]);
            mma16816(acc_i[a][j], aih, bh0[j], bh1[j]);
            mma16816(acc_i[a][j], aih, bl0[j], bl1[j]);
            mma16816(acc_i[a][j], ail, bh0[j], bh1[j]);
          }
        }
      }
    }
    // epilogue: Y[n][m] = (D_r[m][n], D_i[m][n])
    float2* out = buf(tk.y_buf) + (size_t)tk.y_off * R;
#pragma unroll
    for (int a = 0; a < MT; ++a) {
      if (a >= mt_here) break;
#pragma unroll
      for (int j = 0; j < MMA_NT; ++j) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int m = (m0 + a) * 16 + g + ((e & 2) ? 8 : 0);
          const int n = u.nb + 8 * j + 2 * t + (e & 1);
          if (m < R && n < tk.r_out) {
            float2* o = out + (size_t)n * R + m;
            float2 v = make_float2(acc_r[a][j][e], acc_i[a][j][e]);
            if (tk.accumulate) {
              const float2 p = *o;
              v.x += p.x;
              v.y += p.y;
            }
            *o = v;
          }
        }
      }
    }
  }
}

static void make_units(const std::vector<Task>& tasks, int begin, int end, std::vector<Unit>& units) {
  for (int i = begin; i < end; ++i)
    for (int nb = 0; nb < tasks[i].r_out; nb += 8 * MMA_NT) units.push_back(Unit{i, nb});
}

void mma_plan_build(hb_ctx* c, int dir, std::vector<int>& step_units, void** d_units_out) {
  std::vector<Unit> units;
  step_units.clear();
  const std::vector<int>& sb = c->step_begin[dir];
  for (size_t s = 0; s + 1 < sb.size(); ++s) {
    step_units.push_back((int)units.size());
    make_units(c->tasks_h[dir], sb[s], sb[s + 1], units);
  }
  step_units.push_back((int)units.size());
  *d_units_out = upload(units);
}

void mma_step_launch(const void* d_units, int u0, int u1, const Task* d_tasks, const float2* F, float2* x,
                     float2* y, float2* xh, int R, cudaStream_t st) {
  const int n = u1 - u0;
  if (n <= 0) return;
  const int warps_per_cta = 8;
  const int grid = (n + warps_per_cta - 1) / warps_per_cta;
  const Unit* un = static_cast<const Unit*>(d_units) + u0;
  if (R <= 16) mma_step_kernel<1><<<grid, 32 * warps_per_cta, 0, st>>>(un, n, d_tasks, F, x, y, xh, R);
  else if (R <= 32) mma_step_kernel<2><<<grid, 32 * warps_per_cta, 0, st>>>(un, n, d_tasks, F, x, y, xh, R);
  else mma_step_kernel<4><<<grid, 32 * warps_per_cta, 0, st>>>(un, n, d_tasks, F, x, y, xh, R);
  HB_CHECK_LAUNCH();
}

}  // namespace hb
