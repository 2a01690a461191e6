// inclusion.cu - scattering by a curve inclusion on the device (Sec. 3.2).
//
// The curve C is cut into N_s straight segments with centres r^s_i, lengths
// w_i and refractive index n_i at the centres.  Eq. sie (the total field
// vanishes on C) enforced at the centres gives the surface system
// K^{s2s} P = K^{v2s} I (Eq. m_sie), and the total field at the cells is
//     U = (K^{v2v} + K^{s2v} (K^{s2s})^{-1} K^{v2s}) I        (Eq. m_v2v_inclu)
// with
//     K^{s2s}_ij = -g(r^s_i, r^s_j) w_j   (i != j)               (Eq. s2s)
//     K^{s2s}_ii = -(i w_i / 4)(1 + (2i/pi)(ln(gamma w n_i w_i / 4) - 1)),
//                  gamma = e^{gamma_E}: minus the integral over the segment
//                  of the small-argument form of (i/4) H0(w n_i |t|)
//     K^{v2s}_ij = g(r^s_i, r_j),   K^{s2v}_ij = g(r_i, r^s_j) w_j   (Eq. m_v2s, Eq. m_s2v)
// and g = v0 f0 + v1 f1 (Eq. babich) with tau^2, v0, v1 interpolated at the
// points from the tables (Eq. chebinterp), as for K^{v2v}.
//
// K^{v2s} and K^{s2v} are stored dense (2 N_s N_v complex values) or, after
// hb_curve_compress, as butterflies (curve_bf.cu); K^{s2s} is factored by
// LU with partial pivoting once per curve and inverted from the factors, so
// an apply is three products (dense, or butterfly - dense - butterfly) on
// top of the K^{v2v} apply (dense or compressed).  FP64 throughout.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "bessel.cuh"
#include "hb_internal.cuh"

namespace hb {

namespace {

constexpr int CMAX_NI = 16;                              // n_I supported (hb_create's limit)
constexpr double GAMMA_EXP = 1.78107241799019798524;     // e^{Euler's constant}
constexpr long long MAX_SEGMENTS = 16384;

struct PointTables {
  const double* nodes;   // nodes_x (n_I) then nodes_y (n_I)
  const double* tab;     // 3 x N_I x N_I forward tables, row = observation node
  int nI, NI;
  double omega;
};

// Lagrange basis l_k(x) of the n_I nodes in barycentric form (weights bw);
// at a node, the basis indicator.
__device__ __forceinline__ void basis_at(const double* nodes, const double* bw, int nI, double x, double* L) {
  int hit = -1;
  for (int k = 0; k < nI; ++k)
    if (x == nodes[k]) hit = k;
  if (hit >= 0) {
    for (int k = 0; k < nI; ++k) L[k] = (k == hit) ? 1.0 : 0.0;
    return;
  }
  double den = 0.0;
  for (int k = 0; k < nI; ++k) {
    L[k] = bw[k] / (x - nodes[k]);
    den += L[k];
  }
  for (int k = 0; k < nI; ++k) L[k] /= den;
}

// out[a + b*ldo] = sgn * w_b * g(obs_a, src_b) for a < m (w_b = wsrc[b], or 1
// when wsrc is null).  With diag (the observation points are the source
// points, m = n) the entry a == b is the K^{s2s} diagonal of segment a
// (lengths wsrc, index nseg).  One CTA per source point b: first
// G[q][i] = sum_j F_q[i][j] T_j(src_b) (T_j = l_{j1}(x) l_{j2}(z),
// j = j2 n_I + j1) in shared memory, then the threads take the observation
// points, f_q = sum_i T_i(obs_a) G[q][i].
__global__ void __launch_bounds__(256) green_columns_kernel(PointTables P, const double2* __restrict__ obs, long long m,
                                                            const double2* __restrict__ src,
                                                            const double* __restrict__ wsrc,
                                                            const double* __restrict__ nseg, double sgn, int diag,
                                                            double2* __restrict__ out, long long ldo) {
  __shared__ double G[3 * CMAX_NI * CMAX_NI];
  __shared__ double bw[2][CMAX_NI];
  __shared__ double Ls[2][CMAX_NI];
  const int nI = P.nI, NI = P.NI, t = threadIdx.x;
  const long long b = blockIdx.x;
  if (t < 2 * nI) {
    const int d = t / nI, k = t % nI;
    const double* nd = P.nodes + d * nI;
    double p = 1.0;
    for (int q = 0; q < nI; ++q)
      if (q != k) p *= (nd[k] - nd[q]);
    bw[d][k] = 1.0 / p;
  }
  __syncthreads();
  if (t < 2) {
    const double2 s = src[b];
    basis_at(P.nodes + t * nI, bw[t], nI, t == 0 ? s.x : s.y, Ls[t]);
  }
  __syncthreads();
  for (int idx = t; idx < 3 * NI; idx += blockDim.x) {
    const int q = idx / NI, i = idx % NI;
    const double* Fr = P.tab + ((size_t)q * NI + i) * NI;
    double acc = 0.0;
    for (int j2 = 0; j2 < nI; ++j2) {
      double a2 = 0.0;
      for (int j1 = 0; j1 < nI; ++j1) a2 = fma(Fr[j2 * nI + j1], Ls[0][j1], a2);
      acc = fma(Ls[1][j2], a2, acc);
    }
    G[idx] = acc;
  }
  __syncthreads();
  const double wb = wsrc ? wsrc[b] : 1.0;
  for (long long a = t; a < m; a += blockDim.x) {
    double2 val;
    if (diag && a == b) {
      const double w = wsrc[b];
      const double c = (2.0 / HB_PI) * (log(GAMMA_EXP * P.omega * nseg[b] * w / 4.0) - 1.0);
      val = make_double2(0.25 * w * c, -0.25 * w);   // -(i w/4)(1 + i c)
    } else {
      const double2 o = obs[a];
      double Lx[CMAX_NI], Lz[CMAX_NI];
      basis_at(P.nodes, bw[0], nI, o.x, Lx);
      basis_at(P.nodes + nI, bw[1], nI, o.y, Lz);
      double f[3];
      for (int q = 0; q < 3; ++q) {
        const double* Gq = G + q * NI;
        double acc = 0.0;
        for (int i2 = 0; i2 < nI; ++i2) {
          double a2 = 0.0;
          for (int i1 = 0; i1 < nI; ++i1) a2 = fma(Lx[i1], Gq[i2 * nI + i1], a2);
          acc = fma(Lz[i2], a2, acc);
        }
        f[q] = acc;
      }
      const double2 g = hb_green(f[0], f[1], f[2], P.omega);
      val = make_double2(sgn * wb * g.x, sgn * wb * g.y);
    }
    out[(size_t)b * ldo + a] = val;
  }
}

// Batched columns of curve-operator blocks: job q (one CTA) writes
// out[J.out_off + a] = J.w g(obs[J.obs0 + a], J.src) for a < J.m - the
// same evaluation as green_columns_kernel, for sampled blocks whose rows
// are gathered into obs.
__global__ void __launch_bounds__(256) green_jobs_kernel(PointTables P, const double2* __restrict__ obs,
                                                         const GreenCol* __restrict__ jobs,
                                                         double2* __restrict__ out) {
  __shared__ double G[3 * CMAX_NI * CMAX_NI];
  __shared__ double bw[2][CMAX_NI];
  __shared__ double Ls[2][CMAX_NI];
  const int nI = P.nI, NI = P.NI, t = threadIdx.x;
  const GreenCol J = jobs[blockIdx.x];
  if (t < 2 * nI) {
    const int d = t / nI, k = t % nI;
    const double* nd = P.nodes + d * nI;
    double p = 1.0;
    for (int q = 0; q < nI; ++q)
      if (q != k) p *= (nd[k] - nd[q]);
    bw[d][k] = 1.0 / p;
  }
  __syncthreads();
  if (t < 2) basis_at(P.nodes + t * nI, bw[t], nI, t == 0 ? J.src.x : J.src.y, Ls[t]);
  __syncthreads();
  for (int idx = t; idx < 3 * NI; idx += blockDim.x) {
    const int q = idx / NI, i = idx % NI;
    const double* Fr = P.tab + ((size_t)q * NI + i) * NI;
    double acc = 0.0;
    for (int j2 = 0; j2 < nI; ++j2) {
      double a2 = 0.0;
      for (int j1 = 0; j1 < nI; ++j1) a2 = fma(Fr[j2 * nI + j1], Ls[0][j1], a2);
      acc = fma(Ls[1][j2], a2, acc);
    }
    G[idx] = acc;
  }
  __syncthreads();
  for (int a = t; a < J.m; a += blockDim.x) {
    const double2 o = obs[J.obs0 + a];
    double Lx[CMAX_NI], Lz[CMAX_NI];
    basis_at(P.nodes, bw[0], nI, o.x, Lx);
    basis_at(P.nodes + nI, bw[1], nI, o.y, Lz);
    double f[3];
    for (int q = 0; q < 3; ++q) {
      const double* Gq = G + q * NI;
      double acc = 0.0;
      for (int i2 = 0; i2 < nI; ++i2) {
        double a2 = 0.0;
        for (int i1 = 0; i1 < nI; ++i1) a2 = fma(Lx[i1], Gq[i2 * nI + i1], a2);
        acc = fma(Lz[i2], a2, acc);
      }
      f[q] = acc;
    }
    const double2 g = hb_green(f[0], f[1], f[2], P.omega);
    out[J.out_off + a] = make_double2(J.w * g.x, J.w * g.y);
  }
}

__global__ void cell_points_kernel(int nx, long long Nv, double x0, double y0, double h, double2* __restrict__ pts) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < Nv; i += (long long)gridDim.x * blockDim.x) {
    const long long a = i % nx, b = i / nx;
    pts[i] = make_double2(x0 + (a + 0.5) * h, y0 + (b + 0.5) * h);
  }
}

// Step k of the LU factorisation with partial pivoting of the column-major
// n x n matrix A: pivot p = the row of the largest |A_ik|^2 over i >= k
// (lowest index on ties), rows k and p interchanged across all columns,
// multipliers A_ik /= A_kk for i > k.  One CTA of 256 threads.
__global__ void __launch_bounds__(256) lu_pivot_kernel(double2* __restrict__ A, int n, int k, int* __restrict__ piv,
                                                       int* __restrict__ singular) {
  __shared__ double bv[256];
  __shared__ int bi[256];
  const int t = threadIdx.x;
  double2* colk = A + (size_t)k * n;
  double best = -1.0;
  int at = n;
  for (int i = k + t; i < n; i += blockDim.x) {
    const double2 v = colk[i];
    const double m2 = v.x * v.x + v.y * v.y;
    if (m2 > best) {
      best = m2;
      at = i;
    }
  }
  bv[t] = best;
  bi[t] = at;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) {
      const double o = bv[t + s];
      const int oi = bi[t + s];
      if (o > bv[t] || (o == bv[t] && oi < bi[t])) {
        bv[t] = o;
        bi[t] = oi;
      }
    }
    __syncthreads();
  }
  int p = bi[0];
  const bool zero = !(bv[0] > 0.0) || p >= n;   // an all-zero (or NaN) column
  if (p >= n) p = k;
  if (t == 0) {
    piv[k] = p;
    if (zero) *singular = 1;
  }
  if (p != k)
    for (int j = t; j < n; j += blockDim.x) {
      double2* cj = A + (size_t)j * n;
      const double2 a = cj[k];
      cj[k] = cj[p];
      cj[p] = a;
    }
  __syncthreads();
  const double2 d = colk[k];
  const double dd = d.x * d.x + d.y * d.y;
  if (dd > 0.0) {
    const double ir = d.x / dd, ii = -d.y / dd;   // 1 / d
    for (int i = k + 1 + t; i < n; i += blockDim.x) {
      const double2 a = colk[i];
      colk[i] = make_double2(a.x * ir - a.y * ii, a.x * ii + a.y * ir);
    }
  }
}

// Trailing update of step k: A_ij -= A_ik A_kj for i, j > k (column
// j = k + 1 + blockIdx.y).
__global__ void lu_update_kernel(double2* __restrict__ A, int n, int k) {
  const int j = k + 1 + blockIdx.y;
  const double2* colk = A + (size_t)k * n;
  double2* colj = A + (size_t)j * n;
  const double2 akj = colj[k];
  for (int i = k + 1 + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double2 l = colk[i];
    double2 a = colj[i];
    a.x = fma(-l.x, akj.x, fma(l.y, akj.y, a.x));
    a.y = fma(-l.x, akj.y, fma(-l.y, akj.x, a.y));
    colj[i] = a;
  }
}

// y <- A^{-1} y with the factors of lu_pivot_kernel / lu_update_kernel: the
// row interchanges in order, then the unit lower and the upper triangular
// substitutions.  One CTA per column of Y (leading dimension ldy).
__global__ void __launch_bounds__(256) lu_solve_kernel(const double2* __restrict__ A, const int* __restrict__ piv,
                                                       int n, double2* __restrict__ Y, long long ldy) {
  double2* y = Y + (size_t)blockIdx.x * ldy;
  const int t = threadIdx.x;
  if (t == 0)
    for (int k = 0; k < n; ++k) {
      const int p = piv[k];
      if (p != k) {
        const double2 a = y[k];
        y[k] = y[p];
        y[p] = a;
      }
    }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const double2 yk = y[k];
    const double2* colk = A + (size_t)k * n;
    for (int i = k + 1 + t; i < n; i += blockDim.x) {
      const double2 l = colk[i];
      double2 v = y[i];
      v.x = fma(-l.x, yk.x, fma(l.y, yk.y, v.x));
      v.y = fma(-l.x, yk.y, fma(-l.y, yk.x, v.y));
      y[i] = v;
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const double2* colk = A + (size_t)k * n;
    if (t == 0) {
      const double2 d = colk[k], v = y[k];
      const double dd = d.x * d.x + d.y * d.y;
      y[k] = make_double2((v.x * d.x + v.y * d.y) / dd, (v.y * d.x - v.x * d.y) / dd);
    }
    __syncthreads();
    const double2 yk = y[k];
    for (int i = t; i < k; i += blockDim.x) {
      const double2 u = colk[i];
      double2 v = y[i];
      v.x = fma(-u.x, yk.x, fma(u.y, yk.y, v.x));
      v.y = fma(-u.x, yk.y, fma(-u.y, yk.x, v.y));
      y[i] = v;
    }
    __syncthreads();
  }
}

// A = the n x n identity (column-major)
__global__ void identity_kernel(double2* __restrict__ A, long long n) {
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n * n;
       idx += (long long)gridDim.x * blockDim.x)
    A[idx] = make_double2(idx % n == idx / n ? 1.0 : 0.0, 0.0);
}

// Y[:, r] (= or +=) alpha A X[:, r] for r < R; A column-major m x k, X with
// leading dimension ldx, Y with ldy.  One thread per output (row fastest).
__global__ void cgemm_kernel(const double2* __restrict__ A, long long m, long long k, const double2* __restrict__ X,
                             long long ldx, double2* __restrict__ Y, long long ldy, int R, double alpha,
                             int accumulate) {
  const long long total = m * R;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long i = idx % m;
    const int r = (int)(idx / m);
    const double2* x = X + (size_t)r * ldx;
    double re = 0.0, im = 0.0;
    for (long long j = 0; j < k; ++j) {
      const double2 a = A[(size_t)j * m + i];
      const double2 v = x[j];
      re = fma(a.x, v.x, fma(-a.y, v.y, re));
      im = fma(a.x, v.y, fma(a.y, v.x, im));
    }
    double2* y = Y + (size_t)r * ldy + i;
    re *= alpha;
    im *= alpha;
    if (accumulate) {
      re += y->x;
      im += y->y;
    }
    *y = make_double2(re, im);
  }
}

PointTables point_tables(const hb_ctx* c) {
  PointTables P;
  P.nodes = c->d_nodes;
  P.tab = c->d_tab;
  P.nI = c->nI;
  P.NI = c->NI;
  P.omega = c->omega;
  return P;
}

// The three surface operators into column-major outputs (any may be null).
void assemble(const hb_ctx* c, const double2* seg, const double* w, const double* nseg, long long ns,
              const double2* cells, double2* k_s2s, double2* k_v2s, double2* k_s2v, cudaStream_t st) {
  const PointTables P = point_tables(c);
  if (k_s2s) {
    green_columns_kernel<<<(unsigned)ns, 256, 0, st>>>(P, seg, ns, seg, w, nseg, -1.0, 1, k_s2s, ns);
    HB_CHECK_LAUNCH();
  }
  if (k_v2s) {
    green_columns_kernel<<<(unsigned)c->Nv, 256, 0, st>>>(P, seg, ns, cells, nullptr, nullptr, 1.0, 0, k_v2s, ns);
    HB_CHECK_LAUNCH();
  }
  if (k_s2v) {
    green_columns_kernel<<<(unsigned)ns, 256, 0, st>>>(P, cells, c->Nv, seg, w, nullptr, 1.0, 0, k_s2v, c->Nv);
    HB_CHECK_LAUNCH();
  }
}

}  // namespace

void green_jobs(const hb_ctx* c, const double2* d_obs, const GreenCol* d_jobs, long long njobs, double2* d_out,
                cudaStream_t st) {
  const PointTables P = point_tables(c);
  for (long long b0 = 0; b0 < njobs; b0 += (1LL << 30)) {
    const unsigned n = (unsigned)std::min<long long>(njobs - b0, 1LL << 30);
    green_jobs_kernel<<<n, 256, 0, st>>>(P, d_obs, d_jobs + b0, d_out);
    HB_CHECK_LAUNCH();
  }
}

void curve_free(hb_ctx* c) {
  for (void* p : {(void*)c->d_seg, (void*)c->d_segw, (void*)c->d_segn, (void*)c->d_cellpts, (void*)c->d_lu,
                  (void*)c->d_piv, (void*)c->d_kv2s, (void*)c->d_ks2v, (void*)c->d_cy, (void*)c->d_inv})
    dev_free(p);
  c->d_inv = nullptr;
  c->d_seg = nullptr;
  c->d_segw = c->d_segn = nullptr;
  c->d_cellpts = c->d_lu = c->d_kv2s = c->d_ks2v = c->d_cy = nullptr;
  c->d_piv = nullptr;
  c->ns = 0;
  c->cy_cap = 0;
  curve_bf_free(c);
}

void curve_set(hb_ctx* c, const double* centers, const double* lengths, const double* n_seg, long long ns) {
  if (!centers || !lengths || !n_seg) throw arg_error("null curve array");
  if (ns < 1 || ns > MAX_SEGMENTS) throw arg_error("segments %lld outside [1, %lld]", ns, MAX_SEGMENTS);
  for (long long i = 0; i < ns; ++i) {
    if (!std::isfinite(centers[2 * i]) || !std::isfinite(centers[2 * i + 1]))
      throw arg_error("segment %lld: centre not finite", i);
    if (!(lengths[i] > 0) || !std::isfinite(lengths[i])) throw arg_error("segment %lld: length must be positive", i);
    if (!(n_seg[i] > 0) || !std::isfinite(n_seg[i])) throw arg_error("segment %lld: n must be positive", i);
  }
  curve_free(c);   // a curve replaces the previous one; on failure the handle has none
  try {
    std::vector<double2> cen((size_t)ns);
    for (long long i = 0; i < ns; ++i) cen[(size_t)i] = make_double2(centers[2 * i], centers[2 * i + 1]);
    c->d_seg = upload(cen);
    c->d_segw = upload(std::vector<double>(lengths, lengths + ns));
    c->d_segn = upload(std::vector<double>(n_seg, n_seg + ns));
    c->d_cellpts = dev_alloc<double2>((size_t)c->Nv);
    cell_points_kernel<<<(unsigned)std::min<long long>((c->Nv + 255) / 256, 152LL * 8), 256>>>(
        c->nx, c->Nv, c->x0, c->y0, c->h, c->d_cellpts);
    HB_CHECK_LAUNCH();
    c->d_lu = dev_alloc<double2>((size_t)ns * ns);
    c->d_piv = dev_alloc<int>((size_t)ns);
    c->d_kv2s = dev_alloc<double2>((size_t)ns * c->Nv);
    c->d_ks2v = dev_alloc<double2>((size_t)ns * c->Nv);
    std::vector<int> zero(1, 0);
    int* d_sing = upload(zero);
    try {
      assemble(c, c->d_seg, c->d_segw, c->d_segn, ns, c->d_cellpts, c->d_lu, c->d_kv2s, c->d_ks2v, 0);
      const int n = (int)ns;
      for (int k = 0; k < n; ++k) {
        lu_pivot_kernel<<<1, 256>>>(c->d_lu, n, k, c->d_piv, d_sing);
        HB_CHECK_LAUNCH();
        if (k + 1 < n) {
          dim3 grid((unsigned)std::min((n - k - 1 + 255) / 256, 4), (unsigned)(n - k - 1));
          lu_update_kernel<<<grid, 256>>>(c->d_lu, n, k);
          HB_CHECK_LAUNCH();
        }
      }
      HB_CUDA(cudaDeviceSynchronize());
      int sing = 0;
      HB_CUDA(cudaMemcpy(&sing, d_sing, sizeof(int), cudaMemcpyDeviceToHost));
      if (sing) throw Error{HB_ERR_ARG, "K^{s2s} is singular: a zero pivot in its LU factorisation"};
      // the inverse, column by column from the factors (an apply is then one
      // product instead of two sequential triangular solves per column)
      c->d_inv = dev_alloc<double2>((size_t)ns * ns);
      identity_kernel<<<(unsigned)std::min<long long>((ns * ns + 255) / 256, 152LL * 8), 256>>>(c->d_inv, ns);
      HB_CHECK_LAUNCH();
      lu_solve_kernel<<<(unsigned)ns, 256>>>(c->d_lu, c->d_piv, n, c->d_inv, ns);
      HB_CHECK_LAUNCH();
      HB_CUDA(cudaDeviceSynchronize());
    } catch (...) {
      cudaDeviceSynchronize();
      dev_free(d_sing);
      throw;
    }
    dev_free(d_sing);
    c->ns = ns;
  } catch (...) {
    curve_free(c);
    throw;
  }
}

void curve_operators(hb_ctx* c, double2* k_s2s, double2* k_v2s, double2* k_s2v, cudaStream_t st) {
  if (c->ns == 0) throw Error{HB_ERR_STATE, "no curve set (hb_curve_set)"};
  assemble(c, c->d_seg, c->d_segw, c->d_segn, c->ns, c->d_cellpts, k_s2s, k_v2s, k_s2v, st);
}

void apply_inclusion(hb_ctx* c, const double2* s, double2* u, int nrhs, int v2v_dense, cudaStream_t st) {
  NvtxRange nr("hb_apply_inclusion");
  if (c->ns == 0) throw Error{HB_ERR_STATE, "no curve set (hb_curve_set)"};
  if (!v2v_dense && !c->built) throw Error{HB_ERR_STATE, "compressed K^{v2v} before hb_build"};
  if (c->cy_cap < nrhs) {
    dev_free(c->d_cy);
    c->d_cy = nullptr;
    c->cy_cap = 0;
    c->d_cy = dev_alloc<double2>((size_t)c->ns * nrhs * 2);
    c->cy_cap = nrhs;
    HB_CUDA(cudaDeviceSynchronize());
  }
  // U = K^{v2v} I
  if (v2v_dense) dense_apply(c, s, u, nrhs, 0, st);
  else apply_bf(c, s, u, nrhs, 0, c->opt.precision, st);
  const long long ns = c->ns;
  auto grid = [](long long total) { return (unsigned)std::max<long long>(1, std::min<long long>((total + 255) / 256, 152LL * 8)); };
  const bool compressed = c->curve_bf[0] && c->curve_bf[1];
  // Y = K^{v2s} I = h^2 K^{v2s} s
  if (compressed) {
    curve_bf_apply(c, 0, s, c->Nv, c->h * c->h, c->d_cy, ns, 0, nrhs, st);
  } else {
    cgemm_kernel<<<grid(ns * nrhs), 256, 0, st>>>(c->d_kv2s, ns, c->Nv, s, c->Nv, c->d_cy, ns, nrhs, c->h * c->h, 0);
    HB_CHECK_LAUNCH();
  }
  // P = (K^{s2s})^{-1} Y
  double2* P = c->d_cy + (size_t)ns * nrhs;
  cgemm_kernel<<<grid(ns * nrhs), 256, 0, st>>>(c->d_inv, ns, ns, c->d_cy, ns, P, ns, nrhs, 1.0, 0);
  HB_CHECK_LAUNCH();
  // U += K^{s2v} P
  if (compressed) {
    curve_bf_apply(c, 1, P, ns, 1.0, u, c->Nv, 1, nrhs, st);
  } else {
    cgemm_kernel<<<grid(c->Nv * nrhs), 256, 0, st>>>(c->d_ks2v, c->Nv, ns, P, ns, u, c->Nv, nrhs, 1.0, 1);
    HB_CHECK_LAUNCH();
  }
}

}  // namespace hb
