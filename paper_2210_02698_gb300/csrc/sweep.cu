// GPU table builder for media without closed-form ingredients (Sec. 2.3,
// Sec. 4.1): per Chebyshev source node, the factored eikonal (Eq. faceik)
// and the two transport equations of the ingredients (Eq. equVs, d = 2:
// s = -1 for v0, s = 0 for v1) by Lax-Friedrichs sweeping with WENO5
// one-sided derivatives, initialised near the source by the Taylor
// expansions (Eq. expansionT, Eq. expansionV0, Eq. expansionV1), then
// local cubic interpolation of tau^2, v0, v1 to the Chebyshev nodes.
//
// One CTA per source node.  A Gauss-Seidel sweep visits the mesh in one of
// four orderings; an update reads only its own row and column (WENO5 along
// each), so the points of one anti-diagonal never read one another and the
// CTA updates an anti-diagonal at a time, in parallel, with a barrier
// between anti-diagonals.  Along every row and column this is the same
// upwind order as a row-by-row sweep, so each update sees the same new and
// old values: the iterates are those of the sequential sweep, bit for bit.
// The translation unit is compiled without contracted multiply-adds and
// the Taylor values of the fixed points come from the host, so the tables
// equal those of a plain FP64 host implementation of the same scheme.
//
// Scheme (mesh x_i = lo + i h, z_j = lo + j h, field f[j M + i]):
// * factored eikonal tau = tt tb, tt = n0 |r - r0|: H(tb; p, q) =
//   |tt (p, q) + tb grad tt| = n with the Lax-Friedrichs numerical
//   Hamiltonian at the WENO5 derivatives p-, p+, q-, q+ and viscosity
//   alpha = tt; update tb += (n - H_LF) / max(2 alpha / h, dH_LF/dtb at the
//   current WENO weights); points within 5 h of the source (both
//   coordinates) keep their Taylor values; until the largest update over
//   the window is below tol.
// * transports on the window: 2 grad(tau^2) . grad v + c v = f with
//   c = Lap tau^2 - 4 n^2, f = 0 (v0) and c = Lap tau^2, f = Lap v0 (v1),
//   viscosities 2 |d_x tau^2|, 2 |d_z tau^2|; Taylor boxes of 3 h and 1 h;
//   until the largest update over the region of interest is below tol.
// * the three outermost rows and columns (outflow closure) are linear
//   extrapolations of the interior, refreshed after every sweep; WENO
//   stencils past the mesh continue it linearly, the fourth-order central
//   differences of tau^2 and v0 use cubic extrapolation there.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "hb_internal.cuh"

namespace hb {
namespace {

constexpr int SW_THREADS = 256;   // two CTAs (sources) per SM
constexpr int SW_EDGE = 3;            // outflow rows / columns
constexpr int SW_TAYLOR = 46;         // T_2..T_6 (25), B_0..B_4 (15), C_0..C_2 (6)
constexpr double SW_WENO_EPS = 1e-6;
constexpr int SW_FIX_T = 128, SW_FIX_B = 64, SW_FIX_C = 16;   // fixed points per source (boxes of 11^2, 7^2, 3^2)

// f at (i, j), continued linearly past the mesh in i (resp. j)
__device__ __forceinline__ double lin_i(const double* f, int M, int i, int j) {
  const double* r = f + (size_t)j * M;
  if (i < 0) return r[0] + (double)i * (r[1] - r[0]);
  if (i >= M) return r[M - 1] + (double)(i - M + 1) * (r[M - 1] - r[M - 2]);
  return r[i];
}
__device__ __forceinline__ double lin_j(const double* f, int M, int i, int j) {
  if (j < 0) return f[i] + (double)j * (f[(size_t)M + i] - f[i]);
  if (j >= M) {
    const double a = f[(size_t)(M - 1) * M + i], b = f[(size_t)(M - 2) * M + i];
    return a + (double)(j - M + 1) * (a - b);
  }
  return f[(size_t)j * M + i];
}

// f at (i, j), continued past the mesh by the cubic through the four
// values nearest the edge (Lagrange weights at -t, t cells past it)
__device__ __forceinline__ double cub_i(const double* f, int M, int i, int j) {
  if (i >= 0 && i < M) return f[(size_t)j * M + i];
  const int s = i < 0 ? 1 : -1, e = i < 0 ? 0 : M - 1;
  const double t = (double)(i < 0 ? -i : i - M + 1);
  double v = 0.0;
  for (int a = 0; a < 4; ++a) {
    double w = 1.0;
    for (int b = 0; b < 4; ++b)
      if (b != a) w *= (-t - b) / (double)(a - b);
    v += w * f[(size_t)j * M + e + a * s];
  }
  return v;
}
__device__ __forceinline__ double cub_j(const double* f, int M, int i, int j) {
  if (j >= 0 && j < M) return f[(size_t)j * M + i];
  const int s = j < 0 ? 1 : -1, e = j < 0 ? 0 : M - 1;
  const double t = (double)(j < 0 ? -j : j - M + 1);
  double v = 0.0;
  for (int a = 0; a < 4; ++a) {
    double w = 1.0;
    for (int b = 0; b < 4; ++b)
      if (b != a) w *= (-t - b) / (double)(a - b);
    v += w * f[(size_t)(e + a * s) * M + i];
  }
  return v;
}

// WENO5 (Jiang-Peng weights) of five divided differences; *k = the weight
// of v3 minus that of v4 in the result at the current weights
__device__ double weno5(double v1, double v2, double v3, double v4, double v5, double* k) {
  const double p1 = v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0;
  const double p2 = -v2 / 6.0 + 5.0 * v3 / 6.0 + v4 / 3.0;
  const double p3 = v3 / 3.0 + 5.0 * v4 / 6.0 - v5 / 6.0;
  const double e1 = v1 - 2.0 * v2 + v3, f1 = v1 - 4.0 * v2 + 3.0 * v3;
  const double e2 = v2 - 2.0 * v3 + v4, f2 = v2 - v4;
  const double e3 = v3 - 2.0 * v4 + v5, f3 = 3.0 * v3 - 4.0 * v4 + v5;
  const double s1 = 13.0 / 12.0 * e1 * e1 + 0.25 * f1 * f1;
  const double s2 = 13.0 / 12.0 * e2 * e2 + 0.25 * f2 * f2;
  const double s3 = 13.0 / 12.0 * e3 * e3 + 0.25 * f3 * f3;
  const double a1 = 0.1 / ((SW_WENO_EPS + s1) * (SW_WENO_EPS + s1));
  const double a2 = 0.6 / ((SW_WENO_EPS + s2) * (SW_WENO_EPS + s2));
  const double a3 = 0.3 / ((SW_WENO_EPS + s3) * (SW_WENO_EPS + s3));
  const double sum = a1 + a2 + a3;
  *k = (11.0 / 6.0 * a1 + 0.5 * a2 - 0.5 * a3) / sum;
  return (a1 * p1 + a2 * p2 + a3 * p3) / sum;
}

// one-sided derivatives d- and d+ at u[3] of the seven values u[0..6]
// (spacing h), with k- = h d(d-)/du[3] and k+ = -h d(d+)/du[3]
__device__ __forceinline__ void weno_pair(const double* u, double h, double* dm, double* dp, double* km,
                                          double* kp) {
  double d[6];
  for (int k = 0; k < 6; ++k) d[k] = (u[k + 1] - u[k]) / h;
  *dm = weno5(d[0], d[1], d[2], d[3], d[4], km);
  *dp = weno5(d[5], d[4], d[3], d[2], d[1], kp);
}

// p-, p+ (x) and q-, q+ (z) at (i, j); kk = (k of p-, p+, q-, q+)
__device__ __forceinline__ void weno_derivs(const double* f, int M, int i, int j, double h, double* pm, double* pp,
                                            double* qm, double* qp, double* kk) {
  double u[7];
  for (int k = 0; k < 7; ++k) u[k] = lin_i(f, M, i - 3 + k, j);
  weno_pair(u, h, pm, pp, &kk[0], &kk[1]);
  for (int k = 0; k < 7; ++k) u[k] = lin_j(f, M, i, j - 3 + k);
  weno_pair(u, h, qm, qp, &kk[2], &kk[3]);
}

__device__ __forceinline__ bool on_edge(int i, int j, int M) {
  return i < SW_EDGE || j < SW_EDGE || i >= M - SW_EDGE || j >= M - SW_EDGE;
}

// the Taylor-fixed points of one source: mesh index and values
struct SweepFix {
  int nT, nB, nC;
  int pT[SW_FIX_T];
  double tbT[SW_FIX_T], t2T[SW_FIX_T];   // eikonal: initial tb and final tau^2
  int pB[SW_FIX_B];
  double vB[SW_FIX_B];                   // v0 (window indices)
  int pC[SW_FIX_C];
  double vC[SW_FIX_C];                   // v1 (window indices)
};

struct SweepArgs {
  int M, Mw, off;               // mesh and window points a side; the window's first mesh index
  double lo, wlo, h;            // mesh and window origins, spacing
  int g_r0, g_r1;               // eikonal convergence region (mesh indices: the window)
  int w_r0, w_r1;               // transport region of interest (window indices)
  const double* n;              // n on the mesh, M x M
  int NI;
  const double* px;
  const double* pz;             // the Chebyshev node points
  int ns;
  const int* src;               // source k = node src[k]
  const double* taylor;         // ns x 46
  const SweepFix* fix;          // ns
  int max_iter;
  double tol;
  double* scratch;              // ns x stride doubles
  size_t stride;
  unsigned char* masks;         // ns x (M^2 + Mw^2) fixed flags
  double* tau2;
  double* v0;
  double* v1;                   // NI x ns each, [obs][source]
  double* info;                 // ns x 6: iterations and last updates of the three solves
};

// one Gauss-Seidel sweep in ordering o (0..3) of an M x M mesh, an
// anti-diagonal ii + jj = dd at a time; upd(i, j) updates one point
template <class Upd>
__device__ void sweep_once(int o, int M, Upd& upd) {
  for (int dd = 0; dd < 2 * M - 1; ++dd) {
    const int ilo = dd - M + 1 > 0 ? dd - M + 1 : 0, ihi = dd < M - 1 ? dd : M - 1;
    for (int ii = ilo + (int)threadIdx.x; ii <= ihi; ii += (int)blockDim.x) {
      const int jj = dd - ii;
      const int j = (o & 2) ? M - 1 - jj : jj;
      const int i = (o == 1 || o == 2) ? M - 1 - ii : ii;
      upd(i, j);
    }
    __syncthreads();
  }
}

// the outflow closure: the SW_EDGE outermost points of every row, then of
// every column, linear extrapolations of the two nearest inner ones (rows
// first: the corners take the columns' values); fixed points keep theirs
__device__ void extrapolate_edges(double* f, const unsigned char* fixed, int M) {
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    double* r = f + (size_t)j * M;
    for (int i = 0; i < SW_EDGE; ++i) {
      const int t = SW_EDGE - i;
      if (!fixed[(size_t)j * M + i]) r[i] = r[SW_EDGE] + t * (r[SW_EDGE] - r[SW_EDGE + 1]);
      const int k = M - 1 - i;
      if (!fixed[(size_t)j * M + k]) r[k] = r[M - 1 - SW_EDGE] + t * (r[M - 1 - SW_EDGE] - r[M - 2 - SW_EDGE]);
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < SW_EDGE * M; idx += blockDim.x) {
    const int j = idx / M, i = idx % M;
    const int t = SW_EDGE - j;
    const size_t p = (size_t)j * M + i, q = (size_t)(M - 1 - j) * M + i;
    if (!fixed[p]) f[p] = f[(size_t)SW_EDGE * M + i] + t * (f[(size_t)SW_EDGE * M + i] - f[(size_t)(SW_EDGE + 1) * M + i]);
    if (!fixed[q])
      f[q] = f[(size_t)(M - 1 - SW_EDGE) * M + i] +
             t * (f[(size_t)(M - 1 - SW_EDGE) * M + i] - f[(size_t)(M - 2 - SW_EDGE) * M + i]);
  }
  __syncthreads();
}

// fourth-order central differences (cubic continuation past the edge):
// fx, fz (first) and lap (Laplacian), each optional
__device__ void central_diffs(const double* f, int M, double h, double* fx, double* fz, double* lap) {
  for (int p = threadIdx.x; p < M * M; p += blockDim.x) {
    const int j = p / M, i = p % M;
    const double xm2 = cub_i(f, M, i - 2, j), xm1 = cub_i(f, M, i - 1, j), x0 = f[(size_t)j * M + i];
    const double xp1 = cub_i(f, M, i + 1, j), xp2 = cub_i(f, M, i + 2, j);
    const double zm2 = cub_j(f, M, i, j - 2), zm1 = cub_j(f, M, i, j - 1);
    const double zp1 = cub_j(f, M, i, j + 1), zp2 = cub_j(f, M, i, j + 2);
    if (fx) fx[p] = (-xp2 + 8.0 * xp1 - 8.0 * xm1 + xm2) / (12.0 * h);
    if (fz) fz[p] = (-zp2 + 8.0 * zp1 - 8.0 * zm1 + zm2) / (12.0 * h);
    if (lap)
      lap[p] = ((-xp2 + 16.0 * xp1 - 30.0 * x0 + 16.0 * xm1 - xm2) +
                (-zp2 + 16.0 * zp1 - 30.0 * x0 + 16.0 * zm1 - zm2)) /
               (12.0 * h * h);
  }
  __syncthreads();
}

// the largest of the CTA's values v >= 0 (every thread gets it)
__device__ double block_max(double v, unsigned long long* slot) {
  if (threadIdx.x == 0) *slot = 0ull;
  __syncthreads();
  atomicMax(slot, (unsigned long long)__double_as_longlong(v));
  __syncthreads();
  const double r = __longlong_as_double((long long)*slot);
  __syncthreads();
  return r;
}

// local cubic (4 x 4 Lagrange) interpolation of the M x M field f (origin
// lo, spacing h) at (x, z)
__device__ double cubic_at(int M, double lo, double h, const double* f, double x, double z) {
  const double sx = (x - lo) / h, sz = (z - lo) / h;
  int i0 = (int)floor(sx) - 1, j0 = (int)floor(sz) - 1;
  if (i0 < 0) i0 = 0;
  if (j0 < 0) j0 = 0;
  if (i0 > M - 4) i0 = M - 4;
  if (j0 > M - 4) j0 = M - 4;
  double wx[4], wz[4];
  for (int a = 0; a < 4; ++a) {
    wx[a] = 1.0;
    wz[a] = 1.0;
    for (int b = 0; b < 4; ++b) {
      if (b == a) continue;
      wx[a] *= (sx - (i0 + b)) / (double)(a - b);
      wz[a] *= (sz - (j0 + b)) / (double)(a - b);
    }
  }
  double s = 0.0;
  for (int b = 0; b < 4; ++b)
    for (int a = 0; a < 4; ++a) s += wz[b] * wx[a] * f[(size_t)(j0 + b) * M + i0 + a];
  return s;
}

// One CTA per source node: the eikonal on the mesh, then the transports of
// v0 and v1 on the window, then the tables' columns at the nodes.
__global__ void __launch_bounds__(SW_THREADS, 2) sweep_kernel(SweepArgs a) {
  __shared__ unsigned long long red;
  const int k = blockIdx.x;
  const int M = a.M, Mw = a.Mw;
  const size_t N = (size_t)M * M, Nw = (size_t)Mw * Mw;
  const double h = a.h;
  const double x0 = a.px[a.src[k]], z0 = a.pz[a.src[k]];
  const double* T = a.taylor + (size_t)k * SW_TAYLOR;
  const double n0 = sqrt(T[0]);   // T_2 = S0 (X^2 + Z^2), S0 = n0^2
  const SweepFix& F = a.fix[k];
  double* tb = a.scratch + (size_t)k * a.stride;   // factored unknown; later d_x tau^2
  double* tt = tb + N;                             // n0 |r - r0|; later d_z tau^2
  double* gx = tt + N;                             // grad tt; later Lap tau^2
  double* gz = gx + N;
  double* tau2 = gz + N;
  double* ax = tau2 + N;                           // window: d_x tau^2, d_z tau^2, Lap tau^2, n, Lap v0
  double* az = ax + Nw;
  double* lt = az + Nw;
  double* nw = lt + Nw;
  double* rhs = nw + Nw;
  double* v0 = rhs + Nw;
  double* v1 = v0 + Nw;
  unsigned char* fixg = a.masks + (size_t)k * (N + Nw);
  unsigned char* fixw = fixg + N;

  // ---- factored eikonal on the mesh ----
  for (size_t p = threadIdx.x; p < N; p += blockDim.x) {
    const int j = (int)(p / M), i = (int)(p % M);
    const double X = a.lo + i * h - x0, Z = a.lo + j * h - z0;
    const double rho = sqrt(X * X + Z * Z);
    tt[p] = n0 * rho;
    gx[p] = rho > 0 ? n0 * X / rho : 0.0;
    gz[p] = rho > 0 ? n0 * Z / rho : 0.0;
    tb[p] = 1.0;
    fixg[p] = 0;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < F.nT; q += blockDim.x) {
    fixg[F.pT[q]] = 1;
    tb[F.pT[q]] = F.tbT[q];
  }
  __syncthreads();
  double last = 0.0;
  auto eik = [&](int i, int j) {
    const size_t p = (size_t)j * M + i;
    if (fixg[p] || on_edge(i, j, M)) return;
    double pm, pp, qm, qp, kk[4];
    weno_derivs(tb, M, i, j, h, &pm, &pp, &qm, &qp, kk);
    const double A = tt[p] * 0.5 * (pm + pp) + tb[p] * gx[p];
    const double B = tt[p] * 0.5 * (qm + qp) + tb[p] * gz[p];
    const double H = sqrt(A * A + B * B);
    const double alpha = tt[p];
    const double hlf = H - alpha * 0.5 * (pp - pm) - alpha * 0.5 * (qp - qm);
    // the first-order coefficient of tb in hlf, or its value at the
    // current WENO weights where that is larger (no overshoot)
    const double dH = H > 0 ? (A * (tt[p] * 0.5 * (kk[0] - kk[1]) / h + gx[p]) +
                               B * (tt[p] * 0.5 * (kk[2] - kk[3]) / h + gz[p])) / H
                            : 0.0;
    const double kw = dH + alpha * 0.5 * (kk[0] + kk[1] + kk[2] + kk[3]) / h;
    const double d = (a.n[p] - hlf) / fmax(2.0 * alpha / h, kw);
    tb[p] += d;
    if (fabs(d) > last && i >= a.g_r0 && i <= a.g_r1 && j >= a.g_r0 && j <= a.g_r1) last = fabs(d);
  };
  int it;
  double worst = 0.0;
  for (it = 0; it < a.max_iter; ++it) {
    last = 0.0;
    for (int o = 0; o < 4; ++o) {
      sweep_once(o, M, eik);
      extrapolate_edges(tb, fixg, M);
    }
    worst = block_max(last, &red);
    if (worst < a.tol) break;
  }
  if (threadIdx.x == 0) {
    a.info[(size_t)k * 6 + 0] = it;
    a.info[(size_t)k * 6 + 3] = worst;
  }
  for (size_t p = threadIdx.x; p < N; p += blockDim.x) tau2[p] = (tt[p] * tb[p]) * (tt[p] * tb[p]);
  __syncthreads();
  for (int q = threadIdx.x; q < F.nT; q += blockDim.x) tau2[F.pT[q]] = F.t2T[q];
  __syncthreads();
  // derivatives of tau^2 on the mesh (true neighbours at the window's edge)
  central_diffs(tau2, M, h, tb, tt, gx);
  for (size_t q = threadIdx.x; q < Nw; q += blockDim.x) {
    const int j = (int)(q / Mw), i = (int)(q % Mw);
    const size_t p = (size_t)(j + a.off) * M + i + a.off;
    ax[q] = tb[p];
    az[q] = tt[p];
    lt[q] = gx[p];
    nw[q] = a.n[p];
  }
  __syncthreads();

  // ---- transports on the window: s = 0 (v0), s = 1 (v1) ----
  for (int s = 0; s < 2; ++s) {
    double* v = s == 0 ? v0 : v1;
    if (s == 1) central_diffs(v0, Mw, h, nullptr, nullptr, rhs);
    const double start = s == 0 ? T[25] : T[40];   // B_0, C_0
    for (size_t p = threadIdx.x; p < Nw; p += blockDim.x) {
      v[p] = start;
      fixw[p] = 0;
    }
    __syncthreads();
    const int nf = s == 0 ? F.nB : F.nC;
    for (int q = threadIdx.x; q < nf; q += blockDim.x) {
      const int p = s == 0 ? F.pB[q] : F.pC[q];
      fixw[p] = 1;
      v[p] = s == 0 ? F.vB[q] : F.vC[q];
    }
    __syncthreads();
    auto tra = [&](int i, int j) {
      const size_t p = (size_t)j * Mw + i;
      if (fixw[p] || on_edge(i, j, Mw)) return;
      double pm, pp, qm, qp, kk[4];
      weno_derivs(v, Mw, i, j, h, &pm, &pp, &qm, &qp, kk);
      const double c = s == 0 ? lt[p] - 4.0 * nw[p] * nw[p] : lt[p];
      const double f = s == 0 ? 0.0 : rhs[p];
      const double alx = 2.0 * fabs(ax[p]), alz = 2.0 * fabs(az[p]);
      const double hlf = ax[p] * (pm + pp) + az[p] * (qm + qp) + c * v[p] - alx * 0.5 * (pp - pm) -
                         alz * 0.5 * (qp - qm);
      // the first-order coefficient of v in hlf (c v not lagged), or its
      // value at the current WENO weights where that is larger
      const double den = (alx + alz) / h + c;
      if (!(den > 0.25 * (alx + alz) / h)) return;
      const double kw = (ax[p] * (kk[0] - kk[1]) + az[p] * (kk[2] - kk[3]) + 0.5 * alx * (kk[0] + kk[1]) +
                         0.5 * alz * (kk[2] + kk[3])) / h + c;
      const double d = (f - hlf) / fmax(den, kw);
      v[p] += d;
      if (fabs(d) > last && i >= a.w_r0 && i <= a.w_r1 && j >= a.w_r0 && j <= a.w_r1) last = fabs(d);
    };
    worst = 0.0;
    for (it = 0; it < a.max_iter; ++it) {
      last = 0.0;
      for (int o = 0; o < 4; ++o) {
        sweep_once(o, Mw, tra);
        extrapolate_edges(v, fixw, Mw);
      }
      worst = block_max(last, &red);
      if (worst < a.tol) break;
    }
    if (threadIdx.x == 0) {
      a.info[(size_t)k * 6 + 1 + s] = it;
      a.info[(size_t)k * 6 + 4 + s] = worst;
    }
  }

  // ---- the tables' column k at the nodes ----
  for (int i = threadIdx.x; i < a.NI; i += blockDim.x) {
    a.tau2[(size_t)i * a.ns + k] = cubic_at(M, a.lo, h, tau2, a.px[i], a.pz[i]);
    a.v0[(size_t)i * a.ns + k] = cubic_at(Mw, a.wlo, h, v0, a.px[i], a.pz[i]);
    a.v1[(size_t)i * a.ns + k] = cubic_at(Mw, a.wlo, h, v1, a.px[i], a.pz[i]);
  }
}

}  // namespace

// ------------------------------------------------------------------ host ----
namespace {

// homogeneous polynomial of degree deg (deg + 1 coefficients of
// X^(deg - m) Z^m) at (X, Z), and the sum of the pieces k0..k1 stored one
// after the other from c on
double homog_at(const double* c, int deg, double X, double Z) {
  double s = 0.0;
  for (int m = 0; m <= deg; ++m) s += c[m] * std::pow(X, deg - m) * std::pow(Z, m);
  return s;
}
double pieces_at(const double* c, int k0, int k1, double X, double Z) {
  double s = 0.0;
  for (int k = k0; k <= k1; ++k) {
    s += homog_at(c, k, X, Z);
    c += k + 1;
  }
  return s;
}

// a device array freed on scope exit
template <class T>
struct DeviceVec {
  T* p = nullptr;
  DeviceVec() = default;
  DeviceVec(const DeviceVec&) = delete;
  DeviceVec& operator=(const DeviceVec&) = delete;
  ~DeviceVec() { dev_free(p); }
  void alloc(size_t n) { p = dev_alloc<T>(n); }
  void upload(const T* h, size_t n) {
    alloc(n);
    if (n) HB_CUDA(cudaMemcpy(p, h, n * sizeof(T), cudaMemcpyHostToDevice));
  }
  void download(T* h, size_t n) const {
    if (n) HB_CUDA(cudaMemcpy(h, p, n * sizeof(T), cudaMemcpyDeviceToHost));
  }
};

// mesh indices i with |lo + i h - c| <= r h (1 + 1e-12), i in [0, n)
std::vector<int> box_indices(double lo, double h, int n, double c, int r) {
  std::vector<int> out;
  for (int i = 0; i < n; ++i)
    if (std::fabs(lo + i * h - c) <= r * h * (1 + 1e-12)) out.push_back(i);
  return out;
}

}  // namespace

void sweep_tables(int M, double lo, double h, int w0, int w1, int roi0, int roi1, const double* n_mesh, int NI,
                  const double* px, const double* pz, int ns, const int* src, const double* taylor, int max_iter,
                  double tol, double* tau2, double* v0, double* v1, double* info) {
  if (!n_mesh || !px || !pz || !src || !taylor || !tau2 || !v0 || !v1 || !info) throw arg_error("null argument");
  if (!(M >= 8 && h > 0 && w0 >= 0 && w1 < M && w1 - w0 + 1 >= 8 && roi0 >= 0 && roi1 <= w1 - w0 && roi0 <= roi1))
    throw arg_error("bad mesh (M >= 8, h > 0, 0 <= w0, w1 < M, window >= 8 points, roi inside the window)");
  if (NI < 1 || ns < 0 || max_iter < 0 || !(tol >= 0)) throw arg_error("bad sizes or tolerance");
  if ((long long)M * M > (1LL << 28)) throw Error{HB_ERR_UNSUPPORTED, "mesh larger than 2^28 points"};
  for (int k = 0; k < ns; ++k) {
    if (src[k] < 0 || src[k] >= NI) throw arg_error("source %d: node %d outside [0, %d)", k, src[k], NI);
    if (!(taylor[(size_t)k * SW_TAYLOR] > 0)) throw arg_error("source %d: S0 = n0^2 must be positive", k);
  }
  if (ns == 0) return;
  const int Mw = w1 - w0 + 1;
  const double wlo = lo + w0 * h;   // the window's origin
  // the Taylor-fixed points of every source, on the host
  std::vector<SweepFix> fix((size_t)ns);
  for (int k = 0; k < ns; ++k) {
    SweepFix& F = fix[(size_t)k];
    const double x0 = px[src[k]], z0 = pz[src[k]];
    const double* T = taylor + (size_t)k * SW_TAYLOR;
    const double n0 = std::sqrt(T[0]);
    const std::vector<int> bi = box_indices(lo, h, M, x0, 5), bj = box_indices(lo, h, M, z0, 5);
    F.nT = 0;
    for (int j : bj)
      for (int i : bi) {
        if (F.nT == SW_FIX_T) throw Error{HB_ERR_STATE, "eikonal Taylor box larger than expected"};
        const double X = lo + i * h - x0, Z = lo + j * h - z0;
        const double rho = std::sqrt(X * X + Z * Z);
        const double t2 = pieces_at(T, 2, 6, X, Z);
        F.pT[F.nT] = j * M + i;
        F.tbT[F.nT] = rho > 0 ? std::sqrt(t2 > 0 ? t2 : 0.0) / (n0 * rho) : 1.0;
        F.t2T[F.nT] = t2;
        ++F.nT;
      }
    for (int s = 0; s < 2; ++s) {
      const int r = s == 0 ? 3 : 1;
      const std::vector<int> wi = box_indices(wlo, h, Mw, x0, r), wj = box_indices(wlo, h, Mw, z0, r);
      int& nf = s == 0 ? F.nB : F.nC;
      nf = 0;
      for (int j : wj)
        for (int i : wi) {
          if (nf == (s == 0 ? SW_FIX_B : SW_FIX_C)) throw Error{HB_ERR_STATE, "transport Taylor box larger than expected"};
          const double X = wlo + i * h - x0, Z = wlo + j * h - z0;
          if (s == 0) {
            F.pB[nf] = j * Mw + i;
            F.vB[nf] = pieces_at(T + 25, 0, 4, X, Z);
          } else {
            F.pC[nf] = j * Mw + i;
            F.vC[nf] = pieces_at(T + 40, 0, 2, X, Z);
          }
          ++nf;
        }
    }
  }
  const size_t N = (size_t)M * M, Nw = (size_t)Mw * Mw;
  const size_t stride = 5 * N + 7 * Nw;
  DeviceVec<double> d_n, d_px, d_pz, d_tay, d_scr, d_t2, d_v0, d_v1, d_info;
  DeviceVec<int> d_src;
  DeviceVec<SweepFix> d_fix;
  DeviceVec<unsigned char> d_mask;
  d_n.upload(n_mesh, N);
  d_px.upload(px, (size_t)NI);
  d_pz.upload(pz, (size_t)NI);
  d_src.upload(src, (size_t)ns);
  d_tay.upload(taylor, (size_t)ns * SW_TAYLOR);
  d_fix.upload(fix.data(), fix.size());
  d_scr.alloc((size_t)ns * stride);
  d_mask.alloc((size_t)ns * (N + Nw));
  d_t2.alloc((size_t)NI * ns);
  d_v0.alloc((size_t)NI * ns);
  d_v1.alloc((size_t)NI * ns);
  d_info.alloc((size_t)ns * 6);
  SweepArgs A{};
  A.M = M;
  A.Mw = Mw;
  A.off = w0;
  A.lo = lo;
  A.wlo = wlo;
  A.h = h;
  A.g_r0 = w0;
  A.g_r1 = w1;
  A.w_r0 = roi0;
  A.w_r1 = roi1;
  A.n = d_n.p;
  A.NI = NI;
  A.px = d_px.p;
  A.pz = d_pz.p;
  A.ns = ns;
  A.src = d_src.p;
  A.taylor = d_tay.p;
  A.fix = d_fix.p;
  A.max_iter = max_iter;
  A.tol = tol;
  A.scratch = d_scr.p;
  A.stride = stride;
  A.masks = d_mask.p;
  A.tau2 = d_t2.p;
  A.v0 = d_v0.p;
  A.v1 = d_v1.p;
  A.info = d_info.p;
  sweep_kernel<<<(unsigned)ns, SW_THREADS>>>(A);
  HB_CHECK_LAUNCH();
  HB_CUDA(cudaDeviceSynchronize());
  d_t2.download(tau2, (size_t)NI * ns);
  d_v0.download(v0, (size_t)NI * ns);
  d_v1.download(v1, (size_t)NI * ns);
  d_info.download(info, (size_t)ns * 6);
}

// ------------------------------------------------ near-source series ----
// Homogeneous polynomials in the offset (X, Z) = r - r0: piece of degree k
// = k + 1 coefficients of X^(k - m) Z^m.
namespace {
using Poly = std::vector<double>;

Poly zero_poly(int deg) { return Poly((size_t)deg + 1, 0.0); }
int degree(const Poly& p) { return (int)p.size() - 1; }

Poly pmul(const Poly& p, const Poly& q) {
  Poly r = zero_poly(degree(p) + degree(q));
  for (size_t a = 0; a < p.size(); ++a)
    for (size_t b = 0; b < q.size(); ++b) r[a + b] += p[a] * q[b];
  return r;
}
void padd(Poly& acc, const Poly& p, double w) {   // acc += w p (same degree)
  if (p.size() != acc.size()) throw Error{HB_ERR_STATE, "series pieces of different degrees"};
  for (size_t m = 0; m < acc.size(); ++m) acc[m] += w * p[m];
}
// d/dX and d/dZ of a piece of degree k >= 1 (pieces of degree k - 1)
Poly dx(const Poly& p) {
  const int k = degree(p);
  Poly r = zero_poly(std::max(k - 1, 0));
  for (int m = 0; m < k; ++m) r[(size_t)m] = (k - m) * p[(size_t)m];
  return r;
}
Poly dz(const Poly& p) {
  const int k = degree(p);
  Poly r = zero_poly(std::max(k - 1, 0));
  for (int m = 0; m < k; ++m) r[(size_t)m] = (m + 1) * p[(size_t)m + 1];
  return r;
}
Poly lap(const Poly& p) {   // degree k - 2 (zero below degree 2)
  const int k = degree(p);
  if (k < 2) return zero_poly(0);
  Poly r = dx(dx(p));
  padd(r, dz(dz(p)), 1.0);
  return r;
}
Poly grad_dot(const Poly& p, const Poly& q) {   // grad p . grad q
  if (degree(p) < 1 || degree(q) < 1) return zero_poly(std::max(degree(p) + degree(q) - 2, 0));
  Poly r = pmul(dx(p), dx(q));
  padd(r, pmul(dz(p), dz(q)), 1.0);
  return r;
}
}  // namespace

// The 46 Taylor numbers of one source from the series of n^2 about it
// (S_0..S_4, 15 numbers): the recursions of Sec. 2.2 for d = 2 -
// T_2 = S0 (X^2 + Z^2) and (P - 1) S0 T_P = sum_{k=1}^{P-2} S_k T_{P-k}
// - 1/4 sum_{k=2}^{P-2} grad T_{k+1} . grad T_{P-k+1} (Eq. recursiveT);
// B_0 = 1 / (2 sqrt(pi)) and 2 P S0 B_P = - sum_{k=1}^{P-1} grad B_k .
// grad T_{P+2-k} - 1/2 sum_{k<P} B_k Lap T_{P+2-k} + 2 sum_{k<P} B_k
// S_{P-k} (Eq. recursiveB); 2 S0 C_0 = 1/2 Lap B_2, 4 S0 C_1 = 1/2 Lap B_3
// - 1/2 C_0 Lap T_3 (Eq. C0, Eq. C1), 2 (P + 1) S0 C_P = 1/2 Lap B_{P+2} -
// sum_{k=1}^{P-1} grad C_k . grad T_{P+2-k} - 1/2 sum_{k<P} C_k Lap
// T_{P+2-k} (Eq. recursiveC; the (2 - d) terms vanish) - packed as
// T_2..T_6, B_0..B_4, C_0..C_2.
void sweep_taylor_one(const double* s2, double* out) {
  constexpr int PT = 6, PB = 4, PC = 2;
  std::vector<Poly> S;
  for (int k = 0, o = 0; k <= 4; o += k + 1, ++k) S.emplace_back(s2 + o, s2 + o + k + 1);
  auto Sk = [&](int k) { return k <= 4 ? S[(size_t)k] : zero_poly(k); };
  const double S0 = S[0][0];
  if (!(S0 > 0)) throw arg_error("S0 = n0^2 must be positive");
  std::vector<Poly> T = {zero_poly(0), zero_poly(1), Poly{S0, 0.0, S0}};
  for (int P = 3; P <= PT; ++P) {
    Poly acc = zero_poly(P);
    for (int k = 1; k <= P - 2; ++k) padd(acc, pmul(Sk(k), T[(size_t)(P - k)]), 1.0);
    for (int k = 2; k <= P - 2; ++k) padd(acc, grad_dot(T[(size_t)k + 1], T[(size_t)(P - k + 1)]), -0.25);
    for (double& c : acc) c /= (P - 1) * S0;
    T.push_back(acc);
  }
  constexpr double PI = 3.141592653589793;   // the double nearest pi
  std::vector<Poly> B = {Poly{1.0 / (2.0 * std::sqrt(PI))}};
  for (int P = 1; P <= PB; ++P) {
    Poly acc = zero_poly(P);
    for (int k = 1; k <= P - 1; ++k) padd(acc, grad_dot(B[(size_t)k], T[(size_t)(P + 2 - k)]), -1.0);
    for (int k = 0; k <= P - 1; ++k) {
      padd(acc, pmul(B[(size_t)k], lap(T[(size_t)(P + 2 - k)])), -0.5);
      padd(acc, pmul(B[(size_t)k], Sk(P - k)), 2.0);
    }
    for (double& c : acc) c /= 2 * P * S0;
    B.push_back(acc);
  }
  std::vector<Poly> C;
  {
    Poly c0 = lap(B[2]);
    for (double& c : c0) c = 0.5 * c / (2 * S0);
    C.push_back(c0);
    Poly c1 = lap(B[3]);
    for (double& c : c1) c *= 0.5;
    padd(c1, pmul(lap(T[3]), C[0]), -0.5);
    for (double& c : c1) c /= 4 * S0;
    C.push_back(c1);
  }
  for (int P = 2; P <= PC; ++P) {
    Poly acc = lap(B[(size_t)P + 2]);
    for (double& c : acc) c *= 0.5;
    for (int k = 1; k <= P - 1; ++k) padd(acc, grad_dot(C[(size_t)k], T[(size_t)(P + 2 - k)]), -1.0);
    for (int k = 0; k <= P - 1; ++k) padd(acc, pmul(C[(size_t)k], lap(T[(size_t)(P + 2 - k)])), -0.5);
    for (double& c : acc) c /= 2 * (P + 1) * S0;
    C.push_back(acc);
  }
  size_t o = 0;
  for (int k = 2; k <= PT; ++k)
    for (double c : T[(size_t)k]) out[o++] = c;
  for (int k = 0; k <= PB; ++k)
    for (double c : B[(size_t)k]) out[o++] = c;
  for (int k = 0; k <= PC; ++k)
    for (double c : C[(size_t)k]) out[o++] = c;
}

}  // namespace hb
