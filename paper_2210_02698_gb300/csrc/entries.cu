// entries.cu - evaluation of the HB matrix entries K_ij on the device
// (Sec. 3.1 Eq. m_v2v; Sec. 4.1 Eq. chebinterp / Eq. chebinterpblock;
// Eq. babich with N = 1; Eq. termf; Appendix A Eq. HankelIntegral2dlemma),
// and the matrix-free dense apply U = K I and its adjoint.
//
// Interpolation layout.  With T_i(r) = l_{i1}(x) l_{i2}(z) and the grid's
// cell coordinates x_a, z_b, the tensor structure of Eq. chebinterp is
// contracted in stages so that each entry costs O(n_I) FP64 FMAs per
// ingredient instead of O(N_I^2):
//   LX[a][k] = l_k(x_a), LZ[b][k] = l_k(z_b)                     (barycentric)
//   H[q][b][i][j1] = sum_{j2} F_q[i][(j2,j1)] LZ[b][j2]          (per source line b)
//   G_j[q][i]      = sum_{j1} H[q][b_j][i][j1] LX[a_j][j1]        (= (F_q T(r_j))_i)
//   P[q][i1]       = sum_{i2} LZ[b_i][i2] G_j[q][(i2,i1)]         (per observation line)
//   f_q(r_i, r_j)  = sum_{i1} LX[a_i][i1] P[q][i1]
// q = 0, 1, 2 for tau^2, v0, v1.  The adjoint uses the transposed tables.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "bessel.cuh"
#include "hb_internal.cuh"

namespace hb {

constexpr int MAX_NI = 16;   // n_I supported by the fused kernels

// ----------------------------------------------------------- helpers ----
// Barycentric Lagrange basis at the coordinates of one grid axis.
__global__ void lagrange_kernel(const double* __restrict__ nodes, int nI, double origin,
                                double h, int count, double* __restrict__ L) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= count) return;
  double x = origin + (a + 0.5) * h;
  double w[MAX_NI], d[MAX_NI];
  int hit = -1;
  for (int k = 0; k < nI; ++k) {
    double p = 1.0;
    for (int m = 0; m < nI; ++m)
      if (m != k) p *= (nodes[k] - nodes[m]);
    w[k] = 1.0 / p;
    d[k] = x - nodes[k];
    if (d[k] == 0.0) hit = k;
  }
  if (hit >= 0) {
    for (int k = 0; k < nI; ++k) L[(size_t)a * nI + k] = (k == hit) ? 1.0 : 0.0;
    return;
  }
  double den = 0.0;
  for (int k = 0; k < nI; ++k) den += w[k] / d[k];
  for (int k = 0; k < nI; ++k) L[(size_t)a * nI + k] = (w[k] / d[k]) / den;
}

// H[q][b][i][j1] = sum_j2 F_q[i][j2*nI + j1] LZ[b][j2]
__global__ void htable_kernel(const double* __restrict__ F, const double* __restrict__ LZ, int ny,
                              int nI, double* __restrict__ H) {
  const int NI = nI * nI;
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = 3LL * ny * NI * nI;
  if (idx >= total) return;
  int j1 = idx % nI;
  long long t = idx / nI;
  int i = t % NI;
  t /= NI;
  int b = t % ny;
  int q = (int)(t / ny);
  const double* Fq = F + (size_t)q * NI * NI + (size_t)i * NI;
  double acc = 0.0;
  for (int j2 = 0; j2 < nI; ++j2) acc = fma(Fq[j2 * nI + j1], LZ[(size_t)b * nI + j2], acc);
  H[idx] = acc;
}

// Self term K_ii = (i/4) I / h^2, I = (n0 w)^-2 [8 int_0^{pi/4} R H1(R) dth + 4i],
// R = h n0 w / (2 cos th)  (Appendix A); theta quadrature: Gauss-Legendre.
__global__ void self_kernel(const double* __restrict__ ncell, long long Nv, double h, double omega,
                            const double* __restrict__ glx, const double* __restrict__ glw, int ngl,
                            double2* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nv) return;
  double n0 = ncell[i];
  double k = 0.5 * h * n0 * omega;
  double re = 0.0, im = 0.0;
  for (int g = 0; g < ngl; ++g) {
    double th = (HB_PI / 8.0) * (glx[g] + 1.0);   // map [-1,1] -> [0, pi/4]
    double R = k / cos(th);
    Bessel01 b = bessel01(R);
    re = fma(glw[g], R * b.j1, re);
    im = fma(glw[g], R * b.y1, im);
  }
  re *= HB_PI / 8.0;
  im *= HB_PI / 8.0;
  double s = 1.0 / ((n0 * omega) * (n0 * omega));
  double Ire = s * 8.0 * re;
  double Iim = s * (8.0 * im + 4.0);
  // (i/4)(Ire + i Iim) / h^2
  out[i] = make_double2(-0.25 * Iim / (h * h), 0.25 * Ire / (h * h));
}

// Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_n.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(HB_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void setup_tables(hb_ctx* c) {
  const int nI = c->nI, NI = c->NI;
  std::vector<double> nodes(c->nodes_x);
  nodes.insert(nodes.end(), c->nodes_y.begin(), c->nodes_y.end());
  c->d_nodes = upload(nodes);
  std::vector<double> tabs((size_t)6 * NI * NI);
  for (int q = 0; q < 3; ++q)
    for (int i = 0; i < NI; ++i)
      for (int j = 0; j < NI; ++j) {
        tabs[(size_t)q * NI * NI + (size_t)i * NI + j] = c->tab[q][(size_t)i * NI + j];
        tabs[(size_t)(3 + q) * NI * NI + (size_t)i * NI + j] = c->tab[q][(size_t)j * NI + i];
      }
  c->d_tab = upload(tabs);
  c->d_LX = dev_alloc<double>((size_t)c->nx * nI);
  c->d_LZ = dev_alloc<double>((size_t)c->ny * nI);
  lagrange_kernel<<<(c->nx + 127) / 128, 128>>>(c->d_nodes, nI, c->x0, c->h, c->nx, c->d_LX);
  HB_CHECK_LAUNCH();
  lagrange_kernel<<<(c->ny + 127) / 128, 128>>>(c->d_nodes + nI, nI, c->y0, c->h, c->ny, c->d_LZ);
  HB_CHECK_LAUNCH();
  long long htotal = 3LL * c->ny * NI * nI;
  for (int t = 0; t < 2; ++t) {
    c->d_H[t] = dev_alloc<double>(htotal);
    htable_kernel<<<(unsigned)((htotal + 255) / 256), 256>>>(c->d_tab + (size_t)t * 3 * NI * NI,
                                                            c->d_LZ, c->ny, nI, c->d_H[t]);
    HB_CHECK_LAUNCH();
  }
  c->d_ncell = upload(c->n_cells);
  compute_self(c);
}

// The cell-integrated self terms at the handle's omega (the only
// precomputed entry data that depends on it; the tables do not), into
// d_self (allocated on first use).
void compute_self(hb_ctx* c) {
  if (!c->d_self) c->d_self = dev_alloc<double2>(c->Nv);
  std::vector<double> glx, glw;
  gauss_legendre(64, glx, glw);
  // the quadrature rule is scratch: freed on the way out, also when a step throws
  double* d_gl = upload(glx);
  double* d_gw = nullptr;
  try {
    d_gw = upload(glw);
    self_kernel<<<(unsigned)((c->Nv + 127) / 128), 128>>>(c->d_ncell, c->Nv, c->h, c->omega, d_gl, d_gw,
                                                          64, c->d_self);
    HB_CHECK_LAUNCH();
    HB_CUDA(cudaDeviceSynchronize());
  } catch (...) {
    dev_free(d_gl);
    dev_free(d_gw);
    throw;
  }
  dev_free(d_gl);
  dev_free(d_gw);
}

EntryParams entry_params(const hb_ctx* c, int transposed) {
  EntryParams p;
  p.nx = c->nx;
  p.ny = c->ny;
  p.nI = c->nI;
  p.NI = c->NI;
  p.omega = c->omega;
  p.LX = c->d_LX;
  p.LZ = c->d_LZ;
  p.H = c->d_H[transposed ? 1 : 0];
  p.self = c->d_self;
  return p;
}

// ------------------------------------------------------- dense apply ----
// One CTA owns 64 consecutive cells of one grid line (the outputs) and sweeps
// the source line segments of 64 cells of its share of the source lines
// (blockIdx.y of gridDim.y contiguous shares; all lines when gridDim.y = 1).
// Thread t: output o = t & 63, quarter t >> 6 takes every 4th source of the
// segment.  RC right-hand sides per pass.  FP64 throughout.  With one share
// the CTA writes u; with several it writes its unscaled partial sums to
// part[share][r][cell] and dense_reduce_kernel adds the shares in order.
constexpr int DT = 64;

template <int RC, bool ADJ>
__global__ void __launch_bounds__(256) dense_kernel(EntryParams p, const double2* __restrict__ s,
                                                    double2* __restrict__ u, long long Nv, int r0,
                                                    double scale, double2* __restrict__ part) {
  extern __shared__ double smem[];
  const int nI = p.nI;
  double* LXo = smem;                         // DT x 16
  double* M = LXo + DT * MAX_NI;              // 3 x 16 x 16
  double* P = M + 3 * MAX_NI * MAX_NI;        // 3 x DT x 16
  double2* S = reinterpret_cast<double2*>(P + 3 * DT * MAX_NI);  // DT x RC
  double2* red = S + DT * RC;                 // 3 x DT x RC (quarter partial sums)

  const int t = threadIdx.x;
  const int ntx = (p.nx + DT - 1) / DT;
  const int bo = blockIdx.x / ntx;
  const int ao0 = (blockIdx.x % ntx) * DT;
  const int olen = min(DT, p.nx - ao0);
  const int o = t & (DT - 1);
  const int quarter = t >> 6;
  const long long onat = (long long)bo * p.nx + ao0 + o;

  for (int idx = t; idx < DT * nI; idx += blockDim.x) {
    int r = idx / nI, k = idx % nI;
    LXo[r * MAX_NI + k] = (r < olen) ? p.LX[(size_t)(ao0 + r) * nI + k] : 0.0;
  }
  double2 acc[RC];
#pragma unroll
  for (int r = 0; r < RC; ++r) acc[r] = make_double2(0.0, 0.0);
  const int NI = p.NI;

  const int bq0 = (int)((long long)p.ny * blockIdx.y / gridDim.y);
  const int bq1 = (int)((long long)p.ny * (blockIdx.y + 1) / gridDim.y);
  for (int bq = bq0; bq < bq1; ++bq) {
    __syncthreads();
    // M[q][i1][j1] = sum_i2 LZ[bo][i2] H[q][bq][(i2,i1)][j1]
    for (int idx = t; idx < 3 * nI * nI; idx += blockDim.x) {
      int q = idx / (nI * nI), i1 = (idx / nI) % nI, j1 = idx % nI;
      const double* Hq = p.H + (((size_t)q * p.ny + bq) * NI) * nI;
      double a = 0.0;
      for (int i2 = 0; i2 < nI; ++i2)
        a = fma(p.LZ[(size_t)bo * nI + i2], Hq[(size_t)(i2 * nI + i1) * nI + j1], a);
      M[(q * MAX_NI + i1) * MAX_NI + j1] = a;
    }
    __syncthreads();
    for (int aq0 = 0; aq0 < p.nx; aq0 += DT) {
      const int qlen = min(DT, p.nx - aq0);
      // P[q][c][i1] = sum_j1 M[q][i1][j1] LX[a_c][j1]
      for (int idx = t; idx < 3 * DT * nI; idx += blockDim.x) {
        int q = idx / (DT * nI), cc = (idx / nI) % DT, i1 = idx % nI;
        double a = 0.0;
        if (cc < qlen) {
          const double* lx = p.LX + (size_t)(aq0 + cc) * nI;
          for (int j1 = 0; j1 < nI; ++j1) a = fma(M[(q * MAX_NI + i1) * MAX_NI + j1], lx[j1], a);
        }
        P[(q * DT + cc) * MAX_NI + i1] = a;
      }
      for (int idx = t; idx < DT * RC; idx += blockDim.x) {
        int cc = idx / RC, r = idx % RC;
        double2 v = make_double2(0.0, 0.0);
        if (cc < qlen) v = s[(size_t)(r0 + r) * Nv + (size_t)bq * p.nx + aq0 + cc];
        S[cc * RC + r] = v;
      }
      __syncthreads();
      if (o < olen) {
        for (int cc = quarter; cc < qlen; cc += 4) {
          double f[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const double* pq = P + (q * DT + cc) * MAX_NI;
            double a = 0.0;
            for (int i1 = 0; i1 < nI; ++i1) a = fma(LXo[o * MAX_NI + i1], pq[i1], a);
            f[q] = a;
          }
          const long long qnat = (long long)bq * p.nx + aq0 + cc;
          double2 g = (qnat == onat) ? p.self[onat] : hb_green(f[0], f[1], f[2], p.omega);
          if (ADJ) g.y = -g.y;
#pragma unroll
          for (int r = 0; r < RC; ++r) {
            double2 x = S[cc * RC + r];
            acc[r].x = fma(g.x, x.x, fma(-g.y, x.y, acc[r].x));
            acc[r].y = fma(g.x, x.y, fma(g.y, x.x, acc[r].y));
          }
        }
      }
      __syncthreads();
    }
  }
  // reduce the four quarters
  if (quarter > 0) {
#pragma unroll
    for (int r = 0; r < RC; ++r) red[((quarter - 1) * DT + o) * RC + r] = acc[r];
  }
  __syncthreads();
  if (quarter == 0 && o < olen) {
#pragma unroll
    for (int r = 0; r < RC; ++r) {
      double2 a = acc[r];
      for (int qq = 0; qq < 3; ++qq) {
        double2 b = red[(qq * DT + o) * RC + r];
        a.x += b.x;
        a.y += b.y;
      }
      if (part) part[((size_t)blockIdx.y * RC + r) * Nv + onat] = a;
      else u[(size_t)(r0 + r) * Nv + onat] = make_double2(a.x * scale, a.y * scale);
    }
  }
}

// u[r0 + r][cell] = scale * (sum over the shares, in order, of part[share][r][cell])
__global__ void dense_reduce_kernel(const double2* __restrict__ part, double2* __restrict__ u, long long Nv, int rc,
                                    int nsplit, int r0, double scale) {
  const long long n = Nv * rc;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double2 a = make_double2(0.0, 0.0);
    for (int k = 0; k < nsplit; ++k) {
      const double2 b = part[(size_t)k * n + i];
      a.x += b.x;
      a.y += b.y;
    }
    const long long r = i / Nv, cell = i - r * Nv;
    u[(size_t)(r0 + r) * Nv + cell] = make_double2(a.x * scale, a.y * scale);
  }
}

template <int RC, bool ADJ>
static void launch_dense(const EntryParams& p, const double2* s, double2* u, long long Nv, int r0,
                         double scale, int nsplit, double2* part, cudaStream_t st) {
  size_t sm = sizeof(double) * (DT * MAX_NI + 3 * MAX_NI * MAX_NI + 3 * DT * MAX_NI) +
              sizeof(double2) * (DT * RC + 3 * DT * RC);
  auto k = dense_kernel<RC, ADJ>;
  HB_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int ntx = (p.nx + DT - 1) / DT;
  k<<<dim3(ntx * p.ny, nsplit), 256, sm, st>>>(p, s, u, Nv, r0, scale, nsplit > 1 ? part : nullptr);
  HB_CHECK_LAUNCH();
  if (nsplit > 1) {
    const long long n = Nv * RC;
    dense_reduce_kernel<<<(unsigned)std::min<long long>((n + 255) / 256, 152LL * 8), 256, 0, st>>>(
        part, u, Nv, RC, nsplit, r0, scale);
    HB_CHECK_LAUNCH();
  }
}

void dense_apply(hb_ctx* c, const double2* s, double2* u, int nrhs, int adjoint, cudaStream_t st) {
  NvtxRange nr(adjoint ? "hb_apply_dense_adjoint" : "hb_apply_dense");
  EntryParams p = entry_params(c, adjoint);
  const double scale = c->h * c->h;
  // small grids give few output CTAs: split the source lines into shares so
  // that there are at least eight CTAs per SM (the entry evaluation is
  // latency-bound FP64 work)
  int dev = 0, nsm = 0;
  HB_CUDA(cudaGetDevice(&dev));
  HB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const long long cta = (long long)((p.nx + DT - 1) / DT) * p.ny;
  const int nsplit = (int)std::max<long long>(1, std::min<long long>(p.ny, (8LL * nsm + cta - 1) / cta));
  if (nsplit > 1) {
    const size_t need = (size_t)nsplit * 16 * (size_t)c->Nv;
    if (c->dense_part_cap < need) {
      dev_free(c->d_dense_part);
      c->d_dense_part = nullptr;
      c->dense_part_cap = 0;
      c->d_dense_part = dev_alloc<double2>(need);
      c->dense_part_cap = need;
    }
  }
  int r0 = 0;
  while (r0 < nrhs) {
    int left = nrhs - r0;
    int rc = left >= 16 ? 16 : left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1;
#define HB_DENSE_CASE(R)                                                              \
  case R:                                                                             \
    if (adjoint) launch_dense<R, true>(p, s, u, c->Nv, r0, scale, nsplit, c->d_dense_part, st); \
    else launch_dense<R, false>(p, s, u, c->Nv, r0, scale, nsplit, c->d_dense_part, st);       \
    break;
    switch (rc) {
      HB_DENSE_CASE(16)
      HB_DENSE_CASE(8)
      HB_DENSE_CASE(4)
      HB_DENSE_CASE(2)
      HB_DENSE_CASE(1)
    }
#undef HB_DENSE_CASE
    r0 += rc;
  }
}

// ------------------------------------------------------ block entries ----
// Work item = (block, one source column).  meta per block (int64 x 6):
//   row_off, m, col_off, n, out_off, seg_off;  nseg = number of row lines.
// Rows of a block are sorted by natural index, so rows of one grid line are
// contiguous; seg array (int64 x 3 per segment): b, first row, count.
// Output: column-major m x n at out_off; row a of the sorted list goes to
// out row rdst[row_off + a] (identity for the build).
constexpr int SEGC = 8;   // row lines per pass

__global__ void __launch_bounds__(128) block_entries_kernel(
    EntryParams p, const BlockMeta* __restrict__ meta, const long long* __restrict__ items,
    const long long* __restrict__ rows, const int* __restrict__ rdst, const long long* __restrict__ cols,
    const long long* __restrict__ segs, double2* __restrict__ out) {
  __shared__ double G[3][256];
  __shared__ double P[3][SEGC][MAX_NI];
  const int nI = p.nI, NI = p.NI;
  const long long it = items[blockIdx.x];
  const int b = (int)(it >> 20);
  const int jj = (int)(it & 0xFFFFF);
  const BlockMeta bm = meta[b];
  const long long qnat = cols[bm.col_off + jj];
  const int aq = (int)(qnat % p.nx), bq = (int)(qnat / p.nx);
  const int t = threadIdx.x;
  // G[q][i] = sum_j1 H[q][bq][i][j1] LX[aq][j1]
  for (int idx = t; idx < 3 * NI; idx += blockDim.x) {
    int q = idx / NI, i = idx % NI;
    const double* Hq = p.H + (((size_t)q * p.ny + bq) * NI + i) * nI;
    const double* lx = p.LX + (size_t)aq * nI;
    double a = 0.0;
    for (int j1 = 0; j1 < nI; ++j1) a = fma(Hq[j1], lx[j1], a);
    G[q][i] = a;
  }
  for (int s0 = 0; s0 < bm.nseg; s0 += SEGC) {
    const int ns = (int)min((long long)SEGC, bm.nseg - s0);
    __syncthreads();
    for (int idx = t; idx < 3 * ns * nI; idx += blockDim.x) {
      int q = idx / (ns * nI), sl = (idx / nI) % ns, i1 = idx % nI;
      int bo = (int)segs[(bm.seg_off + s0 + sl) * 3];
      const double* lz = p.LZ + (size_t)bo * nI;
      double a = 0.0;
      for (int i2 = 0; i2 < nI; ++i2) a = fma(lz[i2], G[q][i2 * nI + i1], a);
      P[q][sl][i1] = a;
    }
    __syncthreads();
    const long long rfirst = segs[(bm.seg_off + s0) * 3 + 1];
    const long long rlast = segs[(bm.seg_off + s0 + ns - 1) * 3 + 1] + segs[(bm.seg_off + s0 + ns - 1) * 3 + 2];
    for (long long r = rfirst + t; r < rlast; r += blockDim.x) {
      // locate the segment of row r (ns <= 8, linear scan)
      int sl = 0;
      while (sl + 1 < ns && segs[(bm.seg_off + s0 + sl + 1) * 3 + 1] <= r) ++sl;
      const long long onat = rows[bm.row_off + r];
      const int ao = (int)(onat % p.nx);
      const double* lx = p.LX + (size_t)ao * nI;
      double f[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        double a = 0.0;
        for (int i1 = 0; i1 < nI; ++i1) a = fma(lx[i1], P[q][sl][i1], a);
        f[q] = a;
      }
      double2 g = (onat == qnat) ? p.self[onat] : hb_green(f[0], f[1], f[2], p.omega);
      out[bm.out_off + (long long)jj * bm.m + rdst[bm.row_off + r]] = g;
    }
  }
}

// Host side: blocks given as natural-index lists (rows need not be sorted).
void add_block(BlockBatchHost& B, const hb_ctx* c, const long long* rows, long long m,
               const long long* cols, long long n, long long out_off) {
  BlockMeta bm{};
  bm.row_off = (long long)B.rows.size();
  bm.m = m;
  bm.col_off = (long long)B.cols.size();
  bm.n = n;
  bm.out_off = out_off;
  bm.seg_off = (long long)B.segs.size() / 3;
  std::vector<std::pair<long long, int>> order((size_t)m);
  for (long long a = 0; a < m; ++a) order[a] = {rows[a], (int)a};
  std::sort(order.begin(), order.end());
  long long nseg = 0;
  for (long long a = 0; a < m; ++a) {
    long long nat = order[a].first;
    B.rows.push_back(nat);
    B.rdst.push_back(order[a].second);
    long long line = nat / c->nx;
    if (a == 0 || line != order[a - 1].first / c->nx) {
      B.segs.push_back(line);
      B.segs.push_back(a);
      B.segs.push_back(0);
      ++nseg;
    }
    B.segs[B.segs.size() - 1] += 1;
  }
  bm.nseg = nseg;
  B.cols.insert(B.cols.end(), cols, cols + n);
  long long bidx = (long long)B.meta.size();
  for (long long j = 0; j < n; ++j) B.items.push_back((bidx << 20) | j);
  B.meta.push_back(bm);
}

namespace {
// Device scratch of one call, freed when the call returns or throws (after
// the stream has drained, so no launched kernel still reads it).
struct CallScratch {
  cudaStream_t st;
  std::vector<void*> p;
  template <class T>
  T* keep(T* q) {
    p.push_back(q);
    return q;
  }
  ~CallScratch() {
    cudaStreamSynchronize(st);
    for (void* q : p) dev_free(q);
  }
};
}  // namespace

void run_blocks(hb_ctx* c, BlockBatchHost& B, double2* d_out, cudaStream_t st) {
  if (B.items.empty()) return;
  CallScratch sc{st, {}};
  BlockMeta* d_meta = sc.keep(upload(B.meta, st));
  long long* d_items = sc.keep(upload(B.items, st));
  long long* d_rows = sc.keep(upload(B.rows, st));
  int* d_rdst = sc.keep(upload(B.rdst, st));
  long long* d_cols = sc.keep(upload(B.cols, st));
  long long* d_segs = sc.keep(upload(B.segs, st));
  EntryParams p = entry_params(c, 0);
  size_t nitems = B.items.size();
  for (size_t i0 = 0; i0 < nitems; i0 += 1u << 30) {
    unsigned cnt = (unsigned)std::min<size_t>(nitems - i0, 1u << 30);
    block_entries_kernel<<<cnt, 128, 0, st>>>(p, d_meta, d_items + i0, d_rows, d_rdst, d_cols, d_segs, d_out);
    HB_CHECK_LAUNCH();
  }
  HB_CUDA(cudaStreamSynchronize(st));
}

void eval_entries(hb_ctx* c, const long long* rows, int m, const long long* cols, int n, double2* out,
                  cudaStream_t st) {
  BlockBatchHost B;
  add_block(B, c, rows, m, cols, n, 0);
  run_blocks(c, B, out, st);
}

}  // namespace hb
