/* sweep.c - the oracle's table builder for media without closed forms:
 * Lax-Friedrichs WENO sweeping for the factored eikonal and the two
 * transport equations of the HB ingredients (Sec. 2.3, Eq. faceik,
 * Eq. equVs), initialised near the source by the Taylor expansions
 * (Eq. expansionT, Eq. expansionV0, Eq. expansionV1), then local cubic
 * interpolation from the mesh to the Chebyshev nodes (Sec. 4.1).
 *
 * TEST INFRASTRUCTURE ONLY (the oracle package): it writes the stored
 * tables that the CUDA path reads as input, and is called by nothing else.
 * Plain C99 + optional OpenMP over source nodes; FP64 throughout.
 *
 * Mesh: x_i = lo + i h0, z_j = lo + j h0, i, j = 0..M-1, field f[j M + i].
 * The three outermost rows and columns of the mesh (of the window, for the
 * transports) are linear extrapolations of the interior, refreshed after
 * every sweep; values past the edge (the WENO stencils) continue them
 * linearly, those of the central differences are cubic extrapolations.
 *
 * Factored eikonal (Eq. faceik): tau = tt * tb with tt = n0 |r - r0|,
 *   H(tb; p, q) = |tt (p, q) + tb grad tt| = n,  (p, q) = grad tb.
 * Lax-Friedrichs numerical Hamiltonian with WENO5 one-sided derivatives
 * p-, p+, q-, q+ and local viscosity alpha = tt (|dH/dp|, |dH/dq| <= tt):
 *   H_LF = H(tb; (p- + p+)/2, (q- + q+)/2) - alpha (p+ - p-)/2 - alpha (q+ - q-)/2,
 * Gauss-Seidel update tb <- tb + (n - H_LF) / (2 alpha / h0), sweeping the
 * four orderings of the mesh until the largest update of a pass of four
 * sweeps over the window (below) is below tol.  The mesh extends past the
 * unit square by a wide margin so that the outflow closure at the mesh
 * edge (below) does not reach the window.  Points within (P_T - 1) h0 of the source in both
 * coordinates keep their Taylor values (P_T = 6).
 *
 * Transport (Eq. equVs, d = 2), written in Cartesian form with
 * n^2 dv/dtau = grad tau . grad v = grad(tau^2) . grad v / (2 tau):
 *   s = -1:  2 grad(tau^2) . grad v0 + (Lap tau^2 - 4 n^2) v0 = 0,
 *   s =  0:  2 grad(tau^2) . grad v1 +  Lap tau^2        v1 = Lap v0.
 * Same Lax-Friedrichs WENO sweeping with alpha_x = 2 |d_x tau^2|,
 * alpha_z = 2 |d_z tau^2| (so the scheme is upwind in each direction), on
 * a window of the mesh (the unit square plus 14 cells a side), until the
 * largest update over the region of interest (the unit square and the two
 * extra points a side of the cubic interpolation stencils) is below tol;
 * fixed Taylor boxes of half-width (P_B - 1) h0
 * and (P_C - 1) h0 (P_B = 4, P_C = 2).  grad tau^2, Lap tau^2 and Lap v0
 * are fourth-order central differences on the mesh.
 *
 * Taylor input per source (polynomials in the offset (X, Z) = r - r0, a
 * homogeneous piece of degree k stored as k + 1 coefficients of
 * X^(k-m) Z^m): T_2..T_6 (25 numbers), B_0..B_4 (15), C_0..C_2 (6).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define P_T 6
#define P_B 4
#define P_C 2
#define TAYLOR_LEN 46   /* 25 + 15 + 6 */
#define WENO_EPS 1e-6

typedef struct {
  int M;
  double lo, h;
  int r0, r1;   /* a sub-range [r0, r1]^2 of the mesh (window / region of interest) */
} Mesh;

/* f at (i, j) with linear extrapolation in i (j inside the mesh) */
static inline double at_i(const double* f, int M, int i, int j) {
  const double* r = f + (size_t)j * M;
  if (i < 0) return r[0] + (double)i * (r[1] - r[0]);
  if (i >= M) return r[M - 1] + (double)(i - M + 1) * (r[M - 1] - r[M - 2]);
  return r[i];
}

/* f at (i, j) with linear extrapolation in j (i inside the mesh) */
static inline double at_j(const double* f, int M, int i, int j) {
  if (j < 0) return f[i] + (double)j * (f[(size_t)M + i] - f[i]);
  if (j >= M) {
    const double a = f[(size_t)(M - 1) * M + i], b = f[(size_t)(M - 2) * M + i];
    return a + (double)(j - M + 1) * (a - b);
  }
  return f[(size_t)j * M + i];
}

/* f at (i, j) with cubic extrapolation (exact for cubics) in i or in j:
 * used by the central differences, whose stencils reach two cells past
 * the mesh */
static inline double cub_i(const double* f, int M, int i, int j) {
  if (i >= 0 && i < M) return f[(size_t)j * M + i];
  const int s = i < 0 ? 1 : -1, e = i < 0 ? 0 : M - 1;
  const double t = (double)(i < 0 ? -i : i - M + 1);   /* cells past the edge */
  double v = 0.0;
  for (int a = 0; a < 4; ++a) {                        /* Lagrange on edge + a s */
    double w = 1.0;
    for (int b = 0; b < 4; ++b)
      if (b != a) w *= (-t - b) / (double)(a - b);
    v += w * f[(size_t)j * M + e + a * s];
  }
  return v;
}

static inline double cub_j(const double* f, int M, int i, int j) {
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

/* WENO5 combination of the five divided differences (Jiang-Peng weights);
 * *k = 11/6 w1 + 1/2 w2 - 1/2 w3, the weight of v3 minus that of v4 in the
 * result at the current weights */
static double weno5(double v1, double v2, double v3, double v4, double v5, double* k) {
  const double p1 = v1 / 3.0 - 7.0 * v2 / 6.0 + 11.0 * v3 / 6.0;
  const double p2 = -v2 / 6.0 + 5.0 * v3 / 6.0 + v4 / 3.0;
  const double p3 = v3 / 3.0 + 5.0 * v4 / 6.0 - v5 / 6.0;
  const double e1 = v1 - 2.0 * v2 + v3, f1 = v1 - 4.0 * v2 + 3.0 * v3;
  const double e2 = v2 - 2.0 * v3 + v4, f2 = v2 - v4;
  const double e3 = v3 - 2.0 * v4 + v5, f3 = 3.0 * v3 - 4.0 * v4 + v5;
  const double s1 = 13.0 / 12.0 * e1 * e1 + 0.25 * f1 * f1;
  const double s2 = 13.0 / 12.0 * e2 * e2 + 0.25 * f2 * f2;
  const double s3 = 13.0 / 12.0 * e3 * e3 + 0.25 * f3 * f3;
  const double a1 = 0.1 / ((WENO_EPS + s1) * (WENO_EPS + s1));
  const double a2 = 0.6 / ((WENO_EPS + s2) * (WENO_EPS + s2));
  const double a3 = 0.3 / ((WENO_EPS + s3) * (WENO_EPS + s3));
  const double sum = a1 + a2 + a3;
  *k = (11.0 / 6.0 * a1 + 0.5 * a2 - 0.5 * a3) / sum;
  return (a1 * p1 + a2 * p2 + a3 * p3) / sum;
}

/* One-sided WENO5 derivatives d- and d+ from the seven values u[0..6]
 * centred on u[3], spacing h, and k- = h d(d-)/du[3], k+ = -h d(d+)/du[3]
 * at the current weights. */
static inline void weno_pair(const double* u, double h, double* dm, double* dp, double* km, double* kp) {
  double d[6];
  for (int k = 0; k < 6; ++k) d[k] = (u[k + 1] - u[k]) / h;   /* d[k] = D+ u[k] */
  *dm = weno5(d[0], d[1], d[2], d[3], d[4], km);
  *dp = weno5(d[5], d[4], d[3], d[2], d[1], kp);
}

/* WENO derivatives p-, p+ (x) and q-, q+ (z) at (i, j), with the k's of
 * weno_pair in kk[0..3] = (k of p-, k of p+, k of q-, k of q+) */
static inline void derivs(const double* f, int M, int i, int j, double h, double* pm, double* pp, double* qm,
                          double* qp, double* kk) {
  double u[7];
  for (int k = 0; k < 7; ++k) u[k] = at_i(f, M, i - 3 + k, j);
  weno_pair(u, h, pm, pp, &kk[0], &kk[1]);
  for (int k = 0; k < 7; ++k) u[k] = at_j(f, M, i, j - 3 + k);
  weno_pair(u, h, qm, qp, &kk[2], &kk[3]);
}

/* homogeneous polynomial of degree k (k + 1 coefficients) at (X, Z) */
static double hpoly(const double* c, int k, double X, double Z) {
  double s = 0.0;
  for (int m = 0; m <= k; ++m) s += c[m] * pow(X, k - m) * pow(Z, m);
  return s;
}

static double taylor_sum(const double* c, int k0, int k1, double X, double Z) {
  double s = 0.0;
  for (int k = k0; k <= k1; ++k) {
    s += hpoly(c, k, X, Z);
    c += k + 1;
  }
  return s;
}

/* The three outermost rows and columns of the mesh are not updated by the
 * scheme: after every sweep they are linear extrapolations, along the mesh
 * lines, of the two nearest updated values (an outflow closure: the mesh
 * edge only receives characteristics).  Fixed (Taylor) points keep their
 * values. */
#define EDGE 3
static void extrapolate_edges(double* f, const unsigned char* fixed, int M) {
  for (int j = 0; j < M; ++j) {
    double* r = f + (size_t)j * M;
    for (int i = 0; i < EDGE; ++i) {
      const int t = EDGE - i;
      if (!fixed[(size_t)j * M + i]) r[i] = r[EDGE] + t * (r[EDGE] - r[EDGE + 1]);
      const int k = M - 1 - i;
      if (!fixed[(size_t)j * M + k]) r[k] = r[M - 1 - EDGE] + t * (r[M - 1 - EDGE] - r[M - 2 - EDGE]);
    }
  }
  for (int j = 0; j < EDGE; ++j) {
    const int t = EDGE - j;
    for (int i = 0; i < M; ++i) {
      const size_t p = (size_t)j * M + i, q = (size_t)(M - 1 - j) * M + i;
      if (!fixed[p]) f[p] = f[(size_t)EDGE * M + i] + t * (f[(size_t)EDGE * M + i] - f[(size_t)(EDGE + 1) * M + i]);
      if (!fixed[q])
        f[q] = f[(size_t)(M - 1 - EDGE) * M + i] +
               t * (f[(size_t)(M - 1 - EDGE) * M + i] - f[(size_t)(M - 2 - EDGE) * M + i]);
    }
  }
}

static inline int in_roi(const Mesh* g, int i, int j) {
  return i >= g->r0 && i <= g->r1 && j >= g->r0 && j <= g->r1;
}

static inline int on_edge(int i, int j, int M) {
  return i < EDGE || j < EDGE || i >= M - EDGE || j >= M - EDGE;
}

/* Visit the mesh in sweep order o (0..3).  Rows one after the other
 * (lexicographic Gauss-Seidel, the default), or anti-diagonals ii + jj = dd
 * one after the other (g_wavefront != 0).  An update reads its row and its
 * column only, so the points of one anti-diagonal never read each other and
 * may be updated in any order (the order a parallel sweep takes); and along
 * every row and column both orders visit the points in the same upwind
 * order, so each update sees the same new and old values: the two orders
 * compute the same iterates bit for bit. */
static int g_wavefront = 0;

#define SWEEP_BEGIN(o, M)                                                          \
  for (int dd = 0; dd < (g_wavefront ? 2 * (M) - 1 : (M)); ++dd) {                 \
    const int ilo = g_wavefront ? (dd - (M) + 1 > 0 ? dd - (M) + 1 : 0) : 0;       \
    const int ihi = g_wavefront ? (dd < (M) - 1 ? dd : (M) - 1) : (M) - 1;         \
    for (int ii = ilo; ii <= ihi; ++ii) {                                          \
      const int jj = g_wavefront ? dd - ii : dd;                                   \
      const int j = ((o) & 2) ? (M) - 1 - jj : jj;                                 \
      const int i = (((o) == 1) || ((o) == 2)) ? (M) - 1 - ii : ii;                \
      const size_t p = (size_t)j * (M) + i;
#define SWEEP_END \
  }               \
  }

/* 4th-order central first and second differences (cubic extrapolation
 * past the mesh edge) */
static void central_diffs(const double* f, int M, double h, double* fx, double* fz, double* lap) {
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i) {
      const double xm2 = cub_i(f, M, i - 2, j), xm1 = cub_i(f, M, i - 1, j), x0 = f[(size_t)j * M + i];
      const double xp1 = cub_i(f, M, i + 1, j), xp2 = cub_i(f, M, i + 2, j);
      const double zm2 = cub_j(f, M, i, j - 2), zm1 = cub_j(f, M, i, j - 1);
      const double zp1 = cub_j(f, M, i, j + 1), zp2 = cub_j(f, M, i, j + 2);
      const size_t p = (size_t)j * M + i;
      if (fx) fx[p] = (-xp2 + 8.0 * xp1 - 8.0 * xm1 + xm2) / (12.0 * h);
      if (fz) fz[p] = (-zp2 + 8.0 * zp1 - 8.0 * zm1 + zm2) / (12.0 * h);
      if (lap)
        lap[p] = ((-xp2 + 16.0 * xp1 - 30.0 * x0 + 16.0 * xm1 - xm2) +
                  (-zp2 + 16.0 * zp1 - 30.0 * x0 + 16.0 * zm1 - zm2)) /
                 (12.0 * h * h);
    }
}

typedef struct {
  int iters[3];
  double last[3];
} SolveInfo;

/* One source node.  The factored eikonal runs on the mesh g until the
 * largest update of a pass over g's window [r0, r1]^2 is below tol; the
 * window is the sub-mesh w (M_w = r1 - r0 + 1) on which the transports run,
 * until the largest update over w's region of interest [w.r0, w.r1]^2 is
 * below tol.  Out: tau2 on g (M x M), v0 and v1 on w (M_w x M_w).
 * Returns 0, or -1 when out of memory. */
static int solve_source(const Mesh* g, const Mesh* w, const double* n, double x0, double z0, const double* taylor,
                        int max_iter, double tol, double* tau2, double* v0, double* v1, SolveInfo* info) {
  const int M = g->M, Mw = w->M, off = g->r0;
  const size_t N = (size_t)M * M, Nw = (size_t)Mw * Mw;
  const double h = g->h;
  const double* T = taylor;          /* T_2..T_6 */
  const double* B = taylor + 25;     /* B_0..B_4 */
  const double* C = taylor + 40;     /* C_0..C_2 */
  const double n0 = sqrt(T[0]);      /* T_2 = S0 (X^2 + Z^2), S0 = n0^2 */
  double* buf = (double*)malloc((4 * N + 5 * Nw) * sizeof(double));
  unsigned char* fixed = (unsigned char*)malloc(N);
  if (!buf || !fixed) {
    free(buf);
    free(fixed);
    return -1;
  }
  double* tb = buf;                  /* factored unknown */
  double* tt = buf + N;              /* n0 |r - r0| */
  double* gx = buf + 2 * N;          /* grad tt = n0 (r - r0) / |r - r0| */
  double* gz = buf + 3 * N;
  double* ax = buf + 4 * N;          /* on the window: d_x tau^2 */
  double* az = ax + Nw;              /* d_z tau^2 */
  double* lt = az + Nw;              /* Lap tau^2 */
  double* nw = lt + Nw;              /* n */
  double* rhs = nw + Nw;             /* Lap v0 */

  /* ---- factored eikonal on g ---- */
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i) {
      const size_t p = (size_t)j * M + i;
      const double X = g->lo + i * h - x0, Z = g->lo + j * h - z0;
      const double rho = sqrt(X * X + Z * Z);
      tt[p] = n0 * rho;
      gx[p] = rho > 0 ? n0 * X / rho : 0.0;
      gz[p] = rho > 0 ? n0 * Z / rho : 0.0;
      fixed[p] = fabs(X) <= (P_T - 1) * h * (1 + 1e-12) && fabs(Z) <= (P_T - 1) * h * (1 + 1e-12);
      if (fixed[p]) {
        const double t2 = taylor_sum(T, 2, P_T, X, Z);
        tb[p] = rho > 0 ? sqrt(t2 > 0 ? t2 : 0.0) / (n0 * rho) : 1.0;
      } else {
        tb[p] = 1.0;
      }
    }
  int it;
  double last = 0.0;
  for (it = 0; it < max_iter; ++it) {
    last = 0.0;
    for (int o = 0; o < 4; ++o) {
      SWEEP_BEGIN(o, M)
      if (fixed[p] || on_edge(i, j, M)) continue;
      double pm, pp, qm, qp, kk[4];
      derivs(tb, M, i, j, h, &pm, &pp, &qm, &qp, kk);
      const double a = tt[p] * 0.5 * (pm + pp) + tb[p] * gx[p];
      const double b = tt[p] * 0.5 * (qm + qp) + tb[p] * gz[p];
      const double H = sqrt(a * a + b * b);
      const double alpha = tt[p];
      const double hlf = H - alpha * 0.5 * (pp - pm) - alpha * 0.5 * (qp - qm);
      /* divide by the first-order coefficient of tb here in hlf, 2 alpha / h,
       * or by its coefficient at the current WENO weights where that is
       * larger (a full step would then overshoot) */
      const double dH = H > 0 ? (a * (tt[p] * 0.5 * (kk[0] - kk[1]) / h + gx[p]) +
                                 b * (tt[p] * 0.5 * (kk[2] - kk[3]) / h + gz[p])) / H
                              : 0.0;
      const double kw = dH + alpha * 0.5 * (kk[0] + kk[1] + kk[2] + kk[3]) / h;
      const double d = (n[p] - hlf) / fmax(2.0 * alpha / h, kw);
      tb[p] += d;
      if (fabs(d) > last && in_roi(g, i, j)) last = fabs(d);
      SWEEP_END
      extrapolate_edges(tb, fixed, M);
    }
    if (last < tol) break;
  }
  info->iters[0] = it;
  info->last[0] = last;
  for (int j = 0; j < M; ++j)
    for (int i = 0; i < M; ++i) {
      const size_t p = (size_t)j * M + i;
      const double X = g->lo + i * h - x0, Z = g->lo + j * h - z0;
      tau2[p] = fixed[p] ? taylor_sum(T, 2, P_T, X, Z) : (tt[p] * tb[p]) * (tt[p] * tb[p]);
    }
  /* derivatives of tau^2 on g (true neighbours at the window edge), kept on w */
  central_diffs(tau2, M, h, tb, tt, gx);
  for (int j = 0; j < Mw; ++j)
    for (int i = 0; i < Mw; ++i) {
      const size_t q = (size_t)j * Mw + i, p = (size_t)(j + off) * M + i + off;
      ax[q] = tb[p];
      az[q] = tt[p];
      lt[q] = gx[p];
      nw[q] = n[p];
    }

  /* ---- transport on w: s = -1 (v0) then s = 0 (v1) ---- */
  for (int s = 0; s < 2; ++s) {
    double* v = s == 0 ? v0 : v1;
    const int P = s == 0 ? P_B : P_C;
    if (s == 1) central_diffs(v0, Mw, h, NULL, NULL, rhs);
    for (int j = 0; j < Mw; ++j)
      for (int i = 0; i < Mw; ++i) {
        const size_t p = (size_t)j * Mw + i;
        const double X = w->lo + i * h - x0, Z = w->lo + j * h - z0;
        fixed[p] = fabs(X) <= (P - 1) * h * (1 + 1e-12) && fabs(Z) <= (P - 1) * h * (1 + 1e-12);
        if (fixed[p]) v[p] = s == 0 ? taylor_sum(B, 0, P_B, X, Z) : taylor_sum(C, 0, P_C, X, Z);
        else v[p] = s == 0 ? B[0] : C[0];
      }
    for (it = 0; it < max_iter; ++it) {
      last = 0.0;
      for (int o = 0; o < 4; ++o) {
        SWEEP_BEGIN(o, Mw)
        if (fixed[p] || on_edge(i, j, Mw)) continue;
        double pm, pp, qm, qp, kk[4];
        derivs(v, Mw, i, j, h, &pm, &pp, &qm, &qp, kk);
        const double c = s == 0 ? lt[p] - 4.0 * nw[p] * nw[p] : lt[p];
        const double f = s == 0 ? 0.0 : rhs[p];
        const double alx = 2.0 * fabs(ax[p]), alz = 2.0 * fabs(az[p]);
        const double hlf = ax[p] * (pm + pp) + az[p] * (qm + qp) + c * v[p] - alx * 0.5 * (pp - pm) -
                           alz * 0.5 * (qp - qm);
        /* divide by the first-order coefficient of v here in hlf (c v is not
         * lagged: next to the source that would not contract), or by its
         * coefficient at the current WENO weights where that is larger */
        const double den = (alx + alz) / h + c;
        if (!(den > 0.25 * (alx + alz) / h)) continue;
        const double kw = (ax[p] * (kk[0] - kk[1]) + az[p] * (kk[2] - kk[3]) +
                           0.5 * alx * (kk[0] + kk[1]) + 0.5 * alz * (kk[2] + kk[3])) / h + c;
        const double d = (f - hlf) / fmax(den, kw);
        v[p] += d;
        if (fabs(d) > last && in_roi(w, i, j)) last = fabs(d);
        SWEEP_END
        extrapolate_edges(v, fixed, Mw);
      }
      if (last < tol) break;
    }
    info->iters[1 + s] = it;
    info->last[1 + s] = last;
  }
  free(buf);
  free(fixed);
  return 0;
}

/* local cubic (4 x 4 Lagrange) interpolation of f at (x, z) */
static double cubic_at(const Mesh* g, const double* f, double x, double z) {
  const int M = g->M;
  const double sx = (x - g->lo) / g->h, sz = (z - g->lo) / g->h;
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

/* The window mesh of g: rows and columns r0..r1 of g, with its region of
 * interest at [roi0, roi1] of its own indices. */
static Mesh window_of(const Mesh* g, int roi0, int roi1) {
  const Mesh w = {g->r1 - g->r0 + 1, g->lo + g->r0 * g->h, g->h, roi0, roi1};
  return w;
}

static int check_mesh(int M, double h, int w0, int w1, int roi0, int roi1) {
  return M >= 8 && h > 0 && w0 >= 0 && w1 < M && w1 - w0 + 1 >= 8 && roi0 >= 0 && roi1 <= w1 - w0 && roi0 <= roi1;
}

/* Tables for the source nodes src[0..ns-1] (indices into the NI points
 * (px, pz)): column k of tau2/v0/v1 (NI x ns, row-major: [obs][k]) holds
 * the ingredients at every observation point.  Mesh: M x M points
 * x_i = lo + i h; the transports run on its window [w0, w1]^2, whose region
 * of interest is [roi0, roi1]^2 in window indices.  taylor is
 * ns x TAYLOR_LEN; n_mesh is n on the mesh (M x M).  info: ns x 6
 * (iterations and last updates of the three solves).  Returns 0, or -1 on
 * a bad argument or when out of memory. */
/* 0: row-by-row sweeps (default); 1: anti-diagonal (wavefront) sweeps.
 * Set before a call, not during one. */
void hb_oracle_sweep_set_order(int wavefront) { g_wavefront = wavefront != 0; }

/* The visiting order of sweep o on an M x M mesh under the current order
 * setting: out[k] = the k-th point visited (j M + i). */
void hb_oracle_sweep_visit_order(int o, int M, long long* out) {
  long long k = 0;
  SWEEP_BEGIN(o, M)
  out[k++] = (long long)p;
  SWEEP_END
}

int hb_oracle_sweep_tables(int M, double lo, double h, int w0, int w1, int roi0, int roi1, const double* n_mesh,
                           int NI, const double* px, const double* pz, int ns, const int* src, const double* taylor,
                           int max_iter, double tol, double* tau2, double* v0, double* v1, double* info) {
  if (!check_mesh(M, h, w0, w1, roi0, roi1) || NI < 1 || ns < 0) return -1;
  const Mesh g = {M, lo, h, w0, w1};
  const Mesh w = window_of(&g, roi0, roi1);
  const size_t N = (size_t)M * M, Nw = (size_t)w.M * w.M;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int k = 0; k < ns; ++k) {
    double* out = (double*)malloc((N + 2 * Nw) * sizeof(double));
    SolveInfo si;
    const int j = src[k];
    if (!out || solve_source(&g, &w, n_mesh, px[j], pz[j], taylor + (size_t)k * TAYLOR_LEN, max_iter, tol, out,
                             out + N, out + N + Nw, &si) != 0) {
      free(out);
      bad |= 1;
      continue;
    }
    for (int i = 0; i < NI; ++i) {
      tau2[(size_t)i * ns + k] = cubic_at(&g, out, px[i], pz[i]);
      v0[(size_t)i * ns + k] = cubic_at(&w, out + N, px[i], pz[i]);
      v1[(size_t)i * ns + k] = cubic_at(&w, out + N + Nw, px[i], pz[i]);
    }
    for (int q = 0; q < 3; ++q) {
      info[(size_t)k * 6 + q] = si.iters[q];
      info[(size_t)k * 6 + 3 + q] = si.last[q];
    }
    free(out);
  }
  return bad ? -1 : 0;
}

/* The mesh fields of one source at (x0, z0): tau2 on the mesh (M x M), v0
 * and v1 on the window ((w1 - w0 + 1)^2), arguments as above. */
int hb_oracle_sweep_fields(int M, double lo, double h, int w0, int w1, int roi0, int roi1, const double* n_mesh,
                           double x0, double z0, const double* taylor, int max_iter, double tol, double* tau2,
                           double* v0, double* v1, double* info) {
  if (!check_mesh(M, h, w0, w1, roi0, roi1)) return -1;
  const Mesh g = {M, lo, h, w0, w1};
  const Mesh w = window_of(&g, roi0, roi1);
  SolveInfo si;
  if (solve_source(&g, &w, n_mesh, x0, z0, taylor, max_iter, tol, tau2, v0, v1, &si) != 0) return -1;
  for (int q = 0; q < 3; ++q) {
    info[q] = si.iters[q];
    info[3 + q] = si.last[q];
  }
  return 0;
}
