// cpqr.cu - batched interpolative decomposition by column-pivoted
// Householder QR, FP64 complex (Sec. 4.2.1, Eq. ID, Eq. proxy).
//
// For each matrix A (m x n, column-major), K(tau_hat, cols) ~ K(tau_hat,
// skel) V with skel the first r pivots and V = [I | R11^-1 R12] P^T:
//  * step k: the trailing column norms over rows >= k are recomputed (fused
//    into the previous step's update, no downdating); the pivot is the
//    lowest position whose norm is at least the largest minus ID_TIE |R_00|
//    (the largest times 1 - ID_TIE at step 0): columns that are mirror
//    images on the grid have norms equal up to rounding, and the window makes
//    the choice among them independent of how the norms were rounded;
//  * the rank is the first k >= 1 with |R_kk| <= eps |R_00| (k = min(m, n)
//    otherwise); an all-zero matrix gets rank 1 with V = e_0^T;
//  * the reflector for column k is H = I - (2/v^H v) v v^H with
//    v = x + e^{i arg x_0} |x| e_0, so R_kk = -e^{i arg x_0} |x|; v is kept in
//    place below the diagonal.
// Outputs: the rank, the full pivot order (first r = skeleton) and, in place
// of R12, T = R11^-1 R12 (rows < r of the columns at pivot positions >= r);
// emit_v_kernel assembles V from them.
// One CTA of 256 threads per matrix, one warp per column; every reduction
// runs in a fixed order (lane-strided partial sums, then an xor-shuffle
// tree), so results are bitwise reproducible run to run.
#include <cuda_runtime.h>

#include "hb_internal.cuh"

namespace hb {

constexpr int ID_THREADS = 256;
constexpr int ID_WARPS = ID_THREADS / 32;
constexpr double ID_TIE = 1e-12;   // pivot tie window, relative to |R_00|

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(ID_THREADS) id_kernel(const int* __restrict__ M, const int* __restrict__ N,
                                                        const long long* __restrict__ aoff, double2* A,
                                                        double eps, int* __restrict__ rank_out,
                                                        int* __restrict__ perm_out,
                                                        const long long* __restrict__ soff) {
  extern __shared__ unsigned char sm_raw[];
  const int b = blockIdx.x;
  const int m = M[b], n = N[b];
  double2* a = A + aoff[b];
  double2* rd = reinterpret_cast<double2*>(sm_raw);         // n   R_kk (16-byte aligned first)
  double* nrm = reinterpret_cast<double*>(rd + n);          // n
  int* perm = reinterpret_cast<int*>(nrm + n);              // n
  __shared__ int s_piv, s_rank, s_stop;
  __shared__ double s_r00, s_scale;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < n; j += ID_THREADS) perm[j] = j;
  // initial column norms over all rows
  for (int j = warp; j < n; j += ID_WARPS) {
    const double2* col = a + (size_t)j * m;
    double s = 0.0;
    for (int i = lane; i < m; i += 32) s = fma(col[i].x, col[i].x, fma(col[i].y, col[i].y, s));
    s = warp_sum(s);
    if (lane == 0) nrm[j] = sqrt(s);
  }
  if (threadIdx.x == 0) {
    s_rank = min(m, n);
    s_stop = 0;
  }
  __syncthreads();
  const int kmax = min(m, n);
  for (int k = 0; k < kmax; ++k) {
    if (warp == 0) {
      // the largest trailing norm, then the lowest position inside the tie
      // window (both reductions are exact, so their order does not matter)
      double top = 0.0;
      for (int j = k + lane; j < n; j += 32) top = fmax(top, nrm[j]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) top = fmax(top, __shfl_xor_sync(0xffffffffu, top, o));
      const double thr = (k == 0) ? top * (1.0 - ID_TIE) : top - ID_TIE * s_r00;
      int p = n;
      for (int j = k + lane; j < n; j += 32)
        if (nrm[j] >= thr) {
          p = j;
          break;
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) p = min(p, __shfl_xor_sync(0xffffffffu, p, o));
      if (lane == 0) {
        s_piv = p;
        if (k == 0) {
          s_r00 = nrm[p];
          if (top == 0.0) { s_rank = 1; s_stop = 2; }
        } else if (top <= eps * s_r00) {
          s_rank = k;
          s_stop = 1;
        }
        if (!s_stop && p != k) {
          double t = nrm[k]; nrm[k] = nrm[p]; nrm[p] = t;
          int q = perm[k]; perm[k] = perm[p]; perm[p] = q;
        }
      }
    }
    __syncthreads();
    if (s_stop) break;
    const int p = s_piv;
    if (p != k) {
      double2* ck = a + (size_t)k * m;
      double2* cp = a + (size_t)p * m;
      for (int i = threadIdx.x; i < m; i += ID_THREADS) {
        double2 t = ck[i]; ck[i] = cp[i]; cp[i] = t;
      }
      __syncthreads();
    }
    // Householder vector in column k, rows k..m-1
    double2* ck = a + (size_t)k * m;
    if (threadIdx.x == 0) {
      const double alpha = nrm[k];
      const double2 x0 = ck[k];
      const double ax0 = hypot(x0.x, x0.y);
      double2 ph = (ax0 > 0.0) ? make_double2(x0.x / ax0, x0.y / ax0) : make_double2(1.0, 0.0);
      double2 v0 = make_double2(x0.x + ph.x * alpha, x0.y + ph.y * alpha);
      const double vv = alpha * alpha - ax0 * ax0 + (v0.x * v0.x + v0.y * v0.y);
      s_scale = (vv > 0.0) ? 2.0 / vv : 0.0;
      rd[k] = make_double2(-ph.x * alpha, -ph.y * alpha);
      ck[k] = v0;
    }
    __syncthreads();
    const double sc = s_scale;
    // apply to trailing columns and recompute their norms over rows k+1..m-1
    for (int j = k + 1 + warp; j < n; j += ID_WARPS) {
      double2* cj = a + (size_t)j * m;
      double wr = 0.0, wi = 0.0;
      for (int i = k + lane; i < m; i += 32) {
        const double2 v = ck[i], x = cj[i];
        wr = fma(v.x, x.x, fma(v.y, x.y, wr));        // conj(v) x
        wi = fma(v.x, x.y, fma(-v.y, x.x, wi));
      }
      wr = warp_sum(wr) * sc;
      wi = warp_sum(wi) * sc;
      double s = 0.0;
      for (int i = k + lane; i < m; i += 32) {
        const double2 v = ck[i];
        double2 x = cj[i];
        x.x -= wr * v.x - wi * v.y;
        x.y -= wr * v.y + wi * v.x;
        cj[i] = x;
        if (i > k) s = fma(x.x, x.x, fma(x.y, x.y, s));
      }
      s = warp_sum(s);
      if (lane == 0) nrm[j] = sqrt(s);
    }
    __syncthreads();
  }
  __syncthreads();
  const int r = s_rank;
  const bool zero = (s_stop == 2);
  // T = R11^-1 R12, one warp per column of R12; R11 diagonal from rd, strict
  // upper part in place; the result overwrites R12.
  if (!zero) {
    for (int j = r + warp; j < n; j += ID_WARPS) {
      double2* cj = a + (size_t)j * m;
      for (int i = r - 1; i >= 0; --i) {
        double sr = 0.0, si = 0.0;
        for (int l = i + 1 + lane; l < r; l += 32) {
          const double2 R = a[(size_t)l * m + i], t = cj[l];
          sr = fma(R.x, t.x, fma(-R.y, t.y, sr));
          si = fma(R.x, t.y, fma(R.y, t.x, si));
        }
        sr = warp_sum(sr);
        si = warp_sum(si);
        if (lane == 0) {
          const double2 num = make_double2(cj[i].x - sr, cj[i].y - si);
          const double2 d = rd[i];
          const double dd = d.x * d.x + d.y * d.y;
          cj[i] = make_double2((num.x * d.x + num.y * d.y) / dd, (num.y * d.x - num.x * d.y) / dd);
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
  int* pm = perm_out + soff[b];
  for (int j = threadIdx.x; j < n; j += ID_THREADS) pm[j] = perm[j];
  if (threadIdx.x == 0) rank_out[b] = r;
}

// V[k][perm[j]] = (j < r) ? delta_kj : T[k][j]; V column-major with leading
// dimension ld = (ld_is_rank ? r : n) at element offset voff[b].
__global__ void emit_v_kernel(const int* __restrict__ M, const int* __restrict__ N,
                              const long long* __restrict__ aoff, const double2* __restrict__ A,
                              const int* __restrict__ rank, const int* __restrict__ perm,
                              const long long* __restrict__ soff, const long long* __restrict__ voff,
                              int ld_is_rank, double2* __restrict__ V64, float2* __restrict__ V32) {
  const int b = blockIdx.x;
  const int m = M[b], n = N[b], r = rank[b];
  const int ld = ld_is_rank ? r : n;
  const double2* a = A + aoff[b];
  const int* pm = perm + soff[b];
  for (int idx = threadIdx.x; idx < r * n; idx += blockDim.x) {
    const int j = idx / r, kk = idx % r;
    // an all-zero input never ran a reflection, so its T entries read as 0
    double2 val = (j < r) ? make_double2(j == kk ? 1.0 : 0.0, 0.0) : a[(size_t)j * m + kk];
    const size_t o = voff[b] + (size_t)pm[j] * ld + kk;
    if (V64) V64[o] = val;
    if (V32) V32[o] = make_float2((float)val.x, (float)val.y);
  }
}

void id_batch(int count, const int* d_m, const int* d_n, const long long* d_aoff, double2* d_A, double eps,
              int* d_rank, int* d_perm, const long long* d_soff, int max_n, cudaStream_t st) {
  if (count == 0) return;
  size_t sm = (size_t)max_n * (sizeof(double) + sizeof(double2) + sizeof(int));
  HB_CUDA(cudaFuncSetAttribute(id_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(sm, 1)));
  for (int b0 = 0; b0 < count; b0 += 1 << 30) {
    int cnt = std::min(count - b0, 1 << 30);
    id_kernel<<<cnt, ID_THREADS, sm, st>>>(d_m + b0, d_n + b0, d_aoff + b0, d_A, eps, d_rank + b0, d_perm,
                                           d_soff + b0);
    HB_CHECK_LAUNCH();
  }
}

void emit_v(int count, const int* d_m, const int* d_n, const long long* d_aoff, const double2* d_A,
            const int* d_rank, const int* d_perm, const long long* d_soff, const long long* d_voff,
            int ld_is_rank, double2* V64, float2* V32, cudaStream_t st) {
  for (int b0 = 0; b0 < count; b0 += 1 << 30) {
    int cnt = std::min(count - b0, 1 << 30);
    emit_v_kernel<<<cnt, 128, 0, st>>>(d_m + b0, d_n + b0, d_aoff + b0, d_A, d_rank + b0, d_perm,
                                       d_soff + b0, d_voff + b0, ld_is_rank, V64, V32);
    HB_CHECK_LAUNCH();
  }
}

}  // namespace hb

// ---------------------------------------------------------------------------
// hb_id_batch_noalloc: the same batched decompositions without allocating.
//
// Some callers cannot call cudaMalloc: code running under another
// framework's memory manager (which has reserved the device memory for its
// own pool, so a raw cudaMalloc can fail even though memory is free in that
// pool, or would stall every stream with its implicit synchronisation), and
// latency-critical paths that must not take that synchronisation.  For them
// the per-matrix metadata the kernels read from device memory (sizes and
// offsets) lives in this file-scope array instead of a fresh allocation.
// Every GPU that loads the library holds the array until the process exits.
// The pivot order goes straight into the caller's skel buffer, so nothing
// else is needed.  Every call overwrites the metadata it reads, so nothing
// has to start at zero; calls that overlap on the GPU (different streams or
// host threads without a synchronisation between them) race on the array.
//
// The caller's host arrays m, n, a_off are first copied into a file-scope
// host array (ordinary pageable memory, under a mutex) and the device copies
// read that array.  A copy from pageable memory has consumed its source when
// cudaMemcpyAsync returns, so the caller may reuse its arrays on return even
// when they are page-locked (a copy straight from page-locked memory would
// read them only when the stream reaches it).
#include <cstring>
#include <mutex>

namespace hb {

constexpr int ID_NOALLOC_MAX = 65536;                       // matrices per call
constexpr size_t ID_NOALLOC_BYTES = (size_t)ID_NOALLOC_MAX * 32;   // 2 MiB

static __device__ __align__(256) unsigned char g_id_noalloc_scratch[ID_NOALLOC_BYTES];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {};   // device address of the array, per device ordinal
// host staging of the metadata (pageable; guarded by g_noalloc_mu)
alignas(256) unsigned char g_noalloc_host[(size_t)ID_NOALLOC_MAX * 16];

// Set-up, once per device, with that device current: look up the device
// address of the array (its name in host code is only a host-side stand-in).
// The caller holds g_noalloc_mu.
void* noalloc_scratch() {
  int dev = 0;
  HB_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) throw Error{HB_ERR_UNSUPPORTED, "device ordinal above 255"};
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_id_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      throw Error{HB_ERR_CUDA, std::string("cudaGetSymbolAddress(id scratch): ") + cudaGetErrorString(e)};
    }
    g_noalloc_addr[dev] = p;
  }
  return g_noalloc_addr[dev];
}

// s_off[b] = sum_{c<b} n[c], v_off[b] = sum_{c<b} n[c]^2 (one CTA, chunked scan)
__global__ void __launch_bounds__(1024) noalloc_offsets_kernel(const int* __restrict__ n, int count,
                                                                long long* __restrict__ s_off,
                                                                long long* __restrict__ v_off) {
  __shared__ long long ts[1024], tv[1024];
  const int chunk = (count + 1023) / 1024;
  const int b0 = min(count, (int)threadIdx.x * chunk), b1 = min(count, b0 + chunk);
  long long as = 0, av = 0;
  for (int b = b0; b < b1; ++b) {
    as += n[b];
    av += (long long)n[b] * n[b];
  }
  ts[threadIdx.x] = as;
  tv[threadIdx.x] = av;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long rs = 0, rv = 0;
    for (int i = 0; i < 1024; ++i) {
      const long long a = ts[i], v = tv[i];
      ts[i] = rs;
      tv[i] = rv;
      rs += a;
      rv += v;
    }
  }
  __syncthreads();
  as = ts[threadIdx.x];
  av = tv[threadIdx.x];
  for (int b = b0; b < b1; ++b) {
    s_off[b] = as;
    v_off[b] = av;
    as += n[b];
    av += (long long)n[b] * n[b];
  }
}
}  // namespace

void id_batch_noalloc(int count, const int* m, const int* n, const long long* a_off, double2* A, double eps,
                      int* rank, int* skel, double2* V, cudaStream_t st) {
  if (count > ID_NOALLOC_MAX)
    throw arg_error("hb_id_batch_noalloc: count=%d exceeds the static scratch limit of %d matrices", count,
                    ID_NOALLOC_MAX);
  int max_n = 1;
  for (int b = 0; b < count; ++b) {
    if (m[b] < 1 || n[b] < 1) throw arg_error("matrix %d has an empty dimension", b);
    max_n = std::max(max_n, n[b]);
  }
  if (count == 0) return;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  unsigned char* base = static_cast<unsigned char*>(noalloc_scratch());
  int* d_m = reinterpret_cast<int*>(base);
  int* d_n = reinterpret_cast<int*>(base + (size_t)ID_NOALLOC_MAX * 4);
  long long* d_a = reinterpret_cast<long long*>(base + (size_t)ID_NOALLOC_MAX * 8);
  long long* d_s = reinterpret_cast<long long*>(base + (size_t)ID_NOALLOC_MAX * 16);
  long long* d_v = reinterpret_cast<long long*>(base + (size_t)ID_NOALLOC_MAX * 24);
  // one host-to-device copy of the staged metadata: m, n, a_off in the
  // array's order (int m[MAX], int n[MAX], long long a_off[MAX]); only the
  // first count entries of each part are copied
  int* h_m = reinterpret_cast<int*>(g_noalloc_host);
  int* h_n = reinterpret_cast<int*>(g_noalloc_host + (size_t)ID_NOALLOC_MAX * 4);
  long long* h_a = reinterpret_cast<long long*>(g_noalloc_host + (size_t)ID_NOALLOC_MAX * 8);
  std::memcpy(h_m, m, sizeof(int) * count);
  std::memcpy(h_n, n, sizeof(int) * count);
  std::memcpy(h_a, a_off, sizeof(long long) * count);
  HB_CUDA(cudaMemcpyAsync(d_m, h_m, sizeof(int) * count, cudaMemcpyHostToDevice, st));
  HB_CUDA(cudaMemcpyAsync(d_n, h_n, sizeof(int) * count, cudaMemcpyHostToDevice, st));
  HB_CUDA(cudaMemcpyAsync(d_a, h_a, sizeof(long long) * count, cudaMemcpyHostToDevice, st));
  noalloc_offsets_kernel<<<1, 1024, 0, st>>>(d_n, count, d_s, d_v);
  HB_CHECK_LAUNCH();
  id_batch(count, d_m, d_n, d_a, A, eps, rank, skel, d_s, max_n, st);
  emit_v(count, d_m, d_n, d_a, A, rank, skel, d_s, d_v, 0, V, nullptr, st);
}

}  // namespace hb
