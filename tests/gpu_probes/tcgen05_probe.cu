// tcgen05 probe (test program, not part of the library): one CTA issues
// tcgen05.mma.cta_group::1.kind::f16 (bf16 x bf16 -> f32 in TMEM) on
// K-major, unswizzled shared-memory operands and reads the accumulator back
// with tcgen05.ld.  Prints, one per line:
//   exact M N mismatches        - integer product checked element by element
//   layout64 lane row           - where the rows of an M = 64 accumulator land
//   rate M N cycles_per_mma     - back-to-back MMAs from one thread into one accumulator
// Every operand read stays inside the shared buffers; every wait is bounded.
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start >> 4, leading byte offset >> 4 (the
// stride between the two 8-element core matrices along K), stride byte offset
// >> 4 (between 8-row groups), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t par, long long deadline) {
  uint32_t ok = 0;
  while (!ok) {
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(par) : "memory");
    if (!ok && clock64() > deadline) return false;
  }
  return true;
}

// mode 0: one MMA, D (all 128 lanes x 64 columns, zeroed first) to gD;
// mode 1: `count` MMAs back to back, cycles to gC[0]
__global__ void probe(const uint16_t* gA, const uint16_t* gB, float* gD, uint32_t idesc, int mode, int count,
                      long long* gC, int* err) {
  __shared__ __align__(1024) uint16_t sA[8192];
  __shared__ __align__(1024) uint16_t sB[8192];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < 8192; i += 128) {
    sA[i] = gA[i];
    sB[i] = gB[i];
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (mode == 0) {
    uint32_t z[32];
    for (int c = 0; c < 32; ++c) z[c] = 0;
    for (int h = 0; h < 2; ++h) {
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + 32 * h;
      asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                   "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
                   :: "r"(ta), "r"(z[0]), "r"(z[1]), "r"(z[2]), "r"(z[3]), "r"(z[4]), "r"(z[5]), "r"(z[6]), "r"(z[7]),
                   "r"(z[8]), "r"(z[9]), "r"(z[10]), "r"(z[11]), "r"(z[12]), "r"(z[13]), "r"(z[14]), "r"(z[15]),
                   "r"(z[16]), "r"(z[17]), "r"(z[18]), "r"(z[19]), "r"(z[20]), "r"(z[21]), "r"(z[22]), "r"(z[23]),
                   "r"(z[24]), "r"(z[25]), "r"(z[26]), "r"(z[27]), "r"(z[28]), "r"(z[29]), "r"(z[30]), "r"(z[31])
                   : "memory");
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (tid == 0) {
    const uint64_t ad = make_desc(smem_u32(sA), 128, 256);
    const uint64_t bd = make_desc(smem_u32(sB), 128, 256);
    const int n = mode == 0 ? 1 : count;
    const long long t0 = clock64();
    for (int i = 0; i < n; ++i)
      asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                   ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(i) : "memory");
    const long long t1 = clock64();
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&bar))
                 : "memory");
    if (mode == 1) gC[0] = t1 - t0;
  }
  if (!wait_bar(&bar, 0, clock64() + (1LL << 31)) && lane == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (mode == 0) {
    for (int h = 0; h < 2; ++h) {
      uint32_t r[32];
      const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + 32 * h;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                   "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                   : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                     "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                     "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                     "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                     "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                   : "r"(ta));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      for (int c = 0; c < 32; ++c) gD[(warp * 32 + lane) * 64 + 32 * h + c] = __uint_as_float(r[c]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
}

static uint16_t bf16_of(float f) {   // exact for the small integers used here
  uint32_t u;
  memcpy(&u, &f, 4);
  return (uint16_t)(u >> 16);
}

// instruction descriptor: D f32, A and B bf16, both K-major, N >> 3 at bit 17, M >> 4 at bit 24
static uint32_t idesc_of(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// canonical K-major, unswizzled: core matrix (8 rows x 16 bytes) contiguous,
// core (8-row group g, K half c) at g * 256 + c * 128 bytes
static size_t at(int row, int k) { return ((row / 8) * 256 + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2) / 2; }

int main() {
  uint16_t *dA, *dB;
  float* dD;
  long long* dC;
  int* dErr;
  cudaMalloc(&dA, 16384);
  cudaMalloc(&dB, 16384);
  cudaMalloc(&dD, 128 * 64 * 4);
  cudaMalloc(&dC, 8);
  cudaMalloc(&dErr, 4);
  int herr = 0;
  // exact products: D[m][n] = sum_k A[m][k] B[n][k]
  const int shapes[2][2] = {{128, 32}, {64, 32}};
  for (auto& sh : shapes) {
    const int M = sh[0], N = sh[1], K = 16;
    std::vector<uint16_t> hA(8192, 0), hB(8192, 0);
    std::vector<float> A(M * K), B(N * K);
    for (int m = 0; m < M; ++m)
      for (int k = 0; k < K; ++k) hA[at(m, k)] = bf16_of(A[m * K + k] = (float)(((m * 7 + k * 3) % 11) - 5));
    for (int n = 0; n < N; ++n)
      for (int k = 0; k < K; ++k) hB[at(n, k)] = bf16_of(B[n * K + k] = (float)(((n * 5 + k * 13) % 9) - 4));
    cudaMemcpy(dA, hA.data(), 16384, cudaMemcpyHostToDevice);
    cudaMemcpy(dB, hB.data(), 16384, cudaMemcpyHostToDevice);
    cudaMemset(dErr, 0, 4);
    probe<<<1, 128>>>(dA, dB, dD, idesc_of(M, N), 0, 1, dC, dErr);
    if (cudaDeviceSynchronize() != cudaSuccess) return 2;
    std::vector<float> D(128 * 64);
    cudaMemcpy(D.data(), dD, D.size() * 4, cudaMemcpyDeviceToHost);
    cudaMemcpy(&herr, dErr, 4, cudaMemcpyDeviceToHost);
    if (herr) return 3;
    int bad = 0;
    for (int m = 0; m < M; ++m) {
      // M = 128: row m in lane m; M = 64: row m in lane (m % 16) + 32 (m / 16)
      const int l = M == 128 ? m : (m % 16) + 32 * (m / 16);
      for (int n = 0; n < N; ++n) {
        float ref = 0;
        for (int k = 0; k < K; ++k) ref += A[m * K + k] * B[n * K + k];
        if (D[l * 64 + n] != ref) ++bad;
      }
    }
    printf("exact %d %d %d\n", M, N, bad);
  }
  // issue rate, one accumulator
  std::vector<uint16_t> ones(8192, 0x3f80);
  cudaMemcpy(dA, ones.data(), 16384, cudaMemcpyHostToDevice);
  cudaMemcpy(dB, ones.data(), 16384, cudaMemcpyHostToDevice);
  const int rs[4][2] = {{128, 16}, {128, 32}, {128, 64}, {64, 32}};
  for (auto& sh : rs) {
    long long c = 0;
    for (int rep = 0; rep < 2; ++rep) {
      cudaMemset(dErr, 0, 4);
      probe<<<1, 128>>>(dA, dB, dD, idesc_of(sh[0], sh[1]), 1, 4096, dC, dErr);
      if (cudaDeviceSynchronize() != cudaSuccess) return 4;
      cudaMemcpy(&c, dC, 8, cudaMemcpyDeviceToHost);
      cudaMemcpy(&herr, dErr, 4, cudaMemcpyDeviceToHost);
      if (herr) return 5;
    }
    printf("rate %d %d %.2f\n", sh[0], sh[1], c / 4096.0);
  }
  return 0;
}
