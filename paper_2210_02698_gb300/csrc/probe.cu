// probe.cu - measured FP64 peak of the device (the denominator of the
// rooflines of the FP64 paths: the butterfly apply on complex128 factors,
// the matrix-free dense sum, the entry evaluation of the build).
//
// Every thread runs CHAINS independent FP64 fused multiply-add recurrences
// x <- x a + b for `iters` steps; the grid fills every SM with several CTAs,
// so the FP64 pipes, not latency, set the rate.  2 flops per FMA.
#include <cuda_runtime.h>

#include "hb_internal.cuh"

namespace hb {

constexpr int PROBE_CHAINS = 8;

__global__ void __launch_bounds__(256) fp64_fma_kernel(double* out, int iters, double a, double b) {
  double x[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) s += x[c];
  // never true for the arguments used; keeps the chains live
  if (s == -1.0) out[blockIdx.x] = s;
}

}  // namespace hb

extern "C" hb_status hb_fp64_fma_peak(double* tflops, void* stream) {
  try {
    if (!tflops) return HB_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    HB_CUDA(cudaGetDevice(&dev));
    HB_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = nsm * 8, iters = 1 << 14;
    cudaEvent_t e0, e1;
    HB_CUDA(cudaEventCreate(&e0));
    HB_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {   // the first run warms up
      cudaEventRecord(e0, st);
      hb::fp64_fma_kernel<<<grid, 256, 0, st>>>(nullptr, iters, 0.999999, 1e-7);
      cudaEventRecord(e1, st);
      const cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return HB_ERR_CUDA;
      }
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best = ms < best ? ms : best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const double flops = 2.0 * hb::PROBE_CHAINS * (double)iters * 256.0 * grid;
    *tflops = flops / (best * 1e-3) / 1e12;
    return HB_OK;
  } catch (const hb::Error& e) {
    return e.code;
  }
}
