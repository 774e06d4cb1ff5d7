// Measured FMA throughput of this GPU (the arithmetic roofs the HBM and
// tensor measurements do not give): every thread runs 8 independent chains
// of fused multiply-adds, enough to fill the FP32 and FP64 pipes of every SM.
#include "runtime.hpp"

namespace aeth {

template <typename R>
__global__ void __launch_bounds__(256) k_fma_probe(R* __restrict__ out, int iters, R a, R b) {
  R x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = R(threadIdx.x + q) * R(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, b);
  }
  R s = R(0);
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  if (s == R(-1)) out[blockIdx.x] = s;   // keeps the chains live; never true
}

template <typename R>
static aeth_status probe_T(double* flops, int iters) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return AETH_ERR_CUDA;
  const int grid = sms * 8, block = 256;
  R* out = nullptr;
  if (cudaMalloc(&out, grid * sizeof(R)) != cudaSuccess) return AETH_ERR_OOM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const R a = R(0.9999999), b = R(1e-7);
  k_fma_probe<R><<<grid, block>>>(out, iters, a, b);   // warm-up
  cudaEventRecord(e0);
  k_fma_probe<R><<<grid, block>>>(out, iters, a, b);
  cudaEventRecord(e1);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess || ms <= 0.f) return AETH_ERR_CUDA;
  *flops = 2.0 * 8.0 * (double)iters * grid * block / (ms * 1e-3);
  return AETH_OK;
}

}  // namespace aeth

extern "C" aeth_status aeth_probe_fma(int precision, double* flops_per_s) {
  if (!flops_per_s) return AETH_ERR_ARG;
  if (precision == AETH_FP64) return aeth::probe_T<double>(flops_per_s, 1 << 10);
  if (precision == AETH_FP32) return aeth::probe_T<float>(flops_per_s, 1 << 15);
  return AETH_ERR_ARG;
}
