// FP64 fused multiply-add throughput of the device: the ALU roofline of the
// FP64 path (whose GEMV-shaped Riccati passes do about 0.24 flop per byte of
// factors, which on this GPU is more than its FP64 units sustain at the HBM
// rate).  Every thread runs kChains independent FMA chains, so the FP64 pipe,
// not the latency of one chain, sets the rate.
#include <cuda_runtime.h>

#include "spock_internal.h"

namespace spock {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fp64_fma(int iters, double a, double b, double* __restrict__ sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == 12345.678) sink[threadIdx.x] = s;   // keeps the chains live; never true for these inputs
}

// Runs the kernel on `stream` (grid: 8 blocks of 256 threads per SM) and
// returns the FMA rate in TFLOP/s (2 flops per FMA) measured with events.
int fp64_fma_rate(int iters, double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(SPOCK_ERR_CUDA, "cudaGetDevice");
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(SPOCK_ERR_CUDA, "cudaDeviceGetAttribute");
  double* sink = nullptr;
  if (cudaMalloc(&sink, 256 * sizeof(double)) != cudaSuccess) return fail(SPOCK_ERR_OOM, "cudaMalloc");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int grid = sms * 8;
  k_fp64_fma<<<grid, 256, 0, st>>>(iters / 10 + 1, 0.999999, 1e-7, sink);   // warm-up
  cudaEventRecord(e0, st);
  k_fp64_fma<<<grid, 256, 0, st>>>(iters, 0.999999, 1e-7, sink);
  cudaEventRecord(e1, st);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) return fail(SPOCK_ERR_CUDA, cudaGetErrorString(err));
  const double flops = 2.0 * kChains * (double)iters * (double)grid * 256.0;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return SPOCK_OK;
}

}  // namespace spock
