// FP64 fused multiply-add throughput of the device: the ALU roofline of the
// FP64 path (whose GEMV-shaped Riccati passes do about 0.24 flop per byte of
// factors, which on this GPU is more than its FP64 units sustain at the HBM
// rate).
#include <algorithm>

#include <cuda_runtime.h>

#include "spock_internal.h"

namespace spock {

template <int C>
__global__ void __launch_bounds__(256) k_fp64_fma(int iters, double a, double b, double* __restrict__ sink) {
  double x[C];
#pragma unroll
  for (int c = 0; c < C; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < C; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < C; ++c) s += x[c];
  if (s == 12345.678) sink[threadIdx.x] = s;   // keeps the chains live; never true for these inputs
}

// One timed launch (after a warm-up launch) of C chains per thread and
// `bps` blocks of 256 threads per SM; returns TFLOP/s.
template <int C>
static double fma_rate_one(int iters, int bps, int sms, double* sink, cudaStream_t st) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int grid = sms * bps;
  const int it = iters * 8 / C;   // the same FMA count per thread for every C
  k_fp64_fma<C><<<grid, 256, 0, st>>>(it / 10 + 1, 0.999999, 1e-7, sink);
  cudaEventRecord(e0, st);
  k_fp64_fma<C><<<grid, 256, 0, st>>>(it, 0.999999, 1e-7, sink);
  cudaEventRecord(e1, st);
  float ms = 0.f;
  const bool ok = cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok || ms <= 0.f) return -1.0;
  return 2.0 * C * (double)it * (double)grid * 256.0 / (ms * 1e-3) / 1e12;
}

// The FP64 FMA rate in TFLOP/s (2 flops per FMA): the best over 8 or 16
// independent chains per thread and 4 or 8 blocks of 256 threads per SM, so
// that the FP64 pipe, not the latency of a chain or the occupancy, sets it.
int fp64_fma_rate(int iters, double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(SPOCK_ERR_CUDA, "cudaGetDevice");
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(SPOCK_ERR_CUDA, "cudaDeviceGetAttribute");
  double* sink = nullptr;
  if (cudaMalloc(&sink, 256 * sizeof(double)) != cudaSuccess) return fail(SPOCK_ERR_OOM, "cudaMalloc");
  double best = -1.0;
  for (int bps : {4, 8}) {
    best = std::max(best, fma_rate_one<8>(iters, bps, sms, sink, st));
    best = std::max(best, fma_rate_one<16>(iters, bps, sms, sink, st));
  }
  cudaFree(sink);
  const cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return fail(SPOCK_ERR_CUDA, cudaGetErrorString(err));
  if (!(best > 0.0)) return fail(SPOCK_ERR_CUDA, "FMA rate kernel did not run");
  *tflops = best;
  return SPOCK_OK;
}

}  // namespace spock
