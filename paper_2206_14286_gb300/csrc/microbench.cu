// microbench.cu -- issue-rate microbenchmarks behind knn_measure_rate: the
// inputs of the instruction-throughput roofline of Sec. 4 (Eq. 6, Eq. 8-9)
// measured on this GPU instead of derived from unit counts.
//
//   KNN_RATE_MINMAX : FP32 min/max, the compare-and-select operation (COP)
//                     PartialReduce spends per score (Alg. 1 keeps a running
//                     maximum per bin): gamma of Eq. 6.
//   KNN_RATE_FFMA   : FP32 fused multiply-add, the roof of the CUDA-core
//                     (SIMT) FP32 contraction.
//
// Every thread runs kChains independent dependency chains so that the pipe,
// not the latency of one chain, limits the rate; the grid holds 2048 threads
// per SM. Each chain ends in a value that is stored only if it equals a
// sentinel no run produces, so nothing is dead code, and no memory traffic
// enters the timing.
#include "common.cuh"
#include "kernels.h"

namespace tpuknn {

namespace {

constexpr int kChains = 16;
constexpr int kRateThreads = 256, kRateBlocksPerSm = 8;
__device__ float g_rate_sink[kChains];

// Per iteration kChains min/max operations: chain k takes the max (k even)
// or the min (k odd) of itself and its ring neighbour, so no operation
// repeats an earlier one and nothing folds away.
__global__ void __launch_bounds__(kRateThreads) rate_minmax_kernel(int64_t iters, float seed) {
  float x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = seed * (float)(threadIdx.x + 3 * k + 1);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      const float y = x[(k + 1) % kChains];
      if (k & 1)
        asm volatile("min.f32 %0, %0, %1;" : "+f"(x[k]) : "f"(y));
      else
        asm volatile("max.f32 %0, %0, %1;" : "+f"(x[k]) : "f"(y));
    }
  }
#pragma unroll
  for (int k = 0; k < kChains; ++k)
    if (x[k] == 1234.5678f) g_rate_sink[k] = x[k];
}

__global__ void __launch_bounds__(kRateThreads) rate_ffma_kernel(int64_t iters, float seed) {
  float x[kChains];
  const float a = 1.0f - seed * 1e-3f, b = seed * 1e-3f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = seed * (float)(threadIdx.x + k);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[k]) : "f"(a), "f"(b));
  }
#pragma unroll
  for (int k = 0; k < kChains; ++k)
    if (x[k] == 1234.5678f) g_rate_sink[k] = x[k];
}

}  // namespace

cudaError_t measure_rate(int kind, int64_t iters, double* ops_per_s, double* ms_out,
                         cudaStream_t st) {
  const int sms = device_sm_count();
  const unsigned blocks = (unsigned)(sms * kRateBlocksPerSm);
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  auto launch = [&]() {
    if (kind == KNN_RATE_MINMAX)
      rate_minmax_kernel<<<blocks, kRateThreads, 0, st>>>(iters, 0.5f);
    else
      rate_ffma_kernel<<<blocks, kRateThreads, 0, st>>>(iters, 0.5f);
    return cudaGetLastError();
  };
  // one untimed launch (clocks ramp, code loads), then the timed one
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  if (e == cudaSuccess) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (e != cudaSuccess) return e;
  const double ops = (double)blocks * kRateThreads * (double)iters * kChains;
  *ops_per_s = ops / (ms * 1e-3);
  *ms_out = ms;
  return cudaSuccess;
}

}  // namespace tpuknn
