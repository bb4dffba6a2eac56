// common.cuh -- small device/host helpers shared by the library's kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/tpuknn.h"

namespace tpuknn {

// ---------------------------------------------------------------------------
// Programmatic dependent launch inside one search call. A kernel launched
// with launch_pdl may start (and run its prologue) before the previous kernel
// of the stream has finished; it calls pdl_wait() before it touches global
// memory that kernel writes. pdl_wait() returns once the previous grid has
// completed and its writes are visible (at once for a plain launch). A
// kernel calls pdl_trigger() in every CTA to let the next one launch early;
// the next kernel then launches only after every CTA of this one has
// started, so its CTAs never hold back this kernel's.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

constexpr int kMaxK = 4096;       // largest K (and K') a search accepts
constexpr int kMaxD = 4096;       // largest row length
constexpr uint32_t kNegInfBits = 0xff800000u;

// ---------------------------------------------------------------------------
// Ordered 64-bit keys: (score, index) pairs that compare as unsigned integers
// in the order "larger score first, then smaller index" (the tie rule).
// The high word maps the IEEE float to an unsigned integer whose order is the
// float order; the low word is the bitwise complement of the index, so the
// smaller index gives the larger key. Key 0 is below every real pair and
// marks an empty slot.
// ---------------------------------------------------------------------------
// How rows of `dtype` are stored and decoded: KNN_E4M3_T rows are KNN_E4M3
// rows whose scales are all equal.
__host__ __device__ __forceinline__ int stored_dtype(int dtype) {
  return dtype == KNN_E4M3_T ? KNN_E4M3 : dtype;
}

__host__ __device__ __forceinline__ uint32_t f2u(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}
__host__ __device__ __forceinline__ float u2f(uint32_t u) {
  float f;
  memcpy(&f, &u, 4);
  return f;
}
__host__ __device__ __forceinline__ uint32_t float_to_ordered(float f) {
  uint32_t u = f2u(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float ordered_to_float(uint32_t o) {
  uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
  return u2f(u);
}
__host__ __device__ __forceinline__ uint64_t make_key(float score, int32_t idx) {
  return ((uint64_t)float_to_ordered(score) << 32) | (uint64_t)(~(uint32_t)idx);
}
__host__ __device__ __forceinline__ float key_score(uint64_t k) {
  return ordered_to_float((uint32_t)(k >> 32));
}
__host__ __device__ __forceinline__ int32_t key_index(uint64_t k) {
  return (int32_t)(~(uint32_t)(k & 0xffffffffu));
}

__device__ __forceinline__ float neg_inf() { return __uint_as_float(kNegInfBits); }

// ---------------------------------------------------------------------------
// In-place bitonic sort of n (a power of two) 64-bit keys in shared memory,
// descending, by all threads of the block. Ends with __syncthreads().
// ---------------------------------------------------------------------------
__device__ __forceinline__ void bitonic_sort_desc(uint64_t* s, int n) {
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
        int lo = 2 * t - (t & (stride - 1));
        int hi = lo + stride;
        bool desc = ((lo & size) == 0);
        uint64_t a = s[lo], b = s[hi];
        if ((a < b) == desc) {
          s[lo] = b;
          s[hi] = a;
        }
      }
    }
  }
  __syncthreads();
}

__host__ __device__ __forceinline__ int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Round-up helpers.
__host__ __device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ __forceinline__ int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }

}  // namespace tpuknn
