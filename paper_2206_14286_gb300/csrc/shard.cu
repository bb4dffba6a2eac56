// shard.cu -- kernels of the N-sharded search: a database split by rows over
// several GPUs (Sec. 7 runs the search on sharded TPU pods; App. A.1's
// reduction_input_size_override plans the bins for the whole input). Every
// shard runs PartialReduce on its rows with global row indices and the
// global L, then the shards exchange two arrays, each merged by an
// element-wise maximum:
//   1. the M x L bin winners, as 64-bit keys;
//   2. the FP32 scores of the Kp candidates of ExactRescoring, which each
//      shard computes for the rows it holds (the other entries stay empty).
// Keys are exchanged in a signed-order form, key ^ 2^63 read as int64, so a
// plain MAX reduction over int64 (NCCL, gloo, torch) merges them; the empty
// key 0 becomes INT64_MIN, below every real key.
#include "common.cuh"
#include "kernels.h"

namespace tpuknn {

namespace {

constexpr uint64_t kSignBit = 0x8000000000000000ull;

// (value, local index) pairs of PartialReduce -> signed keys with global
// indices (index + add); index -1 (an empty bin) -> the empty key.
__global__ void pairs_to_signed_keys_kernel(const float* __restrict__ v,
                                            const int32_t* __restrict__ a, int64_t n,
                                            int64_t add, int64_t* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int32_t j = a[t];
  const uint64_t k = j < 0 ? 0ull : make_key(v[t], (int32_t)(j + add));
  out[t] = (int64_t)(k ^ kSignBit);
}

__global__ void signed_to_keys_kernel(const int64_t* __restrict__ in, int64_t n,
                                      uint64_t* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = (uint64_t)in[t] ^ kSignBit;
}

// One warp per (query, candidate): the FP32 score of a candidate this shard
// holds (global rows [row0, row0 + n_local)), as a signed key; the empty key
// for the others. Lanes take the elements d = lane, lane + 32, ... and the
// warp sums by butterfly shuffles (the order of the library's re-rank for
// more than 32 candidates).
__global__ void __launch_bounds__(256)
score_owned_kernel(const uint64_t* __restrict__ cand, int64_t M, int Kp,
                   const float* __restrict__ q, int64_t q_stride, const float* __restrict__ x,
                   int64_t n_local, int64_t row0, int D, int metric, int64_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= M * Kp) return;
  const int64_t i = w / Kp;
  const uint64_t key = cand[w];
  const int64_t j = key ? (int64_t)key_index(key) : -1;
  if (j < row0 || j >= row0 + n_local) {
    if (lane == 0) out[w] = (int64_t)kSignBit;  // the empty key
    return;
  }
  const float* qi = q + i * q_stride;
  const float* xr = x + (j - row0) * (int64_t)D;
  float acc = 0.0f;
  for (int d = lane; d < D; d += 32) {
    const float qq = qi[d], xx = xr[d];
    if (metric == KNN_L2) {
      const float t = qq - xx;
      acc = fmaf(t, t, acc);
    } else {
      acc = fmaf(qq, xx, acc);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0)
    out[w] = (int64_t)(make_key(metric == KNN_L2 ? -acc : acc, (int32_t)j) ^ kSignBit);
}

}  // namespace

cudaError_t launch_pairs_to_signed_keys(const float* v, const int32_t* a, int64_t n, int64_t add,
                                        int64_t* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  pairs_to_signed_keys_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(v, a, n, add, out);
  return cudaGetLastError();
}

cudaError_t launch_signed_to_keys(const int64_t* in, int64_t n, uint64_t* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  signed_to_keys_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(in, n, out);
  return cudaGetLastError();
}

cudaError_t launch_score_owned(const uint64_t* cand, int64_t M, int Kp, const float* q,
                               int64_t q_stride, const float* x, int64_t n_local, int64_t row0,
                               int D, int metric, int64_t* out, cudaStream_t st) {
  const int64_t warps = M * Kp;
  if (warps <= 0) return cudaSuccess;
  score_owned_kernel<<<(unsigned)cdiv(warps * 32, 256), 256, 0, st>>>(cand, M, Kp, q, q_stride, x,
                                                                     n_local, row0, D, metric, out);
  return cudaGetLastError();
}

}  // namespace tpuknn
