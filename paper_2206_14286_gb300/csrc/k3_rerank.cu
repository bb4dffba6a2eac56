// k3_rerank.cu -- FP32 scoring of the Kp candidates that leave ExactRescoring
// and selection of the final K (the precision pattern: BF16 / E4M3 decide
// the candidates, FP32 decides their order and values).
//
// Kp <= 32: one warp per query (k3_warp4_kernel for 16-byte aligned FP32
// rows, k3_warp_kernel otherwise), the keys sorted across the lanes. Larger
// Kp: one CTA per query; each warp scores four candidates at a time with lanes
// splitting D (coalesced row reads), then the Kp keys are sorted in shared
// memory. Values: IP <q,x>; L2 sum (q-x)^2 evaluated directly; COS <q,x> of
// the unit-length rows.
#include "common.cuh"
#include "dtypes.cuh"
#include "kernels.h"

namespace tpuknn {

namespace {
__global__ void __launch_bounds__(256)
k3_rerank_kernel(const uint64_t* __restrict__ cand, int Kp, int K, int P2, int D, int metric,
                 const float* __restrict__ qf32, int64_t q_stride,
                 const float* __restrict__ xf32, const void* __restrict__ xlp, int dtype,
                 int pitch, const float* __restrict__ xscale, int64_t N,
                 float* __restrict__ out_val, int32_t* __restrict__ out_idx) {
  extern __shared__ uint64_t sk[];
  const int64_t i = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const float* q = qf32 + i * q_stride;
  // a warp scores kCand candidates together, their row loads in flight at
  // once; per candidate the same sums in the same order as one at a time
  constexpr int kCand = 4;
  for (int c0 = warp * kCand; c0 < Kp; c0 += nwarps * kCand) {
    int32_t jj[kCand];
#pragma unroll
    for (int u = 0; u < kCand; ++u) {
      const uint64_t key = c0 + u < Kp ? cand[i * Kp + c0 + u] : 0;
      const int32_t j = key ? key_index(key) : -1;
      jj[u] = (j >= 0 && j < N) ? j : -1;
    }
    float acc[kCand];
#pragma unroll
    for (int u = 0; u < kCand; ++u) acc[u] = 0.0f;
    for (int d = lane; d < D; d += 32) {
      const float qq = q[d];
      float xv[kCand];
#pragma unroll
      for (int u = 0; u < kCand; ++u)
        xv[u] = jj[u] < 0 ? 0.0f
                          : (xf32 ? xf32[(int64_t)jj[u] * D + d]
                                  : load_stored(xlp, dtype, jj[u], pitch, d, xscale));
#pragma unroll
      for (int u = 0; u < kCand; ++u) {
        if (metric == KNN_L2) {
          const float t = qq - xv[u];
          acc[u] = fmaf(t, t, acc[u]);
        } else {
          acc[u] = fmaf(qq, xv[u], acc[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kCand; ++u) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int u = 0; u < kCand; ++u)
        if (c0 + u < Kp)
          sk[c0 + u] = jj[u] < 0 ? 0 : make_key(metric == KNN_L2 ? -acc[u] : acc[u], jj[u]);
    }
  }
  for (int t = Kp + threadIdx.x; t < P2; t += blockDim.x) sk[t] = 0;
  bitonic_sort_desc(sk, P2);
  for (int t = threadIdx.x; t < K; t += blockDim.x) {
    const uint64_t key = t < Kp ? sk[t] : 0;
    const float s = key_score(key);
    out_idx[i * K + t] = key ? key_index(key) : -1;
    out_val[i * K + t] = key ? (metric == KNN_L2 ? -s : s) : __int_as_float(0x7fc00000);
  }
}
__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int o) {
  const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, o);
  const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), o);
  return ((uint64_t)hi << 32) | lo;
}

// One warp per query for Kp <= 32: the warp scores the candidates one after
// another (lanes split D), lane c keeps candidate c's key, and a bitonic
// network across the lanes sorts the keys (lane 0 = best).
__global__ void __launch_bounds__(256)
k3_warp_kernel(int64_t M, const uint64_t* __restrict__ cand, int Kp, int K, int D, int metric,
               const float* __restrict__ qf32, int64_t q_stride,
               const float* __restrict__ xf32, const void* __restrict__ xlp, int dtype,
               int pitch, const float* __restrict__ xscale, int64_t N,
               float* __restrict__ out_val, int32_t* __restrict__ out_idx) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= M) return;
  const float* q = qf32 + i * q_stride;
  const uint64_t mykey_in = lane < Kp ? cand[i * Kp + lane] : 0;
  uint64_t mine = 0;
  // 8 candidates at a time: their row loads are independent, so they overlap
  for (int c0 = 0; c0 < Kp; c0 += 8) {
    int32_t js[8];
    float acc[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const uint64_t key = __shfl_sync(0xffffffffu, mykey_in, (c0 + u) & 31);
      const int32_t j = (c0 + u < Kp && key) ? key_index(key) : -1;
      js[u] = (j >= 0 && j < N) ? j : -1;
      acc[u] = 0.0f;
    }
    for (int d = lane; d < D; d += 32) {
      const float qq = q[d];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (js[u] < 0) continue;  // warp-uniform
        const float x = xf32 ? xf32[(int64_t)js[u] * D + d]
                             : load_stored(xlp, dtype, js[u], pitch, d, xscale);
        if (metric == KNN_L2) {
          const float t = qq - x;
          acc[u] = fmaf(t, t, acc[u]);
        } else {
          acc[u] = fmaf(qq, x, acc[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      float v = acc[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == c0 + u && js[u] >= 0) mine = make_key(metric == KNN_L2 ? -v : v, js[u]);
    }
  }
  // descending bitonic sort across the 32 lanes
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      const uint64_t other = shfl_xor_u64(mine, jj);
      const bool up = (lane & k) == 0, lower = (lane & jj) == 0;
      const bool keep_max = (up == lower);
      mine = keep_max ? (other > mine ? other : mine) : (other < mine ? other : mine);
    }
  }
  if (lane < K) {
    const float sc = key_score(mine);
    out_idx[i * K + lane] = mine ? key_index(mine) : -1;
    out_val[i * K + lane] = mine ? (metric == KNN_L2 ? -sc : sc) : __int_as_float(0x7fc00000);
  }
}
// The same for FP32 rows with D % 4 == 0 (16-byte aligned rows): a lane
// loads 4 consecutive elements, so one warp instruction reads 512 bytes of
// a row, and the rows of 16 candidates are requested before any is used.
template <int METRIC>
__global__ void __launch_bounds__(128)
k3_warp4_kernel(int64_t M, const uint64_t* __restrict__ cand, int Kp, int K, int D,
                const float* __restrict__ qf32, int64_t q_stride, const float* __restrict__ xf32,
                int64_t N, float* __restrict__ out_val, int32_t* __restrict__ out_idx) {
  constexpr int kB = 16;
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= M) return;
  const float* q = qf32 + i * q_stride;
  const uint64_t mykey_in = lane < Kp ? cand[i * Kp + lane] : 0;
  uint64_t mine = 0;
  for (int c0 = 0; c0 < Kp; c0 += kB) {
    int32_t js[kB];
    float acc[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const uint64_t key = __shfl_sync(0xffffffffu, mykey_in, (c0 + u) & 31);
      const int32_t j = (c0 + u < Kp && key) ? key_index(key) : -1;
      js[u] = (j >= 0 && j < N) ? j : -1;
      acc[u] = 0.0f;
    }
    for (int d0 = 0; d0 < D; d0 += 128) {
      const int d = d0 + lane * 4;
      const bool in = d < D;
      const float4 qv = in ? *reinterpret_cast<const float4*>(q + d) : make_float4(0, 0, 0, 0);
      float4 xv[kB];
#pragma unroll
      for (int u = 0; u < kB; ++u)
        xv[u] = (in && js[u] >= 0) ? __ldg(reinterpret_cast<const float4*>(xf32 + (int64_t)js[u] * D + d))
                                   : make_float4(0, 0, 0, 0);
#pragma unroll
      for (int u = 0; u < kB; ++u) {
        if (METRIC == KNN_L2) {
          // rows past D contribute 0: both sides are zero there
          const float t0 = qv.x - xv[u].x, t1 = qv.y - xv[u].y, t2 = qv.z - xv[u].z,
                      t3 = qv.w - xv[u].w;
          acc[u] = fmaf(t0, t0, acc[u]);
          acc[u] = fmaf(t1, t1, acc[u]);
          acc[u] = fmaf(t2, t2, acc[u]);
          acc[u] = fmaf(t3, t3, acc[u]);
        } else {
          acc[u] = fmaf(qv.x, xv[u].x, acc[u]);
          acc[u] = fmaf(qv.y, xv[u].y, acc[u]);
          acc[u] = fmaf(qv.z, xv[u].z, acc[u]);
          acc[u] = fmaf(qv.w, xv[u].w, acc[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      float v = acc[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == c0 + u && js[u] >= 0) mine = make_key(METRIC == KNN_L2 ? -v : v, js[u]);
    }
  }
#pragma unroll
  for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
    for (int jj = k >> 1; jj > 0; jj >>= 1) {
      const uint64_t other = shfl_xor_u64(mine, jj);
      const bool up = (lane & k) == 0, lower = (lane & jj) == 0;
      const bool keep_max = (up == lower);
      mine = keep_max ? (other > mine ? other : mine) : (other < mine ? other : mine);
    }
  }
  if (lane < K) {
    const float sc = key_score(mine);
    out_idx[i * K + lane] = mine ? key_index(mine) : -1;
    out_val[i * K + lane] = mine ? (METRIC == KNN_L2 ? -sc : sc) : __int_as_float(0x7fc00000);
  }
}
}  // namespace

cudaError_t launch_k3(int64_t M, int D, int metric, const uint64_t* cand, int Kp, int K,
                      const float* qf32, int64_t q_stride, const float* xf32, const void* xlp,
                      int dtype, int pitch, const float* xscale, int64_t N, float* out_val,
                      int32_t* out_idx, cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  const bool vec = xf32 && D % 4 == 0 && q_stride % 4 == 0 &&
                   (reinterpret_cast<uintptr_t>(xf32) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(qf32) & 15) == 0;
  if (Kp <= 32 && K <= 32 && vec) {
    const unsigned blocks = (unsigned)cdiv(M * 32, 128);
    if (metric == KNN_L2)
      k3_warp4_kernel<KNN_L2><<<blocks, 128, 0, st>>>(M, cand, Kp, K, D, qf32, q_stride, xf32, N,
                                                      out_val, out_idx);
    else
      k3_warp4_kernel<KNN_IP><<<blocks, 128, 0, st>>>(M, cand, Kp, K, D, qf32, q_stride, xf32, N,
                                                      out_val, out_idx);
    return cudaGetLastError();
  }
  if (Kp <= 32 && K <= 32) {
    k3_warp_kernel<<<(unsigned)cdiv(M * 32, 256), 256, 0, st>>>(
        M, cand, Kp, K, D, metric, qf32, q_stride, xf32, xlp, dtype, pitch, xscale, N, out_val,
        out_idx);
    return cudaGetLastError();
  }
  const int P2 = next_pow2(Kp > K ? Kp : K);
  const size_t smem = (size_t)P2 * sizeof(uint64_t);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k3_rerank_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k3_rerank_kernel<<<(unsigned)M, 256, smem, st>>>(cand, Kp, K, P2, D, metric, qf32, q_stride,
                                                   xf32, xlp, dtype, pitch, xscale, N, out_val,
                                                   out_idx);
  return cudaGetLastError();
}

}  // namespace tpuknn
