// k5_backward.cu -- gradient of the selected values with respect to the
// queries and the database rows (the differentiation pattern).
//
// With the selected indices held constant, for F = sum_{i,k} g[i,k] f(q_i, x_j),
// j = idx[i,k], f the reported value:
//   IP : df/dq = x,                       df/dx = q
//   L2 : df/dq = 2(q - x),                df/dx = 2(x - q)          (f = ||q-x||^2)
//   COS: df/dq = x/(|q||x|) - f q/|q|^2,  df/dx = q/(|q||x|) - f x/|x|^2
// dq is a gather (one warp per query, k in order: deterministic).
// dx is a scatter-add into the rows that were selected:
//   atomic mode  : one warp per (i, k), FP32 atomic adds;
//   deterministic: per touched row, the entries are linked by atomics, then
//                  the row's owner (its smallest entry) sorts them by entry
//                  number and adds them in that order.
#include <climits>

#include "common.cuh"
#include "dtypes.cuh"
#include "kernels.h"

namespace tpuknn {

namespace {

struct RowSrc {
  const float* xf32;
  const void* xlp;
  int dtype, pitch, D;
  const float* xscale;
  __device__ __forceinline__ float operator()(int64_t j, int d) const {
    return xf32 ? xf32[j * D + d] : load_stored(xlp, dtype, j, pitch, d, xscale);
  }
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-pair factors for the cosine gradient: a = 1/(|q||x|), f = cosine,
// nq2 = |q|^2, nx2 = |x|^2 (all warp-uniform).
struct CosTerms {
  float a, f, nq2, nx2;
};
__device__ __forceinline__ CosTerms cos_terms(const float* q, const RowSrc& xs, int64_t j, int D,
                                              int lane) {
  float dqx = 0.f, dqq = 0.f, dxx = 0.f;
  for (int d = lane; d < D; d += 32) {
    const float qv = q[d], xv = xs(j, d);
    dqx = fmaf(qv, xv, dqx);
    dqq = fmaf(qv, qv, dqq);
    dxx = fmaf(xv, xv, dxx);
  }
  dqx = warp_sum(dqx);
  dqq = warp_sum(dqq);
  dxx = warp_sum(dxx);
  CosTerms t;
  if (dqq == 0.f || dxx == 0.f) {
    t.a = 0.f;
    t.f = 0.f;
    t.nq2 = 1.f;
    t.nx2 = 1.f;
  } else {
    const float nq = sqrtf(dqq), nx = sqrtf(dxx);
    t.a = 1.0f / (nq * nx);
    t.f = dqx * t.a;
    t.nq2 = dqq;
    t.nx2 = dxx;
  }
  return t;
}

__global__ void fill_kernel(float* __restrict__ p, int64_t n, float v) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    p[t] = v;
}
__global__ void fill_i32_kernel(int32_t* __restrict__ p, int64_t n, int32_t v) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    p[t] = v;
}

__global__ void __launch_bounds__(256)
dq_kernel(int64_t M, int D, int K, int metric, const float* __restrict__ q, RowSrc xs, int64_t N,
          const int32_t* __restrict__ idx, const float* __restrict__ g, float* __restrict__ dq) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= M) return;
  const float* qi = q + i * D;
  float* out = dq + i * D;
  for (int d = lane; d < D; d += 32) out[d] = 0.f;
  for (int k = 0; k < K; ++k) {
    const int32_t j = idx[i * K + k];
    if (j < 0 || j >= N) continue;
    const float w = g[i * K + k];
    if (metric == KNN_COS) {
      const CosTerms t = cos_terms(qi, xs, j, D, lane);
      for (int d = lane; d < D; d += 32)
        out[d] += w * (xs(j, d) * t.a - t.f * qi[d] / t.nq2);
    } else if (metric == KNN_L2) {
      for (int d = lane; d < D; d += 32) out[d] += w * 2.0f * (qi[d] - xs(j, d));
    } else {
      for (int d = lane; d < D; d += 32) out[d] += w * xs(j, d);
    }
  }
}

__device__ __forceinline__ float dfdx(int metric, float qv, float xv, const CosTerms& t) {
  if (metric == KNN_IP) return qv;
  if (metric == KNN_L2) return 2.0f * (xv - qv);
  return qv * t.a - t.f * xv / t.nx2;
}

__global__ void __launch_bounds__(256)
dx_atomic_kernel(int64_t E, int D, int K, int metric, const float* __restrict__ q, RowSrc xs,
                 int64_t N, const int32_t* __restrict__ idx, const float* __restrict__ g,
                 float* __restrict__ dx) {
  const int lane = threadIdx.x & 31;
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e >= E) return;
  const int32_t j = idx[e];
  if (j < 0 || j >= N) return;
  const float w = g[e];
  const float* qi = q + (e / K) * D;
  CosTerms t{0.f, 0.f, 1.f, 1.f};
  if (metric == KNN_COS) t = cos_terms(qi, xs, j, D, lane);
  for (int d = lane; d < D; d += 32)
    atomicAdd(&dx[(int64_t)j * D + d], w * dfdx(metric, qi[d], xs(j, d), t));
}

__global__ void link_kernel(int64_t E, const int32_t* __restrict__ idx, int64_t N,
                            int32_t* __restrict__ head, int32_t* __restrict__ minE,
                            int32_t* __restrict__ next) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int32_t j = idx[e];
  if (j < 0 || j >= N) return;
  next[e] = atomicExch(&head[j], (int32_t)e);
  atomicMin(&minE[j], (int32_t)e);
}

constexpr int kOwnCap = 512;  // entries of one row sorted in shared memory

__global__ void __launch_bounds__(128)
dx_ordered_kernel(int64_t E, int D, int K, int metric, const float* __restrict__ q, RowSrc xs,
                  int64_t N, const int32_t* __restrict__ idx, const float* __restrict__ g,
                  const int32_t* __restrict__ head, const int32_t* __restrict__ minE,
                  const int32_t* __restrict__ next, float* __restrict__ dx) {
  __shared__ int32_t buf[4][2][kOwnCap];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e0 >= E) return;
  const int32_t j = idx[e0];
  if (j < 0 || j >= N || minE[j] != (int32_t)e0) return;  // the row's owner only
  int32_t* in = buf[wib][0];
  int32_t* out = buf[wib][1];
  int cnt = 0;
  if (lane == 0) {
    for (int32_t e = head[j]; e >= 0; e = next[e]) {
      if (cnt < kOwnCap) in[cnt] = e;
      ++cnt;
    }
  }
  cnt = __shfl_sync(0xffffffffu, cnt, 0);
  __syncwarp();
  auto add_entry = [&](int32_t e) {
    const float w = g[e];
    const float* qi = q + (int64_t)(e / K) * D;
    CosTerms t{0.f, 0.f, 1.f, 1.f};
    if (metric == KNN_COS) t = cos_terms(qi, xs, j, D, lane);
    for (int d = lane; d < D; d += 32)
      dx[(int64_t)j * D + d] += w * dfdx(metric, qi[d], xs(j, d), t);
  };
  if (cnt <= kOwnCap) {
    // entry numbers are distinct: the rank of each is its position in order
    for (int u = lane; u < cnt; u += 32) {
      const int32_t me = in[u];
      int r = 0;
      for (int w = 0; w < cnt; ++w) r += in[w] < me;
      out[r] = me;
    }
    __syncwarp();
    for (int r = 0; r < cnt; ++r) add_entry(out[r]);
    return;
  }
  // very popular rows: repeated selection of the next entry number
  int32_t cur = -1;
  for (int r = 0; r < cnt; ++r) {
    int32_t best = INT_MAX;
    int u = 0;
    for (int32_t e = head[j]; e >= 0; e = next[e], ++u)
      if ((u & 31) == lane && e > cur && e < best) best = e;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    add_entry(best);
    cur = best;
  }
}

}  // namespace

size_t backward_ws_bytes(int64_t N, int64_t M, int K, int deterministic) {
  if (!deterministic) return 0;
  return (size_t)round_up(N * 4, 256) * 2 + (size_t)round_up(M * K * 4, 256);
}

cudaError_t launch_backward(int64_t M, int D, int K, int metric, const float* q,
                            const float* xf32, const void* xlp, int dtype, int pitch,
                            const float* xscale, int64_t N, const int32_t* idx,
                            const float* g, float* dq, float* dx, int zero_dx, int deterministic,
                            void* ws, cudaStream_t st) {
  RowSrc xs{xf32, xlp, dtype, pitch, D, xscale};
  const int64_t E = M * K;
  const int sms = device_sm_count();
  if (dx && zero_dx) {
    fill_kernel<<<sms * 8, 256, 0, st>>>(dx, N * (int64_t)D, 0.0f);
  }
  if (dq && M > 0) {
    dq_kernel<<<(unsigned)cdiv(M * 32, 256), 256, 0, st>>>(M, D, K, metric, q, xs, N, idx, g, dq);
  }
  if (dx && E > 0) {
    if (!deterministic) {
      dx_atomic_kernel<<<(unsigned)cdiv(E * 32, 256), 256, 0, st>>>(E, D, K, metric, q, xs, N, idx,
                                                                    g, dx);
    } else {
      char* w = reinterpret_cast<char*>(ws);
      int32_t* head = reinterpret_cast<int32_t*>(w);
      int32_t* minE = reinterpret_cast<int32_t*>(w + round_up(N * 4, 256));
      int32_t* next = reinterpret_cast<int32_t*>(w + 2 * round_up(N * 4, 256));
      fill_i32_kernel<<<sms * 4, 256, 0, st>>>(head, N, -1);
      fill_i32_kernel<<<sms * 4, 256, 0, st>>>(minE, N, INT_MAX);
      link_kernel<<<(unsigned)cdiv(E, 256), 256, 0, st>>>(E, idx, N, head, minE, next);
      dx_ordered_kernel<<<(unsigned)cdiv(E * 32, 128), 128, 0, st>>>(E, D, K, metric, q, xs, N, idx,
                                                                     g, head, minE, next, dx);
    }
  }
  return cudaGetLastError();
}

}  // namespace tpuknn
