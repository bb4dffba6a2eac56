// approx_max_k.cu -- the approx_max_k / approx_min_k operator on a score
// matrix the caller already holds (App. A.1: the operator behind Alg. 1,
// without the fused contraction). For every row i of S (M x N, FP32 or BF16,
// row-major) and bin l it keeps the best score and its column, bins j mod L
// or L balanced runs of consecutive columns; optionally ExactRescoring then
// keeps the best K of the L winners (aggregate_to_topk).
//
// The operator reads every score once and is HBM-bound. Bin winners merge in
// an M x L array of ordered 64-bit keys (score, ~column) by atomicMax, so ties
// keep the smaller column whatever the order of the CTAs; approx_min_k
// negates the scores on the way in and the values on the way out.
#include <algorithm>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace tpuknn {

namespace {

// The score, negated for approx_min_k; adding +0 turns -0 into +0, so that
// the two zeros make equal keys and tie to the smaller column.
template <int DT>
__device__ __forceinline__ float load_score(const void* S, int64_t t, float sg) {
  const float v = DT == KNN_BF16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(S)[t])
                                 : reinterpret_cast<const float*>(S)[t];
  return sg * v + 0.0f;
}

// Bins j mod L: thread b of a row owns bin b and walks its columns b, b + L,
// ... of a chunk of kchunk grid rows; neighbouring threads read neighbouring
// columns, so every pass over a grid row is one coalesced sweep.
template <int DT>
__global__ void __launch_bounds__(256)
bin_max_mod_kernel(const void* __restrict__ S, int64_t N, int64_t L, int64_t kchunk, int neg,
                   unsigned long long* __restrict__ G) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (b >= L) return;
  const int64_t k0 = (int64_t)blockIdx.z * kchunk;
  const int64_t k1 = min(cdiv(N, L), k0 + kchunk);
  const float sg = neg ? -1.0f : 1.0f;
  uint64_t best = 0;
  // eight independent loads in flight per thread
  for (int64_t k = k0; k < k1; k += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t j = (k + u) * L + b;
      v[u] = (k + u < k1 && j < N) ? load_score<DT>(S, i * N + j, sg) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t j = (k + u) * L + b;
      if (k + u < k1 && j < N) {
        const uint64_t key = make_key(v[u], (int32_t)j);
        best = key > best ? key : best;
      }
    }
  }
  if (best) atomicMax(&G[i * L + b], (unsigned long long)best);
}

// The same with 16-byte loads (L and N multiples of the V columns a load holds,
// S 16-byte aligned): thread (x, y) of a CTA owns bins V*t .. V*t + V - 1,
// t = blockIdx.x * blockDim.x + x, of row blockIdx.y * blockDim.y + y, and
// keeps each bin's best value and column (strict '>' in increasing column
// order keeps the smaller column on ties; the keys made at the end merge
// across CTAs by atomicMax). A warp reads 32 consecutive 16-byte pieces of a
// grid row, and each thread has four loads in flight.
template <int DT>
__global__ void __launch_bounds__(256)
bin_max_mod_vec_kernel(const void* __restrict__ S, int64_t M, int64_t N, int64_t L,
                       int64_t kchunk, int neg, unsigned long long* __restrict__ G) {
  constexpr int V = DT == KNN_BF16 ? 8 : 4;  // columns per 16-byte load
  constexpr int kEsz = DT == KNN_BF16 ? 2 : 4;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
  if (t * V >= L || i >= M) return;
  const int64_t k0 = (int64_t)blockIdx.z * kchunk;
  const int64_t k1 = min(cdiv(N, L), k0 + kchunk);
  const float sg = neg ? -1.0f : 1.0f;
  const char* row = static_cast<const char*>(S) + i * N * kEsz;
  float bv[V];
  int32_t bj[V];
#pragma unroll
  for (int c = 0; c < V; ++c) {
    bv[c] = neg_inf();
    bj[c] = -1;
  }
  for (int64_t k = k0; k < k1; k += 4) {
    uint4 raw[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t j0 = (k + u) * L + t * V;
      raw[u] = (k + u < k1 && j0 < N)
                   ? __ldg(reinterpret_cast<const uint4*>(row + j0 * kEsz))
                   : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t j0 = (k + u) * L + t * V;
      if (k + u < k1 && j0 < N) {
        float x[V];
        if constexpr (DT == KNN_BF16) {
          const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&raw[u]);
#pragma unroll
          for (int c = 0; c < V; ++c) x[c] = __bfloat162float(h[c]);
        } else {
          const float* f = reinterpret_cast<const float*>(&raw[u]);
#pragma unroll
          for (int c = 0; c < V; ++c) x[c] = f[c];
        }
#pragma unroll
        for (int c = 0; c < V; ++c) {
          const float v = sg * x[c] + 0.0f;
          if (bj[c] < 0 || v > bv[c]) {
            bv[c] = v;
            bj[c] = (int32_t)(j0 + c);
          }
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < V; ++c)
    if (bj[c] >= 0) atomicMax(&G[i * L + t * V + c], (unsigned long long)make_key(bv[c], bj[c]));
}

__device__ __forceinline__ int64_t runs_bin_of(int64_t j, int64_t q, int64_t r) {
  const int64_t big = r * (q + 1);
  return j < big ? j / (q + 1) : r + (j - big) / q;
}

// Contiguous bins: a CTA sweeps `chunk` consecutive columns of one row; a
// thread keeps the best of its current bin and merges it when its columns
// (blockDim apart) move to another bin.
template <int DT>
__global__ void __launch_bounds__(256)
bin_max_runs_kernel(const void* __restrict__ S, int64_t N, int64_t L, int64_t chunk, int neg,
                    unsigned long long* __restrict__ G) {
  const int64_t i = blockIdx.y;
  const int64_t j0 = (int64_t)blockIdx.x * chunk;
  const int64_t j1 = min(N, j0 + chunk);
  const int64_t q = N / L, r = N % L;
  const float sg = neg ? -1.0f : 1.0f;
  int64_t cur = -1, end = 0;
  uint64_t best = 0;
  const int64_t step = blockDim.x;
  for (int64_t j8 = j0 + threadIdx.x; j8 < j1; j8 += 8 * step) {
    // eight independent loads in flight per thread
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t j = j8 + u * step;
      v[u] = j < j1 ? load_score<DT>(S, i * N + j, sg) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t j = j8 + u * step;
      if (j < j1) {
        if (j >= end) {
          if (best) atomicMax(&G[i * L + cur], (unsigned long long)best);
          cur = runs_bin_of(j, q, r);
          end = (cur + 1) * q + min(cur + 1, r);
          best = 0;
        }
        const uint64_t key = make_key(v[u], (int32_t)j);
        best = key > best ? key : best;
      }
    }
  }
  if (best) atomicMax(&G[i * L + cur], (unsigned long long)best);
}

// The same with 16-byte loads (N a multiple of the V columns a load holds, S
// 16-byte aligned): a thread reads V consecutive columns at a time, blockDim
// * V columns apart, and keeps the best value and column of its current bin.
template <int DT>
__global__ void __launch_bounds__(256)
bin_max_runs_vec_kernel(const void* __restrict__ S, int64_t N, int64_t L, int64_t chunk, int neg,
                        unsigned long long* __restrict__ G) {
  constexpr int V = DT == KNN_BF16 ? 8 : 4;
  constexpr int kEsz = DT == KNN_BF16 ? 2 : 4;
  const int64_t i = blockIdx.y;
  const int64_t j0 = (int64_t)blockIdx.x * chunk;
  const int64_t j1 = min(N, j0 + chunk);
  const int64_t q = N / L, r = N % L;
  const float sg = neg ? -1.0f : 1.0f;
  const char* row = static_cast<const char*>(S) + i * N * kEsz;
  int64_t cur = -1, end = 0;
  float bv = neg_inf();
  int32_t bj = -1;
  auto flush = [&]() {
    if (bj >= 0) atomicMax(&G[i * L + cur], (unsigned long long)make_key(bv, bj));
  };
  const int64_t step = (int64_t)blockDim.x * V;
  for (int64_t jv = j0 + (int64_t)threadIdx.x * V; jv < j1; jv += 4 * step) {
    uint4 raw[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t j = jv + u * step;
      raw[u] = j < j1 ? __ldg(reinterpret_cast<const uint4*>(row + j * kEsz))
                      : make_uint4(0, 0, 0, 0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t j = jv + u * step;
      if (j < j1) {
        float x[V];
        if constexpr (DT == KNN_BF16) {
          const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&raw[u]);
#pragma unroll
          for (int c = 0; c < V; ++c) x[c] = __bfloat162float(h[c]);
        } else {
          const float* f = reinterpret_cast<const float*>(&raw[u]);
#pragma unroll
          for (int c = 0; c < V; ++c) x[c] = f[c];
        }
#pragma unroll
        for (int c = 0; c < V; ++c) {
          const int64_t jj = j + c;
          if (jj >= end) {
            flush();
            cur = runs_bin_of(jj, q, r);
            end = (cur + 1) * q + min(cur + 1, r);
            bv = neg_inf();
            bj = -1;
          }
          const float v = sg * x[c] + 0.0f;
          if (bj < 0 || v > bv) {
            bv = v;
            bj = (int32_t)jj;
          }
        }
      }
    }
  }
  flush();
}

// Keys to (value, index) pairs, values back in the caller's orientation.
__global__ void keys_to_pairs_kernel(const uint64_t* __restrict__ keys, int64_t n, int neg,
                                     float* __restrict__ out_v, int32_t* __restrict__ out_a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint64_t k = keys[t];
  out_v[t] = k ? (neg ? -key_score(k) : key_score(k)) : __int_as_float(0x7fc00000);
  out_a[t] = k ? key_index(k) : -1;
}

}  // namespace

cudaError_t launch_bin_max(const void* S, int dtype, int64_t M, int64_t N, int64_t L, int bin_map,
                           int neg, unsigned long long* G, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (M > 65535) {
    // grid y holds at most 65535 rows: split the rows
    const int esz = dtype == KNN_BF16 ? 2 : 4;
    for (int64_t m0 = 0; m0 < M; m0 += 65535) {
      const int64_t mc = min((int64_t)65535, M - m0);
      cudaError_t e = launch_bin_max(static_cast<const char*>(S) + m0 * N * esz, dtype, mc, N, L,
                                     bin_map, neg, G + m0 * L, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  const int sms = device_sm_count();
  const int vcols = dtype == KNN_BF16 ? 8 : 4;
  if (bin_map == KNN_BINS_MOD && L % vcols == 0 && N % vcols == 0 &&
      (reinterpret_cast<uintptr_t>(S) & 15) == 0) {
    // 16-byte loads: a CTA is rows x threads, the threads of a row covering
    // its L / vcols vectors of a grid row
    const int64_t tpr = L / vcols;
    const int bdx = (int)std::min<int64_t>(256, round_up(tpr, 32));
    const int bdy = 256 / bdx;
    const int64_t bx = cdiv(tpr, bdx), by = cdiv(M, bdy);
    const int64_t grid_rows = cdiv(N, L);
    int64_t kz = cdiv((int64_t)sms * 8, bx * by);
    if (kz > grid_rows) kz = grid_rows;
    if (kz < 1) kz = 1;
    if (kz > 65535) kz = 65535;
    const int64_t kchunk = cdiv(grid_rows, kz);
    kz = cdiv(grid_rows, kchunk);
    if (bx > 0x7fffffffLL || by > 65535) return cudaErrorInvalidValue;
    dim3 grid((unsigned)bx, (unsigned)by, (unsigned)kz), block((unsigned)bdx, (unsigned)bdy);
    if (dtype == KNN_BF16)
      bin_max_mod_vec_kernel<KNN_BF16><<<grid, block, 0, st>>>(S, M, N, L, kchunk, neg, G);
    else
      bin_max_mod_vec_kernel<KNN_F32><<<grid, block, 0, st>>>(S, M, N, L, kchunk, neg, G);
  } else if (bin_map == KNN_BINS_MOD) {
    const int64_t grid_rows = cdiv(N, L);
    const int64_t bx = cdiv(L, 256);
    // enough CTAs to fill the GPU a few times over
    int64_t kz = cdiv((int64_t)sms * 8, bx * M);
    if (kz > grid_rows) kz = grid_rows;
    if (kz < 1) kz = 1;
    if (kz > 65535) kz = 65535;
    const int64_t kchunk = cdiv(grid_rows, kz);
    kz = cdiv(grid_rows, kchunk);
    dim3 grid((unsigned)bx, (unsigned)M, (unsigned)kz);
    if (dtype == KNN_BF16)
      bin_max_mod_kernel<KNN_BF16><<<grid, 256, 0, st>>>(S, N, L, kchunk, neg, G);
    else
      bin_max_mod_kernel<KNN_F32><<<grid, 256, 0, st>>>(S, N, L, kchunk, neg, G);
  } else {
    const bool vec = N % vcols == 0 && (reinterpret_cast<uintptr_t>(S) & 15) == 0;
    // columns per CTA: 32 vectors per thread, or 32 columns per thread
    const int64_t chunk = 256 * 32 * (vec ? vcols : 1);
    const int64_t bx = cdiv(N, chunk);
    if (bx > 0x7fffffffLL) return cudaErrorInvalidValue;
    dim3 grid((unsigned)bx, (unsigned)M);
    if (vec) {
      if (dtype == KNN_BF16)
        bin_max_runs_vec_kernel<KNN_BF16><<<grid, 256, 0, st>>>(S, N, L, chunk, neg, G);
      else
        bin_max_runs_vec_kernel<KNN_F32><<<grid, 256, 0, st>>>(S, N, L, chunk, neg, G);
    } else if (dtype == KNN_BF16) {
      bin_max_runs_kernel<KNN_BF16><<<grid, 256, 0, st>>>(S, N, L, chunk, neg, G);
    } else {
      bin_max_runs_kernel<KNN_F32><<<grid, 256, 0, st>>>(S, N, L, chunk, neg, G);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_keys_to_pairs(const uint64_t* keys, int64_t n, int neg, float* out_v,
                                 int32_t* out_a, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  keys_to_pairs_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(keys, n, neg, out_v, out_a);
  return cudaGetLastError();
}

}  // namespace tpuknn
