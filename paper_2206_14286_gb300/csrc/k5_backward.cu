// k5_backward.cu -- gradient of the selected values with respect to the
// queries and the database rows (the differentiation pattern).
//
// With the selected indices held constant, for F = sum_{i,k} g[i,k] f(q_i, x_j),
// j = idx[i,k], f the reported value:
//   IP : df/dq = x,                       df/dx = q
//   L2 : df/dq = 2(q - x),                df/dx = 2(x - q)          (f = ||q-x||^2)
//   COS: df/dq = x/(|q||x|) - f q/|q|^2,  df/dx = q/(|q||x|) - f x/|x|^2
// dq is a gather (one warp per query, k in order: deterministic).
// dx is a scatter-add into the rows that were selected, two ways:
//   row path     : (deterministic; taken with a workspace for a zero-filled dx,
//                  or when asked) the entries of each row are linked by
//                  atomics and the touched rows listed; then one launch
//                  writes zeros into the untouched rows (if dx is to be
//                  zeroed), sums each touched row's entries in entry-number
//                  order (from zero or from the row's current values) and
//                  writes the row once, and computes dq, in separate blocks;
//   atomic path  : zero fill if asked, then one warp per (i, k) with FP32
//                  atomic adds (16-byte vector adds when D is a multiple of 4
//                  and the rows are aligned).
#include <algorithm>
#include <climits>
#include <cstdint>

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

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

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
__global__ void zero4_kernel(float4* __restrict__ p, int64_t n4) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n4;
       t += (int64_t)gridDim.x * blockDim.x)
    p[t] = make_float4(0.f, 0.f, 0.f, 0.f);
}
// Empty lists (head = -1) and an empty list of touched rows.
__global__ void links_init_kernel(int32_t* __restrict__ head, int64_t n,
                                  int32_t* __restrict__ ntouched) {
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t0 == 0) *ntouched = 0;
  for (int64_t t = t0; t < n; t += (int64_t)gridDim.x * blockDim.x) head[t] = -1;
}

// Columns of one chunk that a lane owns: d = c0 + lane + 32 t, t < kCols.
constexpr int kCols = 8;
constexpr int kChunk = 32 * kCols;

// dq of query i, k in order. The chunk's partial sums stay in registers while
// the rows of four neighbours are loaded at once (the loads of a row do not
// wait for the previous row's adds), and the chunk is written once.
template <int METRIC>
__device__ __forceinline__ void dq_row(int64_t i, int D, int K, const float* __restrict__ q,
                                       const RowSrc& xs, int64_t N,
                                       const int32_t* __restrict__ idx,
                                       const float* __restrict__ g, float* __restrict__ dq) {
  const int lane = threadIdx.x & 31;
  const float* qi = q + i * D;
  for (int c0 = 0; c0 < D; c0 += kChunk) {
    float acc[kCols], qv[kCols];
#pragma unroll
    for (int t = 0; t < kCols; ++t) {
      const int d = c0 + lane + 32 * t;
      acc[t] = 0.f;
      qv[t] = (METRIC != KNN_IP && d < D) ? qi[d] : 0.f;
    }
    for (int kb = 0; kb < K; kb += 32) {
      const int nk = min(32, K - kb);
      int32_t jl = -1;
      float wl = 0.f;
      if (lane < nk) {
        jl = idx[i * K + kb + lane];
        wl = g[i * K + kb + lane];
      }
      for (int k0 = 0; k0 < nk; k0 += 4) {
        int32_t jj[4];
        float ww[4], xv[4][kCols];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          jj[u] = __shfl_sync(0xffffffffu, jl, k0 + u);  // lanes >= nk hold -1
          ww[u] = __shfl_sync(0xffffffffu, wl, k0 + u);
          const bool ok = jj[u] >= 0 && jj[u] < N;
#pragma unroll
          for (int t = 0; t < kCols; ++t) {
            const int d = c0 + lane + 32 * t;
            xv[u][t] = (ok && d < D) ? xs(jj[u], d) : 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (jj[u] < 0 || jj[u] >= N) continue;  // warp-uniform
          if (METRIC == KNN_COS) {
            const CosTerms ct = cos_terms(qi, xs, jj[u], D, lane);
#pragma unroll
            for (int t = 0; t < kCols; ++t)
              acc[t] += ww[u] * (xv[u][t] * ct.a - ct.f * qv[t] / ct.nq2);
          } else if (METRIC == KNN_L2) {
#pragma unroll
            for (int t = 0; t < kCols; ++t) acc[t] += ww[u] * 2.0f * (qv[t] - xv[u][t]);
          } else {
#pragma unroll
            for (int t = 0; t < kCols; ++t) acc[t] += ww[u] * xv[u][t];
          }
        }
      }
    }
#pragma unroll
    for (int t = 0; t < kCols; ++t) {
      const int d = c0 + lane + 32 * t;
      if (d < D) dq[i * D + d] = acc[t];
    }
  }
}

template <int METRIC>
__global__ void __launch_bounds__(256)
dq_kernel(int64_t M, int D, int K, const float* __restrict__ q, RowSrc xs, int64_t N,
          const int32_t* __restrict__ idx, const float* __restrict__ g, float* __restrict__ dq) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i < M) dq_row<METRIC>(i, D, K, q, xs, N, idx, g, dq);
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

// The same scatter with one 16-byte atomic add per four columns (rows of dx
// and q 16-byte aligned, D a multiple of 4): a quarter of the atomic operations.
template <int METRIC>
__global__ void __launch_bounds__(256)
dx_atomic4_kernel(int64_t E, int D, int K, const float* __restrict__ q, RowSrc xs, int64_t N,
                  const int32_t* __restrict__ idx, const float* __restrict__ g,
                  float* __restrict__ dx) {
  const int lane = threadIdx.x & 31;
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e >= E) return;
  const int32_t j = idx[e];
  if (j < 0 || j >= N) return;
  const float w = g[e];
  const float* qi = q + (e / K) * D;
  CosTerms t{0.f, 0.f, 1.f, 1.f};
  if (METRIC == KNN_COS) t = cos_terms(qi, xs, j, D, lane);
  for (int d = 4 * lane; d < D; d += 128) {
    const float4 qv = *reinterpret_cast<const float4*>(qi + d);
    float4 v;
    if (METRIC == KNN_IP) {
      v = make_float4(w * qv.x, w * qv.y, w * qv.z, w * qv.w);
    } else {
      v.x = w * dfdx(METRIC, qv.x, xs(j, d), t);
      v.y = w * dfdx(METRIC, qv.y, xs(j, d + 1), t);
      v.z = w * dfdx(METRIC, qv.z, xs(j, d + 2), t);
      v.w = w * dfdx(METRIC, qv.w, xs(j, d + 3), t);
    }
    atomicAdd(reinterpret_cast<float4*>(dx + (int64_t)j * D + d), v);
  }
}

// Entry e joins the list of its row (head / next); the first entry of a row
// to arrive appends the row to the list of touched rows, one atomic add on
// the count per warp (a single counter would serialise an add per row).
__global__ void link_kernel(int64_t E, const int32_t* __restrict__ idx, int64_t N,
                            int32_t* __restrict__ head, int32_t* __restrict__ next,
                            int32_t* __restrict__ touched, int32_t* __restrict__ ntouched) {
  const int lane = threadIdx.x & 31;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t j = e < E ? idx[e] : -1;
  bool first = false;
  if (j >= 0 && j < N) {
    const int32_t prev = atomicExch(&head[j], (int32_t)e);
    next[e] = prev;
    first = prev < 0;
  }
  const unsigned m = __ballot_sync(0xffffffffu, first);
  if (m == 0) return;
  const int leader = __ffs(m) - 1;
  int32_t base = 0;
  if (lane == leader) base = atomicAdd(ntouched, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (first) touched[base + __popc(m & ((1u << lane) - 1u))] = j;
}

// Zeros into the rows of dx that no entry selected (head < 0): each of
// nwarps warps takes 32 consecutive rows at a time, reads their list heads in one load
// (the next batch's heads are loaded before this batch's stores) and writes
// the empty rows, 16-byte stores when VEC. Rows with entries are left to
// touched_rows, so the two write disjoint rows.
template <bool VEC>
__device__ __forceinline__ void zero_untouched(int64_t warp, int64_t nwarps, int64_t N, int D,
                                               const int32_t* __restrict__ head,
                                               float* __restrict__ dx) {
  const int lane = threadIdx.x & 31;
  const int64_t step = nwarps * 32;
  int64_t j0 = warp * 32;
  int32_t hl = j0 + lane < N ? head[j0 + lane] : 0;
  for (; j0 < N; j0 += step) {
    unsigned zero = __ballot_sync(0xffffffffu, j0 + lane < N && hl < 0);
    const int64_t jn = j0 + step + lane;
    hl = jn < N ? head[jn] : 0;
    while (zero) {
      float* row = dx + (j0 + __ffs(zero) - 1) * D;
      zero &= zero - 1;
      if (VEC) {
        for (int d = 4 * lane; d < D; d += 128)
          *reinterpret_cast<float4*>(row + d) = make_float4(0.f, 0.f, 0.f, 0.f);
      } else {
        for (int d = lane; d < D; d += 32) row[d] = 0.f;
      }
    }
  }
}

// The rows with entries, written once each, deterministically: each of
// nwarps warps takes kTouchBatch rows of the touched list at a time; the lane of each row walks
// that row's list, keeping up to kRowCap entry numbers in ascending order
// (insertion) with their weights in shared memory, all walks at once. Then
// the whole warp sums each row's entries in entry-number order, in
// registers, starting from zero (ZERO) or from the row's current values,
// kRowPar rows side by side (their loads in flight together), and stores
// the rows. Rows
// with more than kRowCap entries take the slow way (zeros if ZERO, then the
// entries added in order by repeated selection of the next entry number).
// VEC: D a multiple of 4, dx and q 16-byte aligned; a lane owns 4 adjacent
// columns of each 128.
constexpr int kRowCap = 8;
constexpr int kTouchBatch = 16;
constexpr int kRowPar = 4;  // touched rows summed side by side

// The warp's shared memory for touched_rows; stride kRowCap + 1 words
// between lanes: no bank conflicts.
struct TouchSmem {
  int32_t ent[kTouchBatch][kRowCap + 1];
  float wgt[kTouchBatch][kRowCap + 1];
};

template <int METRIC, bool VEC, bool ZERO>
__device__ __forceinline__ void touched_rows(int64_t warp, int64_t nwarps, TouchSmem& sm, int D,
                                             int K, const float* __restrict__ q, const RowSrc& xs,
                                             const float* __restrict__ g,
                                             const int32_t* __restrict__ head,
                                             const int32_t* __restrict__ next,
                                             const int32_t* __restrict__ touched,
                                             const int32_t* __restrict__ ntouched,
                                             float* __restrict__ dx) {
  const int lane = threadIdx.x & 31;
  const int64_t T = *ntouched;
  auto col = [&](int c0, int u) {
    return VEC ? c0 + 4 * lane + 128 * (u >> 2) + (u & 3) : c0 + lane + 32 * u;
  };
  for (int64_t t0 = warp * kTouchBatch; t0 < T; t0 += nwarps * kTouchBatch) {
    const bool mine_row = lane < kTouchBatch && t0 + lane < T;
    const int32_t jl = mine_row ? touched[t0 + lane] : -1;
    const int32_t hl = mine_row ? head[jl] : -1;
    int cnt = 0;
    if (mine_row) {
      int32_t* mine = sm.ent[lane];
      for (int32_t e = hl; e >= 0; e = next[e]) {
        if (cnt < kRowCap) {
          int p = cnt;
          while (p > 0 && mine[p - 1] > e) {
            mine[p] = mine[p - 1];
            --p;
          }
          mine[p] = e;
        }
        ++cnt;
      }
#pragma unroll
      for (int r = 0; r < kRowCap; ++r)  // loads issued together
        if (r < cnt) sm.wgt[lane][r] = g[mine[r]];
    }
    __syncwarp();
    // rows with at most kRowCap entries, kRowPar at a time (their loads in
    // flight together); each row's entries in entry-number order
    unsigned fast = __ballot_sync(0xffffffffu, mine_row && cnt <= kRowCap);
    unsigned slow = __ballot_sync(0xffffffffu, mine_row && cnt > kRowCap);
    while (fast) {
      int rr[kRowPar], cc[kRowPar];
      int64_t jj[kRowPar];
      int cmax = 0;
#pragma unroll
      for (int p = 0; p < kRowPar; ++p) {
        const int r0 = fast ? __ffs(fast) - 1 : -1;
        if (fast) fast &= fast - 1;
        rr[p] = r0;
        jj[p] = __shfl_sync(0xffffffffu, jl, r0 < 0 ? 0 : r0);
        cc[p] = r0 < 0 ? 0 : __shfl_sync(0xffffffffu, cnt, r0 < 0 ? 0 : r0);
        cmax = max(cmax, cc[p]);
      }
      for (int c0 = 0; c0 < D; c0 += kChunk) {
        float acc[kRowPar][kCols], xv[kRowPar][kCols];
#pragma unroll
        for (int p = 0; p < kRowPar; ++p) {
#pragma unroll
          for (int u = 0; u < kCols; ++u) {
            const int d = col(c0, u);
            const bool ok = cc[p] > 0 && d < D;
            acc[p][u] = (!ZERO && ok) ? dx[jj[p] * D + d] : 0.f;
            xv[p][u] = (METRIC != KNN_IP && ok) ? xs(jj[p], d) : 0.f;
          }
        }
        for (int r = 0; r < cmax; ++r) {
          float qv[kRowPar][kCols];
          const float* qi[kRowPar];
#pragma unroll
          for (int p = 0; p < kRowPar; ++p) {
            const bool ok = r < cc[p];
            qi[p] = q + (int64_t)((ok ? sm.ent[rr[p]][r] : 0) / K) * D;
#pragma unroll
            for (int u = 0; u < kCols; ++u) {
              const int d = col(c0, u);
              qv[p][u] = (ok && d < D) ? qi[p][d] : 0.f;
            }
          }
#pragma unroll
          for (int p = 0; p < kRowPar; ++p) {
            if (r >= cc[p]) continue;  // warp-uniform
            const float w = sm.wgt[rr[p]][r];
            CosTerms t{0.f, 0.f, 1.f, 1.f};
            if (METRIC == KNN_COS) t = cos_terms(qi[p], xs, jj[p], D, lane);
#pragma unroll
            for (int u = 0; u < kCols; ++u) acc[p][u] += w * dfdx(METRIC, qv[p][u], xv[p][u], t);
          }
        }
#pragma unroll
        for (int p = 0; p < kRowPar; ++p) {
          if (cc[p] == 0) continue;
#pragma unroll
          for (int u = 0; u < kCols; ++u) {
            const int d = col(c0, u);
            if (d < D) dx[jj[p] * D + d] = acc[p][u];
          }
        }
      }
    }
    // rows with more entries: zeros if ZERO, then the entries in order by
    // repeated selection of the next entry number, added by the lane owning
    // each column (the same lane that wrote its zero)
    while (slow) {
      const int r0 = __ffs(slow) - 1;
      slow &= slow - 1;
      const int64_t j = __shfl_sync(0xffffffffu, jl, r0);
      const int c = __shfl_sync(0xffffffffu, cnt, r0);
      const int32_t h = __shfl_sync(0xffffffffu, hl, r0);
      float* row = dx + j * D;
      if (ZERO)
        for (int d = lane; d < D; d += 32) row[d] = 0.f;
      int32_t cur = -1;
      for (int r = 0; r < c; ++r) {
        int32_t best = INT_MAX;
        int u = 0;
        for (int32_t e = h; e >= 0; e = next[e], ++u)
          if ((u & 31) == lane && e > cur && e < best) best = e;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
        const float w = g[best];
        const float* qi = q + (int64_t)(best / K) * D;
        CosTerms t{0.f, 0.f, 1.f, 1.f};
        if (METRIC == KNN_COS) t = cos_terms(qi, xs, j, D, lane);
        for (int d = lane; d < D; d += 32) row[d] += w * dfdx(METRIC, qi[d], xs(j, d), t);
        cur = best;
      }
    }
    __syncwarp();
  }
}

// Everything of a backward with a workspace after the lists are built, in
// one launch of three kinds of blocks that write disjoint memory:
//   [0, nz)            zeros into the untouched rows (ZERO; persistent);
//   [nz, nz + nt)      the touched rows (persistent over the touched list);
//   [nz + nt, ...)     dq, one query per warp.
// The zero fill is bound by HBM writes, the other two by the latency of their
// dependent loads, so they run side by side instead of one after another.
struct BwdArgs {
  int64_t M, N;
  int D, K;
  const float* q;
  RowSrc xs;
  const int32_t* idx;
  const float* g;
  const int32_t *head, *next, *touched, *ntouched;
  float *dq, *dx;
};

template <int METRIC, bool VEC, bool ZERO>
__global__ void __launch_bounds__(256)
backward_rows_kernel(BwdArgs a, int nz, int nt) {
  __shared__ TouchSmem sm[8];
  const int wib = threadIdx.x >> 5;
  const int64_t b = blockIdx.x;
  if (b < nz) {
    if (ZERO) zero_untouched<VEC>(b * 8 + wib, (int64_t)nz * 8, a.N, a.D, a.head, a.dx);
    return;
  }
  if (b < nz + nt) {
    touched_rows<METRIC, VEC, ZERO>((b - nz) * 8 + wib, (int64_t)nt * 8, sm[wib], a.D, a.K, a.q,
                                    a.xs, a.g, a.head, a.next, a.touched, a.ntouched, a.dx);
    return;
  }
  const int64_t i = (b - nz - nt) * 8 + wib;
  if (i < a.M) dq_row<METRIC>(i, a.D, a.K, a.q, a.xs, a.N, a.idx, a.g, a.dq);
}

// Resident blocks per SM of a kernel at 256 threads (cached per kernel).
template <typename Kern>
int blocks_per_sm(Kern kern, int* cache) {
  if (*cache == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, 256, 0) != cudaSuccess || b < 1)
      b = 1;
    *cache = b;
  }
  return *cache;
}

template <int METRIC, bool ZERO>
void launch_backward_rows(const BwdArgs& a, bool vec, int sms, cudaStream_t st) {
  static int per_sm[2] = {0, 0};
  auto kern = vec ? backward_rows_kernel<METRIC, true, ZERO>
                  : backward_rows_kernel<METRIC, false, ZERO>;
  const int64_t wave = (int64_t)sms * blocks_per_sm(kern, &per_sm[vec]);
  // the zero fill keeps two thirds of the resident blocks (it needs the
  // warps to keep HBM busy with writes; a third measured 0.19 against 0.13 ms
  // for 1 GB); the touched rows get the other third, or the whole wave
  // without the fill (fewer blocks if the list cannot fill them); dq one
  // block per 8 queries, in the slots that free up
  const int64_t rows_max = std::min(a.N, a.M * a.K);
  const int nz =
      ZERO ? (int)std::max<int64_t>(1, std::min<int64_t>(wave * 2 / 3, cdiv(cdiv(a.N, 32), 8)))
           : 0;
  const int nt = (int)std::max<int64_t>(
      1, std::min<int64_t>(ZERO ? wave / 3 : wave, cdiv(cdiv(rows_max, kTouchBatch), 8)));
  const int64_t nq = a.dq ? cdiv(a.M, 8) : 0;
  kern<<<(unsigned)(nz + nt + nq), 256, 0, st>>>(a, nz, nt);
}

template <bool ZERO>
void launch_backward_rows_metric(int metric, const BwdArgs& a, bool vec, int sms,
                                 cudaStream_t st) {
  if (metric == KNN_IP)
    launch_backward_rows<KNN_IP, ZERO>(a, vec, sms, st);
  else if (metric == KNN_L2)
    launch_backward_rows<KNN_L2, ZERO>(a, vec, sms, st);
  else
    launch_backward_rows<KNN_COS, ZERO>(a, vec, sms, st);
}

void launch_fill_zero(float* p, int64_t n, int sms, cudaStream_t st) {
  if (n % 4 == 0 && aligned16(p))
    zero4_kernel<<<sms * 8, 256, 0, st>>>(reinterpret_cast<float4*>(p), n / 4);
  else
    fill_kernel<<<sms * 8, 256, 0, st>>>(p, n, 0.0f);
}

// Workspace of the row path: list heads (N), links (E), touched rows
// (min(N, E)), and the touched count.
struct Links {
  int32_t *head, *next, *touched, *ntouched;
};
Links links_in(void* ws, int64_t N, int64_t E) {
  char* w = reinterpret_cast<char*>(ws);
  Links l;
  l.head = reinterpret_cast<int32_t*>(w);
  w += round_up(N * 4, 256);
  l.next = reinterpret_cast<int32_t*>(w);
  w += round_up(E * 4, 256);
  l.touched = reinterpret_cast<int32_t*>(w);
  w += round_up(std::min(N, E) * 4, 256);
  l.ntouched = reinterpret_cast<int32_t*>(w);
  return l;
}

}  // namespace

size_t backward_ws_bytes(int64_t N, int64_t M, int K) {
  const int64_t E = M * K;
  return (size_t)(round_up(N * 4, 256) + round_up(E * 4, 256) + round_up(std::min(N, E) * 4, 256) +
                  256);
}

cudaError_t launch_backward(int64_t M, int D, int K, int metric, const float* q,
                            const float* xf32, const void* xlp, int dtype, int pitch,
                            const float* xscale, int64_t N, const int32_t* idx,
                            const float* g, float* dq, float* dx, int zero_dx, int deterministic,
                            void* ws, cudaStream_t st) {
  RowSrc xs{xf32, xlp, dtype, pitch, D, xscale};
  const int64_t E = M * K;
  const int sms = device_sm_count();
  // row path (deterministic): with a workspace when dx is zero-filled (one
  // launch; faster than fill + atomics), or when asked to be deterministic.
  // Otherwise zero fill (if asked) and FP32 atomic adds (adding into an
  // existing dx, the atomics' read-modify-write in L2 is the faster way).
  if (dx && ws && E > 0 && (zero_dx || deterministic)) {
    const Links l = links_in(ws, N, E);
    links_init_kernel<<<sms * 4, 256, 0, st>>>(l.head, N, l.ntouched);
    link_kernel<<<(unsigned)cdiv(E, 256), 256, 0, st>>>(E, idx, N, l.head, l.next, l.touched,
                                                        l.ntouched);
    const BwdArgs a{M, N, D, K, q, xs, idx, g, l.head, l.next, l.touched, l.ntouched, dq, dx};
    const bool vec = D % 4 == 0 && aligned16(dx) && aligned16(q);
    if (zero_dx)
      launch_backward_rows_metric<true>(metric, a, vec, sms, st);
    else
      launch_backward_rows_metric<false>(metric, a, vec, sms, st);
    return cudaGetLastError();
  }
  if (dx && zero_dx) launch_fill_zero(dx, N * (int64_t)D, sms, st);
  if (dq && M > 0) {
    const unsigned grid = (unsigned)cdiv(M * 32, 256);
    if (metric == KNN_IP)
      dq_kernel<KNN_IP><<<grid, 256, 0, st>>>(M, D, K, q, xs, N, idx, g, dq);
    else if (metric == KNN_L2)
      dq_kernel<KNN_L2><<<grid, 256, 0, st>>>(M, D, K, q, xs, N, idx, g, dq);
    else
      dq_kernel<KNN_COS><<<grid, 256, 0, st>>>(M, D, K, q, xs, N, idx, g, dq);
  }
  if (dx && E > 0) {
    const bool vec4 = D % 4 == 0 && aligned16(dx) && aligned16(q);
    const unsigned grid = (unsigned)cdiv(E * 32, 256);
    if (vec4) {
      if (metric == KNN_IP)
        dx_atomic4_kernel<KNN_IP><<<grid, 256, 0, st>>>(E, D, K, q, xs, N, idx, g, dx);
      else if (metric == KNN_L2)
        dx_atomic4_kernel<KNN_L2><<<grid, 256, 0, st>>>(E, D, K, q, xs, N, idx, g, dx);
      else
        dx_atomic4_kernel<KNN_COS><<<grid, 256, 0, st>>>(E, D, K, q, xs, N, idx, g, dx);
    } else {
      dx_atomic_kernel<<<grid, 256, 0, st>>>(E, D, K, metric, q, xs, N, idx, g, dx);
    }
  }
  return cudaGetLastError();
}

}  // namespace tpuknn
