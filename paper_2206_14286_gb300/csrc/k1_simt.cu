// k1_simt.cu -- PartialReduce (Alg. 1) fused with an FP32 SIMT contraction.
//
// The plain FP32 path: no tensor cores, exact FP32 scores and exact indices.
// Tiling follows Alg. 2 (App. A.3): a block of BQ = 64 queries stays fixed
// while the CTA walks tiles of BW = 64 database rows; the D loop runs in
// chunks of 16 through shared memory with FFMA on a 4 x 4 register tile per
// thread; after each tile the compare/select of Alg. 1 (strict '>' while the
// row index grows, so ties keep the smaller index) updates the running best
// of each (query, bin) the thread owns. A thread owns 4 queries x 4 bins and
// the bins never change across tiles (tile t covers rows t*Lk + strip*64 +
// [0, 64)), so the running state lives in registers and only M x L partials
// per split reach memory (Eq. 20's 2*4*M*L output bytes per split).
#include "common.cuh"
#include "kernels.h"

namespace tpuknn {

namespace {
constexpr int BQ = 64, BW = 64, BD = 16, PADW = 68;

template <int METRIC>
__global__ void __launch_bounds__(256)
k1_simt_kernel(const float* __restrict__ X, const float* __restrict__ hnorm,
               const float* __restrict__ Qp, K1Plan p, float* __restrict__ part_v,
               int32_t* __restrict__ part_a) {
  __shared__ __align__(16) float Qs[BD][PADW];
  __shared__ __align__(16) float Xs[BD][PADW];
  const int tid = threadIdx.x, tq = tid >> 4, tb = tid & 15;
  int64_t cta = blockIdx.x;
  const int64_t qtile = cta % p.nqtiles;
  cta /= p.nqtiles;
  const int64_t strip = cta % p.nstrips;
  const int64_t split = cta / p.nstrips;
  const int64_t i0 = qtile * BQ, b0 = strip * BW;
  const int64_t t_begin = split * p.tiles_per_split;
  const int64_t t_end = min(p.ntiles, t_begin + p.tiles_per_split);

  float v[4][4];
  int32_t a[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      v[r][c] = neg_inf();
      a[r][c] = -1;
    }

  // loader mapping: 64 rows x 16 columns, one float4 per thread
  const int lrow = tid >> 2, lcol = (tid & 3) * 4;
  const int64_t qrow = i0 + lrow;
  const bool qvalid = qrow < p.M;

  for (int64_t t = t_begin; t < t_end; ++t) {
    const int64_t row0 = t * p.Lk + b0;
    const int64_t xrow = row0 + lrow;
    const bool xvalid = (b0 + lrow < p.Lk) && (xrow < p.N);
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = 0.0f;

    for (int d0 = 0; d0 < p.pitch; d0 += BD) {
      float4 qv = qvalid ? *reinterpret_cast<const float4*>(Qp + qrow * p.pitch + d0 + lcol)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
      float4 xv = xvalid ? *reinterpret_cast<const float4*>(X + xrow * p.pitch + d0 + lcol)
                         : make_float4(0.f, 0.f, 0.f, 0.f);
      __syncthreads();
      Qs[lcol + 0][lrow] = qv.x;
      Qs[lcol + 1][lrow] = qv.y;
      Qs[lcol + 2][lrow] = qv.z;
      Qs[lcol + 3][lrow] = qv.w;
      Xs[lcol + 0][lrow] = xv.x;
      Xs[lcol + 1][lrow] = xv.y;
      Xs[lcol + 2][lrow] = xv.z;
      Xs[lcol + 3][lrow] = xv.w;
      __syncthreads();
#pragma unroll
      for (int dd = 0; dd < BD; ++dd) {
        float4 q4 = *reinterpret_cast<const float4*>(&Qs[dd][tq * 4]);
        float4 x4 = *reinterpret_cast<const float4*>(&Xs[dd][tb * 4]);
        float qa[4] = {q4.x, q4.y, q4.z, q4.w};
        float xa[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(qa[r], xa[c], acc[r][c]);
      }
    }
    // Alg. 1 compare/select per (query, bin)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t b = b0 + tb * 4 + c;
      const int64_t j = row0 + tb * 4 + c;
      const bool valid = (b < p.Lk) && (j < p.N);
      const float hb = (METRIC == KNN_L2 && valid) ? hnorm[j] : 0.0f;
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float s = acc[r][c] - hb;
        if (valid && s > v[r][c]) {
          v[r][c] = s;
          a[r][c] = (int32_t)j;
        }
      }
    }
  }
  // partials of this split
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t i = i0 + tq * 4 + r;
    if (i >= p.M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t b = b0 + tb * 4 + c;
      if (b >= p.Lk) continue;
      const int64_t o = (split * p.M + i) * p.Lk + b;
      part_v[o] = v[r][c];
      part_a[o] = a[r][c];
    }
  }
}
}  // namespace

cudaError_t launch_k1_simt(const K1Plan& p, const float* X, const float* hnorm, const float* Qp,
                           Partials out, cudaStream_t st) {
  if (p.BW != BW || p.BQ != BQ || (p.pitch % BD) != 0) return cudaErrorInvalidValue;
  int64_t blocks = p.nsplits * p.nstrips * p.nqtiles;
  if (blocks <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (p.metric == KNN_L2)
    k1_simt_kernel<KNN_L2><<<(unsigned)blocks, 256, 0, st>>>(X, hnorm, Qp, p, out.v, out.a);
  else
    k1_simt_kernel<KNN_IP><<<(unsigned)blocks, 256, 0, st>>>(X, hnorm, Qp, p, out.v, out.a);
  return cudaGetLastError();
}

}  // namespace tpuknn
