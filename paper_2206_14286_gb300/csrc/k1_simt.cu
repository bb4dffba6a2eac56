// k1_simt.cu -- PartialReduce (Alg. 1) fused with an FP32 SIMT contraction.
//
// The plain FP32 path: no tensor cores, exact FP32 scores and exact indices.
// Tiling follows Alg. 2 (App. A.3): a block of BQ = 128 queries stays fixed
// while the CTA walks tiles of BW = 64 database rows; the D loop runs in
// chunks of BD = 16 through double-buffered shared memory (the next chunk's
// global loads are in registers while the current chunk is multiplied), with
// FFMA on an 8 x 4 register tile per thread; after each tile the
// compare/select of Alg. 1 (strict '>' while the row index grows, so ties
// keep the smaller index) updates the running best of each (query, bin) the
// thread owns. A thread owns 8 queries x 4 bins and the bins never change
// across tiles (tile t covers rows t*Lk + strip*64 + [0, 64)); the running
// (value, row) state of the CTA's 128 x 64 pairs lives in shared memory (one
// 16-byte load and at most two 16-byte stores per query row and tile), which
// leaves the registers to the accumulators and the operand prefetch, and only
// M x L partials per split reach memory (Eq. 20's 2*4*M*L output bytes per
// split).
#include "common.cuh"
#include "kernels.h"

namespace tpuknn {

namespace {
constexpr int BQ = 128, BW = 64, BD = 16;
constexpr int PADQ = BQ + 4, PADW = BW + 4;  // row padding of the transposed tiles
constexpr int TQ = 8, TB = 4;                // queries x bins per thread
constexpr int kSimtThreads = 256;            // (BQ / TQ) x (BW / TB) threads

template <int METRIC>
__global__ void __launch_bounds__(kSimtThreads, 2)
k1_simt_kernel(const float* __restrict__ X, const float* __restrict__ hnorm,
               const float* __restrict__ Qp, K1Plan p, float* __restrict__ part_v,
               int32_t* __restrict__ part_a) {
  __shared__ __align__(16) float Qs[2][BD][PADQ];
  __shared__ __align__(16) float Xs[2][BD][PADW];
  // running best (value, row) of each (query, bin) of the CTA: [BQ][BW]
  extern __shared__ __align__(16) float simt_state[];
  float* sv = simt_state;
  int32_t* sa = reinterpret_cast<int32_t*>(simt_state + BQ * BW);
  const int tid = threadIdx.x, tq = tid >> 4, tb = tid & 15;
  int64_t cta = blockIdx.x;
  const int64_t qtile = cta % p.nqtiles;
  cta /= p.nqtiles;
  const int64_t strip = cta % p.nstrips;
  const int64_t split = cta / p.nstrips;
  const int64_t i0 = qtile * BQ, b0 = strip * BW;
  const int64_t t_begin = split * p.tiles_per_split;
  const int64_t t_end = min(p.ntiles, t_begin + p.tiles_per_split);

  // this thread's entries: rows tq*TQ + r, columns tb*TB .. tb*TB + 3
#pragma unroll
  for (int r = 0; r < TQ; ++r) {
    const int o = (tq * TQ + r) * BW + tb * TB;
    *reinterpret_cast<float4*>(sv + o) = make_float4(neg_inf(), neg_inf(), neg_inf(), neg_inf());
    *reinterpret_cast<int4*>(sa + o) = make_int4(-1, -1, -1, -1);
  }

  // loader mapping: a chunk is BQ query rows and BW database rows of BD
  // floats; thread tid loads the float4 at column lcol of rows lrow (and
  // lrow + 64 for the queries)
  const int lrow = tid >> 2, lcol = (tid & 3) * 4;
  const bool qv0 = i0 + lrow < p.M, qv1 = i0 + lrow + 64 < p.M;
  const float* qp0 = Qp + (qv0 ? (i0 + lrow) * p.pitch + lcol : 0);
  const float* qp1 = Qp + (qv1 ? (i0 + lrow + 64) * p.pitch + lcol : 0);
  const int nchunks = p.pitch / BD;

  for (int64_t t = t_begin; t < t_end; ++t) {
    const int64_t row0 = t * p.Lk + b0;
    const int64_t xrow = row0 + lrow;
    const bool xvalid = (b0 + lrow < p.Lk) && (xrow < p.N);
    const float* xp = X + (xvalid ? xrow * p.pitch + lcol : 0);
    float acc[TQ][TB];
#pragma unroll
    for (int r = 0; r < TQ; ++r)
#pragma unroll
      for (int c = 0; c < TB; ++c) acc[r][c] = 0.0f;

    auto fetch = [&](int d0, float4& q0, float4& q1, float4& x0) {
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      q0 = qv0 ? __ldg(reinterpret_cast<const float4*>(qp0 + d0)) : z;
      q1 = qv1 ? __ldg(reinterpret_cast<const float4*>(qp1 + d0)) : z;
      x0 = xvalid ? __ldg(reinterpret_cast<const float4*>(xp + d0)) : z;
    };
    auto stash = [&](int buf, const float4& q0, const float4& q1, const float4& x0) {
      Qs[buf][lcol + 0][lrow] = q0.x;
      Qs[buf][lcol + 1][lrow] = q0.y;
      Qs[buf][lcol + 2][lrow] = q0.z;
      Qs[buf][lcol + 3][lrow] = q0.w;
      Qs[buf][lcol + 0][lrow + 64] = q1.x;
      Qs[buf][lcol + 1][lrow + 64] = q1.y;
      Qs[buf][lcol + 2][lrow + 64] = q1.z;
      Qs[buf][lcol + 3][lrow + 64] = q1.w;
      Xs[buf][lcol + 0][lrow] = x0.x;
      Xs[buf][lcol + 1][lrow] = x0.y;
      Xs[buf][lcol + 2][lrow] = x0.z;
      Xs[buf][lcol + 3][lrow] = x0.w;
    };
    float4 nq0, nq1, nx0;
    fetch(0, nq0, nq1, nx0);
    // the previous tile's last chunk may still be read from buffer 0 or 1:
    // every thread has passed its compare/select before buffers are refilled
    __syncthreads();
    stash(0, nq0, nq1, nx0);
    __syncthreads();
    for (int ch = 0; ch < nchunks; ++ch) {
      const int buf = ch & 1;
      if (ch + 1 < nchunks) fetch((ch + 1) * BD, nq0, nq1, nx0);
#pragma unroll
      for (int dd = 0; dd < BD; ++dd) {
        const float4 qa4 = *reinterpret_cast<const float4*>(&Qs[buf][dd][tq * TQ]);
        const float4 qb4 = *reinterpret_cast<const float4*>(&Qs[buf][dd][tq * TQ + 4]);
        const float4 x4 = *reinterpret_cast<const float4*>(&Xs[buf][dd][tb * TB]);
        const float qa[TQ] = {qa4.x, qa4.y, qa4.z, qa4.w, qb4.x, qb4.y, qb4.z, qb4.w};
        const float xa[TB] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
        for (int r = 0; r < TQ; ++r)
#pragma unroll
          for (int c = 0; c < TB; ++c) acc[r][c] = fmaf(qa[r], xa[c], acc[r][c]);
      }
      if (ch + 1 < nchunks) {
        // the other buffer was last read in chunk ch - 1, before the barrier
        // that ended it
        stash(buf ^ 1, nq0, nq1, nx0);
        __syncthreads();
      }
    }
    // Alg. 1 compare/select per (query, bin), against the state in shared memory
    float hb[TB];
    bool valid[TB];
#pragma unroll
    for (int c = 0; c < TB; ++c) {
      const int64_t b = b0 + tb * TB + c;
      const int64_t j = row0 + tb * TB + c;
      valid[c] = (b < p.Lk) && (j < p.N);
      hb[c] = (METRIC == KNN_L2 && valid[c]) ? hnorm[j] : 0.0f;
    }
#pragma unroll
    for (int r = 0; r < TQ; ++r) {
      const int o = (tq * TQ + r) * BW + tb * TB;
      float4 bv = *reinterpret_cast<const float4*>(sv + o);
      int4 ba = *reinterpret_cast<const int4*>(sa + o);
      float* bvp = reinterpret_cast<float*>(&bv);
      int* bap = reinterpret_cast<int*>(&ba);
      bool upd = false;
#pragma unroll
      for (int c = 0; c < TB; ++c) {
        const float sc = acc[r][c] - hb[c];
        if (valid[c] && sc > bvp[c]) {
          bvp[c] = sc;
          bap[c] = (int32_t)(row0 + tb * TB + c);
          upd = true;
        }
      }
      if (upd) {
        *reinterpret_cast<float4*>(sv + o) = bv;
        *reinterpret_cast<int4*>(sa + o) = ba;
      }
    }
  }
  // partials of this split
#pragma unroll
  for (int r = 0; r < TQ; ++r) {
    const int64_t i = i0 + tq * TQ + r;
    if (i >= p.M) continue;
#pragma unroll
    for (int c = 0; c < TB; ++c) {
      const int64_t b = b0 + tb * TB + c;
      if (b >= p.Lk) continue;
      const int64_t o = (split * p.M + i) * p.Lk + b;
      const int so = (tq * TQ + r) * BW + tb * TB + c;
      part_v[o] = sv[so];
      part_a[o] = sa[so];
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
  const size_t smem = (size_t)BQ * BW * 8;
  if (p.metric == KNN_L2) {
    cudaError_t e = cudaFuncSetAttribute(k1_simt_kernel<KNN_L2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k1_simt_kernel<KNN_L2><<<(unsigned)blocks, kSimtThreads, smem, st>>>(X, hnorm, Qp, p, out.v,
                                                                          out.a);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k1_simt_kernel<KNN_IP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k1_simt_kernel<KNN_IP><<<(unsigned)blocks, kSimtThreads, smem, st>>>(X, hnorm, Qp, p, out.v,
                                                                          out.a);
  }
  return cudaGetLastError();
}

}  // namespace tpuknn
