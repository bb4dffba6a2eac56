// k1_tc.cu -- PartialReduce (Alg. 1) fused with a tcgen05 tensor-core
// contraction (BF16 or FP8-E4M3 inputs, FP32 accumulation in tensor memory).
//
// Structure of one CTA (one per SM, 640 threads = 5 warpgroups):
//   warp 0      : TMA producer. Loads the CTA's query tile once (it stays in
//                 shared memory), then streams database tiles of 128 rows
//                 through an S-stage ring (mbarrier full/empty pairs).
//   warp 1      : allocates tensor memory and issues tcgen05.mma (one thread):
//                 D[128 rows x BQ queries] = X_tile . Q_tile^T, accumulators
//                 double-buffered in TMEM so the epilogue of tile t overlaps
//                 the MMAs of tile t+1.
//   warps 2, 3  : idle (they complete the first warpgroup, which gives up
//                 registers with setmaxnreg so the epilogue can hold its state).
//   warps 4..19 : epilogue, four warpgroups. Each thread owns one TMEM lane
//                 (= one database row of the tile = one bin, because a tile is
//                 one strip of one row of the [ntiles x Lk] bin grid) and a
//                 quarter of the query columns. Four warps per scheduler hide
//                 the latency of each 16-column TMEM load behind the others'
//                 work (two warps with half the columns each: 1.10 against
//                 0.96 ms on 2M x 96 E4M3 rows, 2000 queries).
//                 Per score it applies the metric (L2: subtract the half norm,
//                 App. A.2 Eq. 19; E4M3: multiply by the row scale) and keeps a
//                 running maximum per (query, bin) in registers.
//
// The running maximum is a packed key: the FP32 score with its low c bits
// replaced by (2^c - 1 - tile ordinal). One FMNMX then keeps value and
// position together (2 COPs per score for IP, 3 for L2, against the 3
// compare/select COPs of Alg. 1). Dropping c <= 13 low bits changes a score by
// less than 2^-(23-c) of its magnitude (<= 2^-10 = 1e-3 relative), below the
// BF16 tolerance; the row index is recovered exactly from the code.
//
// Every mbarrier wait is bounded (2 s); a wait that runs out sets a device
// flag (read by knn_sync_status), raises a CTA-wide abort flag, and the CTA
// drains its in-flight copies and MMAs (again with bounded waits) and frees
// its tensor memory before exiting.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace tpuknn {

namespace {

constexpr int kThreads = 640;
constexpr int kCtrlRegs = 56, kEpiRegs = 104;  // 128*56 + 512*104 <= 640*96 (launch)
constexpr int kRows = 128;          // database rows per tile (MMA M)
constexpr int kKBlockBytes = 128;   // one 128-byte swizzle span along D

struct TcArgs {
  int64_t N, M, Lk, ntiles, tiles_per_split, nstrips, nqtiles;
  int nkb;            // 128-byte blocks along D
  int nksteps;        // MMA K-steps (32 bytes of D each)
  int stages;
  uint32_t q_bytes, stage_bytes;
  uint32_t code_bits;
  int atomic_merge;   // 1: red.max of order-mapped keys into part[M][Lk], code = global tile
  uint32_t idesc;
  const float* hnorm;
  const float* xscale;
  const float* qscale;
  uint32_t* part;
};


// 16 consecutive FP32 columns of this thread's TMEM lane, not waited for.
__device__ __forceinline__ void tmem_ld16n(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
               :
               : "memory");
}
// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------
template <int DT, int METRIC, int BQ>
__global__ void __launch_bounds__(kThreads, 1)
k1_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmQ,
             const TcArgs a) {
  constexpr int PART = BQ / 4;  // query columns of one epilogue warpgroup
  constexpr uint32_t TMEM_COLS = 2 * BQ;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  uint8_t* sQ = smem;
  uint8_t* sA = sQ + a.q_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + (size_t)a.stages * a.stage_bytes);
  const int S = a.stages;
  // barrier indices
  const uint32_t b_full = smem_u32(bars), b_empty = smem_u32(bars + S);
  const uint32_t b_accf = smem_u32(bars + 2 * S), b_acce = smem_u32(bars + 2 * S + 2);
  const uint32_t b_q = smem_u32(bars + 2 * S + 4), b_done = smem_u32(bars + 2 * S + 5);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 6);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* s_qscale = reinterpret_cast<float*>(tmem_slot + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  int64_t cta = blockIdx.x;
  const int64_t qtile = cta % a.nqtiles;
  cta /= a.nqtiles;
  const int64_t strip = cta % a.nstrips;
  const int64_t split = cta / a.nstrips;
  const int64_t t_begin = split * a.tiles_per_split;
  const int64_t t_end = min(a.ntiles, t_begin + a.tiles_per_split);
  const int nt = (int)(t_end - t_begin);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(b_full + 8 * s, 1);
      mbar_init(b_empty + 8 * s, 1);
    }
    mbar_init(b_accf, 1);
    mbar_init(b_accf + 8, 1);
    mbar_init(b_acce, 16);
    mbar_init(b_acce + 8, 16);
    mbar_init(b_q, 1);
    mbar_init(b_done, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (DT == KNN_E4M3 && METRIC == KNN_L2) {
    for (int c = threadIdx.x; c < BQ; c += kThreads) {
      const int64_t i = qtile * BQ + c;
      s_qscale[c] = i < a.M ? a.qscale[i] : 0.0f;
    }
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp < 4) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kCtrlRegs));
    if (warp == 0 && lane == 0) {
      // ---------------------------------------------------------- producer
      mbar_expect_tx(b_q, a.q_bytes);
      const int qrow = (int)(qtile * BQ);
      for (int kb = 0; kb < a.nkb; ++kb)
        tma_load_2d(smem_u32(sQ + (size_t)kb * BQ * kKBlockBytes), &tmQ, b_q,
                    kb * (kKBlockBytes / (DT == KNN_BF16 ? 2 : 1)), qrow);
      int issued = 0, s = 0;
      uint32_t ph = 0;
      for (int it = 0; it < nt; ++it) {
        if (it >= S && !mbar_wait_sleep(b_empty + 8 * s, ph ^ 1u, abort_flag)) break;
        mbar_expect_tx(b_full + 8 * s, a.stage_bytes);
        const int row0 = (int)((t_begin + it) * a.Lk + strip * kRows);
        uint8_t* dst = sA + (size_t)s * a.stage_bytes;
        for (int kb = 0; kb < a.nkb; ++kb)
          tma_load_2d(smem_u32(dst + (size_t)kb * kRows * kKBlockBytes), &tmX, b_full + 8 * s,
                      kb * (kKBlockBytes / (DT == KNN_BF16 ? 2 : 1)), row0);
        issued = it + 1;
        if (++s == S) {
          s = 0;
          ph ^= 1u;
        }
      }
      // drain: the last min(issued, S) copies and the query tile land before
      // the CTA can exit, also after a give-up
      for (int k = 0; k < S && k < issued; ++k) {
        if (--s < 0) {
          s = S - 1;
          ph ^= 1u;
        }
        mbar_drain(b_full + 8 * s, ph);
      }
      mbar_drain(b_q, 0);
    } else if (warp == 1) {
      // ---------------------------------------------------------- MMA issuer
      if (lane == 0) {
        if (mbar_wait(b_q, 0, abort_flag)) {
          const uint32_t q_base = smem_u32(sQ);
          int s = 0;
          uint32_t ph = 0;
          for (int it = 0; it < nt; ++it) {
            const int ab = it & 1;
            const uint32_t aph = (uint32_t)((it >> 1) & 1);
            if (!mbar_wait(b_full + 8 * s, ph, abort_flag)) break;
            if (it >= 2 && !mbar_wait(b_acce + 8 * ab, aph ^ 1u, abort_flag)) break;
            tc_fence_after();
            const uint32_t a_base = smem_u32(sA + (size_t)s * a.stage_bytes);
            const uint32_t d_tmem = tmem_base + (uint32_t)(ab * BQ);
            for (int ks = 0; ks < a.nksteps; ++ks) {
              const int kb = ks >> 2, kk = ks & 3;
              const uint64_t ad = smem_desc_sw128(a_base + kb * kRows * kKBlockBytes + kk * 32);
              const uint64_t bd = smem_desc_sw128(q_base + kb * BQ * kKBlockBytes + kk * 32);
              tc_mma<DT>(d_tmem, ad, bd, a.idesc, ks > 0 ? 1u : 0u);
            }
            tc_commit(b_empty + 8 * s);
            tc_commit(b_accf + 8 * ab);
            if (++s == S) {
              s = 0;
              ph ^= 1u;
            }
          }
        }
        // all MMAs have completed before tensor memory is released (also
        // after a give-up: the MMAs already issued still write TMEM)
        tc_commit(b_done);
        mbar_drain(b_done, 0);
      }
      __syncwarp();
      // wait until the epilogue has read its last accumulator
      asm volatile("bar.sync 1, %0;" ::"n"(32 + 512) : "memory");
      tc_fence_after();
      tmem_dealloc(tmem_base, TMEM_COLS);
    }
    return;
  }

  // ------------------------------------------------------------ epilogue
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kEpiRegs));
  constexpr int NC = PART / 16;
  const int quad = warp & 3;
  const int part = (warp - 4) >> 2;  // query columns part*PART ..
  const int lrow = quad * 32 + lane;
  const int64_t bin = strip * kRows + lrow;
  const bool bin_ok = bin < a.Lk;
  const uint32_t mask = a.code_bits ? ((1u << a.code_bits) - 1u) : 0u;
  const uint32_t nmask = ~mask;
  const int64_t code_t0 = a.atomic_merge ? t_begin : 0;
  float v[PART];
#pragma unroll
  for (int c = 0; c < PART; ++c) v[c] = __uint_as_float(kNegInfBits);

  // per-row factors of the next tile are loaded one tile ahead
  float bias_n = 0.0f, mul_n = 1.0f;
  {
    const int64_t j = t_begin * a.Lk + bin;
    if (bin_ok && j < a.N) {
      if (METRIC == KNN_L2) bias_n = a.hnorm[j];
      if (DT == KNN_E4M3) mul_n = a.xscale[j];
    }
  }
  for (int it = 0; it < nt; ++it) {
    const int ab = it & 1;
    const uint32_t aph = (uint32_t)((it >> 1) & 1);
    const int64_t j = (t_begin + it) * a.Lk + bin;
    const bool valid = bin_ok && (j < a.N);
    const float bias = bias_n, mul = mul_n;
    if (it + 1 < nt) {
      const int64_t jn = j + a.Lk;
      if (bin_ok && jn < a.N) {
        if (METRIC == KNN_L2) bias_n = a.hnorm[jn];
        if (DT == KNN_E4M3) mul_n = a.xscale[jn];
      }
    }
    if (!warp_all(mbar_wait_sleep(b_accf + 8 * ab, aph, abort_flag))) break;
    tc_fence_after();
    // invalid lanes turn every key into -inf: no divergence, no extra select
    const uint32_t km = valid ? nmask : 0u;
    const uint32_t kc = valid ? (mask - (uint32_t)(code_t0 + it)) : kNegInfBits;
    const uint32_t col0 =
        tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(ab * BQ + part * PART);
    uint32_t ra[16], rb[16];
    tmem_ld16n(col0, ra);
    tmem_wait16(ra);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      uint32_t(&cur)[16] = (c & 1) ? rb : ra;
      uint32_t(&nxt)[16] = (c & 1) ? ra : rb;
      if (c + 1 < NC) tmem_ld16n(col0 + (uint32_t)((c + 1) * 16), nxt);
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        float sc = __uint_as_float(cur[k]);
        if (DT == KNN_E4M3) {
          if (METRIC == KNN_L2)
            sc = fmaf(sc, mul * s_qscale[part * PART + c * 16 + k], -bias);
          else
            sc = sc * mul;
        } else if (METRIC == KNN_L2) {
          sc = sc - bias;
        }
        const float key = __uint_as_float((__float_as_uint(sc) & km) | kc);
        v[c * 16 + k] = fmaxf(v[c * 16 + k], key);
      }
      if (c + 1 < NC) tmem_wait16(nxt);
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(b_acce + 8 * ab);
  }
  tc_fence_before();
  asm volatile("bar.arrive 1, %0;" ::"n"(32 + 512) : "memory");
  if (bin_ok) {
#pragma unroll
    for (int c = 0; c < PART; ++c) {
      const int64_t i = qtile * BQ + part * PART + c;
      if (i >= a.M) continue;
      const uint32_t u = __float_as_uint(v[c]);
      if (a.atomic_merge) {
        if (u != kNegInfBits) atomicMax(&a.part[i * a.Lk + bin], float_to_ordered(v[c]));
      } else {
        a.part[(split * a.M + i) * a.Lk + bin] = u;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* m, const void* base, int dtype, int64_t rows, int pitch, int box_rows) {
  auto enc = get_encode();
  if (!enc) return false;
  const int esz = dtype == KNN_BF16 ? 2 : 1;
  cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)pitch * esz};
  cuuint32_t box[2] = {(cuuint32_t)(kKBlockBytes / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, dtype == KNN_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8,
                   2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int DT, int METRIC, int BQ>
cudaError_t launch_variant(const CUtensorMap& mx, const CUtensorMap& mq, const TcArgs& a,
                           size_t smem, int64_t blocks, cudaStream_t st) {
  auto kern = k1_tc_kernel<DT, METRIC, BQ>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)blocks, kThreads, smem, st>>>(mx, mq, a);
  return cudaGetLastError();
}

template <int DT, int BQ>
cudaError_t launch_metric(int metric, const CUtensorMap& mx, const CUtensorMap& mq,
                          const TcArgs& a, size_t smem, int64_t blocks, cudaStream_t st) {
  if (metric == KNN_L2) return launch_variant<DT, KNN_L2, BQ>(mx, mq, a, smem, blocks, st);
  return launch_variant<DT, KNN_IP, BQ>(mx, mq, a, smem, blocks, st);
}

}  // namespace

// Largest query tile the kernel can keep resident for this row length.
int k1_tc_query_tile(int dtype, int D) {
  const int esz = dtype == KNN_BF16 ? 2 : 1;
  const int pitch = (int)round_up(D, 16);
  const int nkb = (int)cdiv((int64_t)pitch * esz, kKBlockBytes);
  if (nkb <= 2) return 256;
  if (nkb <= 4) return 128;
  return 0;
}

cudaError_t launch_k1_tc(const K1Plan& p, const void* X, const float* xscale, const float* hnorm,
                         const void* Qp, const float* qscale, Partials out, cudaStream_t st) {
  if (p.dtype != KNN_BF16 && p.dtype != KNN_E4M3) return cudaErrorNotSupported;
  if (p.BW != kRows || (p.BQ != 128 && p.BQ != 256)) return cudaErrorNotSupported;
  const int esz = p.dtype == KNN_BF16 ? 2 : 1;
  TcArgs a{};
  a.N = p.N;
  a.M = p.M;
  a.Lk = p.Lk;
  a.ntiles = p.ntiles;
  a.tiles_per_split = p.tiles_per_split;
  a.nstrips = p.nstrips;
  a.nqtiles = p.nqtiles;
  a.nkb = (int)cdiv((int64_t)p.pitch * esz, kKBlockBytes);
  a.nksteps = (int)cdiv((int64_t)p.pitch * esz, 32);
  a.q_bytes = (uint32_t)(a.nkb * p.BQ * kKBlockBytes);
  a.stage_bytes = (uint32_t)(a.nkb * kRows * kKBlockBytes);
  const size_t budget = 227 * 1024 - 1024 - 512 - (size_t)p.BQ * 4;
  if (a.q_bytes + 2 * (size_t)a.stage_bytes > budget) return cudaErrorNotSupported;
  int stages = (int)((budget - a.q_bytes) / a.stage_bytes);
  a.stages = stages > 6 ? 6 : stages;
  a.code_bits = (uint32_t)p.code_bits;
  a.atomic_merge = p.atomic_merge ? 1 : 0;
  // instruction descriptor: D = F32, A/B = BF16 (kind::f16) or E4M3 (kind::f8f6f4),
  // both K-major, N = BQ, M = 128
  uint32_t idesc = (1u << 4);
  if (p.dtype == KNN_BF16) idesc |= (1u << 7) | (1u << 10);
  idesc |= ((uint32_t)(p.BQ >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
  a.idesc = idesc;
  a.hnorm = hnorm;
  a.xscale = xscale;
  a.qscale = qscale;
  a.part = reinterpret_cast<uint32_t*>(out.v);
  if (p.metric == KNN_L2 && !hnorm) return cudaErrorInvalidValue;
  if (p.dtype == KNN_E4M3 && (!xscale || !qscale)) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (reinterpret_cast<uintptr_t>(Qp) & 15))
    return cudaErrorInvalidValue;
  const int64_t blocks = p.nsplits * p.nstrips * p.nqtiles;
  if (blocks <= 0 || p.M <= 0) return cudaSuccess;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  CUtensorMap mx, mq;
  if (!make_map(&mx, X, p.dtype, p.N, p.pitch, kRows)) return cudaErrorInvalidValue;
  if (!make_map(&mq, Qp, p.dtype, p.M, p.pitch, p.BQ)) return cudaErrorInvalidValue;
  size_t smem = 1024 + a.q_bytes + (size_t)a.stages * a.stage_bytes + 512 + (size_t)p.BQ * 4;
  // A CTA with BQ = 256 allocates all 512 TMEM columns: keep it alone on its SM.
  if (p.BQ == 256 && smem < 120 * 1024) smem = 120 * 1024;
  if (p.dtype == KNN_BF16) {
    if (p.BQ == 256) return launch_metric<KNN_BF16, 256>(p.metric, mx, mq, a, smem, blocks, st);
    return launch_metric<KNN_BF16, 128>(p.metric, mx, mq, a, smem, blocks, st);
  }
  if (p.BQ == 256) return launch_metric<KNN_E4M3, 256>(p.metric, mx, mq, a, smem, blocks, st);
  return launch_metric<KNN_E4M3, 128>(p.metric, mx, mq, a, smem, blocks, st);
}


bool k1_tc_take_timeout() { return tc_take_timeout_local(); }
bool k1_tc_set_wait_limit(unsigned long long ns) { return tc_set_wait_limit_local(ns); }

}  // namespace tpuknn
