// k1_tcq.cu -- PartialReduce with contiguous bins (Alg. 1: l = ShiftRight(j, W),
// generalised to L balanced runs of rows) fused with a tcgen05 BF16
// contraction, queries on the tensor-memory lanes.
//
// One CTA (640 threads, one per SM) owns 128 queries and a contiguous range
// of database rows, walked in tiles of 256 rows:
//   warp 0      : TMA producer. The query tile stays in shared memory; each
//                 tile's 128-byte K blocks (256 rows x 64 BF16) stream through
//                 an S-stage ring.
//   warp 2      : (L2 only) writes each tile's half norms as an extra K block
//                 (-h split into three BF16 parts) into a 2-slot ring, so the
//                 contraction itself yields the relaxed score <q,x> - |x|^2/2
//                 (App. A.2, Eq. 19); its global loads run four tiles ahead.
//   warp 1      : TMEM allocation and tcgen05.mma issue (one thread):
//                 D[128 queries x 256 rows] (M = 128, N = 256: 128 cycles of
//                 tensor work per instruction), two accumulator buffers.
//   warps 4..19 : epilogue, four warpgroups: two per accumulator buffer (even
//                 and odd tiles), each owning 128 of the tile's 256 columns. A
//                 thread owns one query (its TMEM lane). Columns are consecutive
//                 database rows, so each run of 16 columns inside one bin is
//                 reduced by tcgen05.ld.red.max (the load returns the 16 scores
//                 and their maximum) and compared once. Only when that maximum beats the bin's best so far
//                 does the thread look for its column; a bin boundary inside a
//                 run is handled column by column. Each thread keeps just the
//                 current bin's best score and row; when the bin ends it merges
//                 them into G[query][bin] with a 64-bit atomicMax on the
//                 ordered key (score, ~row), so ties keep the smaller row and
//                 bins split between CTAs merge exactly.
//   warp 3      : idle.
// All waits are bounded (see tc_ptx.cuh).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace tpuknn {

namespace {

constexpr int kThreadsQ = 640;  // 4 control warps + 4 epilogue warpgroups
constexpr int kQ = 128;          // queries per CTA: MMA M, TMEM lanes
constexpr int kBN = 256;         // database rows per tile: MMA N
constexpr int kNumAcc = 2;       // accumulator buffers of kBN columns
constexpr int kSpan = 128;       // bytes of one 128-byte swizzle span (one K block)
constexpr int kStageBytes = kBN * kSpan;   // one K block of a tile
constexpr int kExtA = kQ * 32;   // K = 16 BF16 block of the query tile
constexpr int kExtB = kBN * 32;  // K = 16 BF16 block of a database tile
constexpr int kExtSlots = 2;

struct TcqArgs {
  int64_t N, M, L;
  int64_t bq, br;                  // bins: q = N / L, r = N % L
  int64_t rows_per_cta, nranges, nqtiles;
  int nkb, nksteps, stages;
  uint32_t a_bytes;
  int ext;
  uint32_t idesc;
  const float* hnorm;
  unsigned long long* G;
};

__device__ __forceinline__ int64_t bin_of(int64_t p, int64_t q, int64_t r) {
  const int64_t big = r * (q + 1);
  return p < big ? p / (q + 1) : r + (p - big) / q;
}
__device__ __forceinline__ int64_t bin_end(int64_t b, int64_t q, int64_t r) {
  return (b + 1) * q + min(b + 1, r);
}

// 64 columns of this thread's lane as four runs of 16, with the maximum of
// each run (tcgen05.ld.red), waited for.
__device__ __forceinline__ void tmem_ld4x16_max(uint32_t taddr, float (&r)[4][16], float (&m)[4]) {
  asm volatile(
      "tcgen05.ld.red.sync.aligned.32x32b.x16.max.f32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, %16, [%68];\n\t"
      "tcgen05.ld.red.sync.aligned.32x32b.x16.max.f32 {%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32}, %33, [%69];\n\t"
      "tcgen05.ld.red.sync.aligned.32x32b.x16.max.f32 {%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49}, %50, [%70];\n\t"
      "tcgen05.ld.red.sync.aligned.32x32b.x16.max.f32 {%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63,%64,%65,%66}, %67, [%71];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=f"(r[0][0]), "=f"(r[0][1]), "=f"(r[0][2]), "=f"(r[0][3]), "=f"(r[0][4]), "=f"(r[0][5]), "=f"(r[0][6]), "=f"(r[0][7]), "=f"(r[0][8]), "=f"(r[0][9]), "=f"(r[0][10]), "=f"(r[0][11]), "=f"(r[0][12]), "=f"(r[0][13]), "=f"(r[0][14]), "=f"(r[0][15]), "=f"(m[0]),
        "=f"(r[1][0]), "=f"(r[1][1]), "=f"(r[1][2]), "=f"(r[1][3]), "=f"(r[1][4]), "=f"(r[1][5]), "=f"(r[1][6]), "=f"(r[1][7]), "=f"(r[1][8]), "=f"(r[1][9]), "=f"(r[1][10]), "=f"(r[1][11]), "=f"(r[1][12]), "=f"(r[1][13]), "=f"(r[1][14]), "=f"(r[1][15]), "=f"(m[1]),
        "=f"(r[2][0]), "=f"(r[2][1]), "=f"(r[2][2]), "=f"(r[2][3]), "=f"(r[2][4]), "=f"(r[2][5]), "=f"(r[2][6]), "=f"(r[2][7]), "=f"(r[2][8]), "=f"(r[2][9]), "=f"(r[2][10]), "=f"(r[2][11]), "=f"(r[2][12]), "=f"(r[2][13]), "=f"(r[2][14]), "=f"(r[2][15]), "=f"(m[2]),
        "=f"(r[3][0]), "=f"(r[3][1]), "=f"(r[3][2]), "=f"(r[3][3]), "=f"(r[3][4]), "=f"(r[3][5]), "=f"(r[3][6]), "=f"(r[3][7]), "=f"(r[3][8]), "=f"(r[3][9]), "=f"(r[3][10]), "=f"(r[3][11]), "=f"(r[3][12]), "=f"(r[3][13]), "=f"(r[3][14]), "=f"(r[3][15]), "=f"(m[3])
      : "r"(taddr), "r"(taddr + 16u), "r"(taddr + 32u), "r"(taddr + 48u)
      : "memory");
}

// 16 columns of this thread's lane (runtime column), waited for.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]), "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15])
      : "r"(taddr)
      : "memory");
}

// byte offset of (row r, 16-byte piece kc) in a K = 16 BF16 block without swizzle
__device__ __forceinline__ uint32_t ext_off(int r, int kc) {
  return (uint32_t)((r >> 3) * 256 + kc * 128 + (r & 7) * 16);
}

__global__ void __launch_bounds__(kThreadsQ, 1)
k1_tcq_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmQ,
              const TcqArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  const int S = a.stages;
  uint8_t* sA = smem;                                      // queries, SW128
  uint8_t* sB = sA + a.a_bytes;                            // S stages of one K block
  uint8_t* sAext = sB + (size_t)S * kStageBytes;           // ones block (L2)
  uint8_t* sBext = sAext + (a.ext ? kExtA : 0);            // 2 half-norm blocks (L2)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sBext + (a.ext ? kExtSlots * kExtB : 0));
  const uint32_t b_full = smem_u32(bars), b_empty = smem_u32(bars + S);
  const uint32_t b_accf = smem_u32(bars + 2 * S), b_acce = smem_u32(bars + 2 * S + kNumAcc);
  const uint32_t b_xf = smem_u32(bars + 2 * S + 2 * kNumAcc);
  const uint32_t b_xe = smem_u32(bars + 2 * S + 2 * kNumAcc + kExtSlots);
  const uint32_t b_q = smem_u32(bars + 2 * S + 2 * kNumAcc + 2 * kExtSlots);
  const uint32_t b_done = smem_u32(bars + 2 * S + 2 * kNumAcc + 2 * kExtSlots + 1);
  uint32_t* tmem_slot =
      reinterpret_cast<uint32_t*>(bars + 2 * S + 2 * kNumAcc + 2 * kExtSlots + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t qtile = blockIdx.x % a.nqtiles;
  const int64_t range = blockIdx.x / a.nqtiles;
  const int64_t P0 = range * a.rows_per_cta;
  const int64_t P1 = min(a.N, P0 + a.rows_per_cta);
  const int nt = (int)cdiv(P1 - P0, kBN);

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(b_full + 8 * s, 1);
      mbar_init(b_empty + 8 * s, 1);
    }
    for (int b = 0; b < kNumAcc; ++b) {
      mbar_init(b_accf + 8 * b, 1);
      mbar_init(b_acce + 8 * b, 8);
    }
    for (int e = 0; e < kExtSlots; ++e) {
      mbar_init(b_xf + 8 * e, 1);
      mbar_init(b_xe + 8 * e, 1);
    }
    mbar_init(b_q, 1);
    mbar_init(b_done, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (a.ext) {
    // the queries' ones block: K index 0..2 = 1, the rest 0; and the second
    // 16-byte piece of every half-norm block is always zero
    const __nv_bfloat16 one = __float2bfloat16_rn(1.0f), zero = __float2bfloat16_rn(0.0f);
    for (int r = threadIdx.x; r < kQ; r += kThreadsQ) {
      __nv_bfloat16 v[8] = {one, one, one, zero, zero, zero, zero, zero};
      *reinterpret_cast<uint4*>(sAext + ext_off(r, 0)) = *reinterpret_cast<uint4*>(v);
      *reinterpret_cast<uint4*>(sAext + ext_off(r, 1)) = make_uint4(0, 0, 0, 0);
    }
    for (int t = threadIdx.x; t < kExtSlots * kBN; t += kThreadsQ)
      *reinterpret_cast<uint4*>(sBext + (size_t)(t / kBN) * kExtB + ext_off(t % kBN, 1)) =
          make_uint4(0, 0, 0, 0);
    fence_proxy_async_smem();
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), kNumAcc * kBN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // -------------------------------------------------------------- producer
    // The whole warp runs the loop (waits included) and stays converged; one
    // lane issues the copies.
    if (lane == 0) {
      mbar_expect_tx(b_q, a.a_bytes);
      for (int kb = 0; kb < a.nkb; ++kb)
        tma_load_2d(smem_u32(sA + (size_t)kb * kQ * kSpan), &tmQ, b_q, kb * (kSpan / 2),
                    (int)(qtile * kQ));
    }
    __syncwarp();
    // ring position (stage s, phase ph) is kept incrementally: no division
    int s = 0, it = 0, kb = 0, issued = 0;
    uint32_t ph = 0;
    const int total = nt * a.nkb;
    for (int g = 0; g < total; ++g) {
      if (g >= S && !mbar_wait_sleep(b_empty + 8 * s, ph ^ 1u, abort_flag, 64)) break;
      if (lane == 0) {
        mbar_expect_tx(b_full + 8 * s, kStageBytes);
        tma_load_2d(smem_u32(sB + (size_t)s * kStageBytes), &tmX, b_full + 8 * s,
                    kb * (kSpan / 2), (int)(P0 + (int64_t)it * kBN));
      }
      __syncwarp();
      issued = g + 1;
      if (++kb == a.nkb) {
        kb = 0;
        ++it;
      }
      if (++s == S) {
        s = 0;
        ph ^= 1u;
      }
    }
    // drain: the last min(issued, S) copies land before the CTA can exit
    // (walk the ring backwards from the next position)
    for (int k = 0; k < S && k < issued; ++k) {
      if (--s < 0) {
        s = S - 1;
        ph ^= 1u;
      }
      mbar_wait_sleep(b_full + 8 * s, ph, abort_flag, 64);
    }
    mbar_wait_sleep(b_q, 0, abort_flag, 64);
    return;
  }
  if (warp == 1) {
    // -------------------------------------------------------------- MMA issuer
    // The whole warp runs the loop and the waits; one lane issues the MMAs and
    // the commits.
    if (mbar_wait(b_q, 0, abort_flag)) {
      const uint64_t a_desc = smem_desc_sw128(smem_u32(sA));
      const uint64_t b_desc = smem_desc_sw128(smem_u32(sB));
      const uint64_t ax_desc = smem_desc_noswz(smem_u32(sAext), 128, 256);
      const uint64_t bx_desc = smem_desc_noswz(smem_u32(sBext), 128, 256);
      int s = 0;
      uint32_t ph = 0;
      bool run = true;
      for (int it = 0; it < nt && run; ++it) {
        const int ab = it & 1;
        const uint32_t aph = (uint32_t)((it >> 1) & 1);
        if (it >= kNumAcc && !mbar_wait(b_acce + 8 * ab, aph ^ 1u, abort_flag)) break;
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + (uint32_t)(ab * kBN);
        for (int kb = 0; kb < a.nkb; ++kb) {
          if (!mbar_wait(b_full + 8 * s, ph, abort_flag)) {
            run = false;
            break;
          }
          if (lane == 0) {
            // descriptors advance by (bytes >> 4) in their address field
            const uint64_t ad = a_desc + (uint64_t)((kb * kQ * kSpan) >> 4);
            const uint64_t bd = b_desc + (uint64_t)((s * kStageBytes) >> 4);
            const int steps = min(4, a.nksteps - kb * 4);
            for (int kk = 0; kk < steps; ++kk)
              tc_mma<KNN_BF16>(d_tmem, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2),
                               a.idesc, (kb | kk) ? 1u : 0u);
            tc_commit(b_empty + 8 * s);
          }
          __syncwarp();
          if (++s == S) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (!run) break;
        if (a.ext) {
          const int e = it & 1;
          if (!mbar_wait(b_xf + 8 * e, (uint32_t)((it >> 1) & 1), abort_flag)) break;
          if (lane == 0) {
            tc_mma<KNN_BF16>(d_tmem, ax_desc, bx_desc + (uint64_t)((e * kExtB) >> 4), a.idesc,
                             1u);
            tc_commit(b_xe + 8 * e);
          }
          __syncwarp();
        }
        if (lane == 0) tc_commit(b_accf + 8 * ab);
        __syncwarp();
      }
    }
    // all MMAs have completed before tensor memory is released
    if (lane == 0) tc_commit(b_done);
    __syncwarp();
    mbar_wait(b_done, 0, abort_flag);
    asm volatile("bar.sync 1, %0;" ::"n"(32 + 512) : "memory");
    tc_fence_after();
    tmem_dealloc(tmem_base, kNumAcc * kBN);
    return;
  }
  if (warp == 2) {
    // ---------------------------------------------------------- L2 half norms
    if (!a.ext) return;
    // each lane owns rows lane + 32 u (u < 8) of every tile; the loads of the
    // next four tiles are in flight while a tile is written
    float hb[4][8];
    auto load = [&](int it, float (&h)[8]) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t p = P0 + (int64_t)it * kBN + lane + 32 * u;
        h[u] = (it < nt && p < a.N) ? a.hnorm[p] : 0.0f;
      }
    };
#pragma unroll
    for (int k = 0; k < 4; ++k) load(k, hb[k]);
    bool run = true;
    for (int it0 = 0; it0 < nt && run; it0 += 4) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int it = it0 + k;
        if (it >= nt || !run) break;
        const int e = it & 1;
        int ok = 1;
        if (lane == 0 && it >= kExtSlots)
          ok = mbar_wait_sleep(b_xe + 8 * e, (uint32_t)(((it >> 1) & 1) ^ 1), abort_flag, 64) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          run = false;
          break;
        }
        uint8_t* ext = sBext + (size_t)e * kExtB;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float h = hb[k][u];
          const __nv_bfloat16 hi = __float2bfloat16_rn(h);
          const float rem1 = h - __bfloat162float(hi);
          const __nv_bfloat16 mid = __float2bfloat16_rn(rem1);
          const __nv_bfloat16 lo = __float2bfloat16_rn(rem1 - __bfloat162float(mid));
          const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
          __nv_bfloat16 v[8] = {__hneg(hi), __hneg(mid), __hneg(lo), z, z, z, z, z};
          *reinterpret_cast<uint4*>(ext + ext_off(lane + 32 * u, 0)) =
              *reinterpret_cast<uint4*>(v);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(b_xf + 8 * e);
        load(it + 4, hb[k]);
      }
    }
    return;
  }
  if (warp < 4) return;

  // ---------------------------------------------------------------- epilogue
  const int quad = warp & 3;
  const int egrp = (warp - 4) >> 2;  // 0..3
  const int ab = egrp & 1;           // accumulator buffer = tile parity
  const int chalf = egrp >> 1;       // columns chalf*128 .. +127 of each tile
  const int64_t qi = qtile * kQ + quad * 32 + lane;
  const bool q_ok = qi < a.M;
  unsigned long long* gq = a.G + (q_ok ? qi : 0) * a.L;
  int64_t cur_bin = bin_of(P0, a.bq, a.br);
  int64_t seg_end = bin_end(cur_bin, a.bq, a.br);
  float best = __uint_as_float(kNegInfBits);
  int64_t best_row = -1;
  auto flush = [&]() {
    if (q_ok && best_row >= 0)
      atomicMax(&gq[cur_bin], (unsigned long long)make_key(best, (int32_t)best_row));
  };
  for (int it = ab; it < nt; it += 2) {
    const uint32_t aph = (uint32_t)((it >> 1) & 1);
    if (!mbar_wait_sleep(b_accf + 8 * ab, aph, abort_flag, 128)) break;
    tc_fence_after();
    const uint32_t tbase = tmem_base + ((uint32_t)(quad * 32) << 16) +
                           (uint32_t)(ab * kBN + chalf * 128);
    const int64_t pbase = P0 + (int64_t)it * kBN + chalf * 128;
#pragma unroll 1
    for (int rd = 0; rd < 2; ++rd) {
      const int64_t p0 = pbase + rd * 64;
      const uint32_t tcol = tbase + (uint32_t)(rd * 64);
      if (p0 >= P1) break;  // warp-uniform
      if (p0 + 64 <= seg_end && p0 + 64 <= P1) {
        // common case: the 64 rows lie inside the current bin (warp-uniform):
        // one compare per 16 scores
        float r[4][16], m[4];
        __syncwarp();
        tmem_ld4x16_max(tcol, r, m);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          if (m[g] > best) {
            int pos = 0;
#pragma unroll
            for (int k = 15; k >= 0; --k) pos = (r[g][k] == m[g]) ? k : pos;
            best = m[g];
            best_row = p0 + g * 16 + pos;
          }
        }
      } else {
        // a bin boundary or the end of the range falls in these rows (rare):
        // walk them column by column, 16 at a time
#pragma unroll 1
        for (int g = 0; g < 4; ++g) {
          const int64_t pg = p0 + g * 16;
          if (pg >= P1) break;  // warp-uniform
          float r[16];
          __syncwarp();
          tmem_ld16(tcol + (uint32_t)(g * 16), r);
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int64_t p = pg + k;
            if (p < P1) {
              while (p >= seg_end) {
                flush();
                ++cur_bin;
                seg_end = bin_end(cur_bin, a.bq, a.br);
                best = __uint_as_float(kNegInfBits);
                best_row = -1;
              }
              if (r[k] > best) {
                best = r[k];
                best_row = p;
              }
            }
          }
        }
      }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(b_acce + 8 * ab);
  }
  tc_fence_before();
  asm volatile("bar.arrive 1, %0;" ::"n"(32 + 512) : "memory");
  flush();
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode_q() {
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

bool make_map_bf16(CUtensorMap* m, const void* base, int64_t rows, int pitch, int box_rows) {
  auto enc = get_encode_q();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
  cuuint32_t box[2] = {(cuuint32_t)(kSpan / 2), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct TcqShape {
  int nkb, nksteps, stages;
  uint32_t a_bytes;
  size_t smem;
};

bool tcq_shape(int D, int metric, TcqShape* sh) {
  const int pitch = (int)round_up(D, 16);
  sh->nkb = (int)cdiv((int64_t)pitch * 2, kSpan);
  sh->nksteps = (int)cdiv((int64_t)pitch * 2, 32);
  sh->a_bytes = (uint32_t)(sh->nkb * kQ * kSpan);
  const int ext = metric == KNN_L2;
  const size_t fixed = 1024 + sh->a_bytes + (ext ? kExtA + kExtSlots * kExtB : 0) + 512;
  const size_t budget = 227 * 1024;
  if (fixed + 3 * (size_t)kStageBytes > budget) return false;
  int stages = (int)((budget - fixed) / kStageBytes);
  sh->stages = stages > 8 ? 8 : stages;
  sh->smem = fixed + (size_t)sh->stages * kStageBytes;
  return true;
}

}  // namespace

bool k1_tcq_supported(int dtype, int D, int metric) {
  TcqShape sh;
  return dtype == KNN_BF16 && metric >= KNN_IP && metric <= KNN_COS && tcq_shape(D, metric, &sh);
}

void k1_tcq_grid(int64_t N, int64_t M, int64_t* nqtiles, int64_t* nranges, int64_t* rows_per_cta) {
  const int64_t sms = device_sm_count();
  *nqtiles = cdiv(M, kQ);
  int64_t nr = *nqtiles >= sms ? 1 : (sms + *nqtiles / 2) / *nqtiles;
  const int64_t ntile = cdiv(N, kBN);
  if (nr > ntile) nr = ntile;
  if (nr < 1) nr = 1;
  *rows_per_cta = cdiv(ntile, nr) * kBN;
  *nranges = cdiv(N, *rows_per_cta);
}

cudaError_t launch_k1_tcq(int64_t N, int64_t M, int64_t L, int D, int metric, const void* X,
                          const float* hnorm, const void* Qp, unsigned long long* G,
                          cudaStream_t st) {
  TcqShape sh;
  if (!tcq_shape(D, metric, &sh)) return cudaErrorNotSupported;
  if (metric == KNN_L2 && !hnorm) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (reinterpret_cast<uintptr_t>(Qp) & 15))
    return cudaErrorInvalidValue;
  if (M <= 0) return cudaSuccess;
  TcqArgs a{};
  a.N = N;
  a.M = M;
  a.L = L;
  a.bq = N / L;
  a.br = N % L;
  k1_tcq_grid(N, M, &a.nqtiles, &a.nranges, &a.rows_per_cta);
  a.nkb = sh.nkb;
  a.nksteps = sh.nksteps;
  a.stages = sh.stages;
  a.a_bytes = sh.a_bytes;
  a.ext = metric == KNN_L2 ? 1 : 0;
  // D = F32, A = B = BF16, both K-major, N = 128, M = 128
  a.idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
            ((uint32_t)(kQ >> 4) << 24);
  a.hnorm = hnorm;
  a.G = G;
  const int pitch = (int)round_up(D, 16);
  CUtensorMap mx, mq;
  if (!make_map_bf16(&mx, X, N, pitch, kBN)) return cudaErrorInvalidValue;
  if (!make_map_bf16(&mq, Qp, M, pitch, kQ)) return cudaErrorInvalidValue;
  const int64_t blocks = a.nqtiles * a.nranges;
  cudaError_t e = cudaFuncSetAttribute(k1_tcq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sh.smem);
  if (e != cudaSuccess) return e;
  k1_tcq_kernel<<<(unsigned)blocks, kThreadsQ, sh.smem, st>>>(mx, mq, a);
  return cudaGetLastError();
}

bool k1_tcq_take_timeout() { return tc_take_timeout_local(); }

}  // namespace tpuknn
