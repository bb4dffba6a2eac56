// k1_tcs.cu -- PartialReduce with bins j mod L (Alg. 1) fused with a tcgen05
// BF16 contraction, queries on the tensor-memory lanes and each bin's rows
// side by side in the accumulator.
//
// Row j = t*L + b lies in bin b; the database is read as a [T x L*pitch] grid
// (grid row t holds rows t*L .. t*L + L - 1). One pipeline step covers 16 bins
// b0..b0+15 and 16 grid rows t0..t0+15: 256 database rows, loaded per K block
// by ONE 3-D TMA box whose outer dimension is the bin, so accumulator column
// n = (b - b0)*16 + (t - t0)
// and every run of 16 consecutive columns holds 16 rows of ONE bin. The
// epilogue reduces such a run with a single tcgen05.ld.red.max (the load
// returns the 16 scores and their maximum) and compares the maximum once with
// the bin's best so far; only on a new best does it look for the column. That
// is about one compare per 16 scores instead of a compare (and a key pack)
// per score, which keeps the CUDA-core work well below the tensor-core time.
//
// One CTA (640 threads, one per SM) owns a contiguous run of steps and takes
// kq query tiles of 256 (two M = 128 halves, A operand resident in shared
// memory) in turn over it, one segment each; kq > 1 only when the tiles do
// not spread evenly over the SMs (the host picks kq and the runs):
//   warp 0      : TMA producer (the query tile once per segment; per step and
//                 128-byte K block one 16 x 16-row box into a 32 KB stage of
//                 an S-stage ring).
//   warp 1      : TMEM allocation (512 columns: one 128 x 256 FP32 accumulator
//                 per query half) and tcgen05.mma issue. Half 0 of a step is
//                 computed and handed to its epilogue while half 1 is
//                 computed, so each half's drain overlaps the other's MMAs.
//   warp 2      : (L2 only) each step's half norms as an extra K = 16 block
//                 (-h split into three BF16 parts against a ones block of the
//                 queries), so the accumulator holds the relaxed score
//                 <q,x> - |x|^2/2 (App. A.2, Eq. 19).
//   warps 4..19 : epilogue, four warpgroups (query half x column half); a
//                 thread owns one query and 8 bins of the step; it keeps each
//                 bin's best score and grid row, and when the CTA moves to
//                 the next group of bins it merges them into G[query][bin] by
//                 64-bit atomicMax on the ordered key (score, ~row): ties
//                 keep the smaller row, and bins split between CTAs merge
//                 exactly.
//   warp 3      : idle.
// Steps that reach past the last full grid row or the last bin take a
// column-by-column path with a validity test. Rows of the ragged last grid
// row (t = floor(N/L), b < N mod L) are scored by k1_tcs_tail. All waits are
// bounded (see tc_ptx.cuh).
#include <algorithm>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "dtypes.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace tpuknn {

namespace {

constexpr int kThreadsS = 640;   // 4 control warps + 4 epilogue warpgroups
constexpr int kQH = 128;         // queries per half: MMA M, TMEM lanes
constexpr int kQT = 256;         // queries per CTA
constexpr int kRowsBin = 16;     // grid rows per bin per step
constexpr int kSpanS = 128;      // bytes of one 128-byte swizzle span (one K block)
constexpr int kExtAS = kQH * 32;             // ones block (K = 16 BF16)

// Step layouts: BS bins x 16 grid rows (or BS * 16 consecutive rows) per step.
//   BS = 16: MMA N = 256, one accumulator per query half, 32 KB stages; the
//            layout of the K-loop modes (rows longer than 128 elements).
//   BS = 8 : MMA N = 128, two accumulators per query half (a step's MMAs
//            write the buffer the step before last used, so they never wait
//            for the previous step's drain), 16 KB stages: twice as many steps
//            fit in the ring, which hides more of the load latency.
template <int BS>
struct StepT {
  static constexpr int kCols = BS * kRowsBin;   // MMA N, accumulator columns
  static constexpr int kStage = kCols * kSpanS; // one K block of a step
  static constexpr int kExtB = kCols * 32;      // half-norm block of a step
  static constexpr int kNB = BS == 8 ? 2 : 1;   // accumulators per query half
  static constexpr int kXS = BS == 8 ? 4 : 2;   // half-norm block slots
  static constexpr int kBPW = BS / 2;           // bins per epilogue warpgroup
};
// Register split (setmaxnreg): the control warpgroup gives up registers so
// the epilogue can keep four 16-column runs in flight. 128*64 + 512*104 =
// 61440 = 640*96, the registers the kernel is launched with (checked on the
// host before every launch).
constexpr int kCtrlRegsS = 64, kEpiRegsS = 104;

struct TcsArgs {
  int64_t N, M, L, T;              // T = floor(N / L) full grid rows
  int64_t ntg, nbg;                // grid-row groups of 16, bin groups of 16 (j mod L)
  int64_t bq, br;                  // contiguous bins: q = N / L, r = N mod L
  int64_t steps_per_q, nqt;        // steps over the whole database; query tiles
  int64_t parts, steps_per_part;   // the database steps split into `parts` ranges
  int64_t kq, groups;              // query tiles one CTA takes in turn; tile groups
  int pitch;                       // row length in elements (multiple of 16)
  int nkb, nksteps, stages;
  uint32_t stage_bytes;            // one K block of a step (+ of the queries when streamed)
  uint32_t a_bytes;
  int ext;
  uint32_t idesc;
  const float* hnorm;
  const float* xscale;             // E4M3: the database-wide scale (xscale[0])
  unsigned long long* G;
};

// 64 columns of this thread's lane as four runs of 16 with their maxima, waited for.
__device__ __forceinline__ void tmem_ld4x16_max_s(uint32_t taddr, float (&r)[4][16], float (&m)[4]) {
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

// 16 columns of this thread's lane, waited for.
__device__ __forceinline__ void tmem_ld16s(uint32_t taddr, float (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3]), "=f"(r[4]), "=f"(r[5]), "=f"(r[6]), "=f"(r[7]), "=f"(r[8]), "=f"(r[9]), "=f"(r[10]), "=f"(r[11]), "=f"(r[12]), "=f"(r[13]), "=f"(r[14]), "=f"(r[15])
      : "r"(taddr)
      : "memory");
}

// byte offset of (row r, 16-byte piece kc) in a K = 16 BF16 block without swizzle
__device__ __forceinline__ uint32_t ext_off_s(int r, int kc) {
  return (uint32_t)((r >> 3) * 256 + kc * 128 + (r & 7) * 16);
}

// Modes of the K loop:
//   kFused   : rows up to 128 elements. The whole step's K blocks are resident
//              together; each query half runs all its MMAs in one unrolled run
//              (NKS K-steps), so each half's drain overlaps the other's MMAs.
//   kKLoopA  : longer rows, query tile resident. The step walks its K blocks
//              one stage at a time, each stage feeding both halves; both
//              accumulators close at the end of the step (their drain is short
//              against a long step).
//   kKLoopQ  : rows too long for a resident query tile: a stage carries the K
//              block of the 256 queries too.
constexpr int kFused = 0, kKLoopA = 1, kKLoopQ = 2;

// Bin maps: kBinsMod (bin = j mod L, steps over the [T][L] grid view) and
// kBinsRun (Alg. 1's ShiftRight generalised to L balanced runs of consecutive
// rows; a step is 256 consecutive rows, and a thread follows one current bin).
constexpr int kBinsMod = 0, kBinsRun = 1;

__device__ __forceinline__ int64_t run_bin_of(int64_t p, int64_t q, int64_t r) {
  const int64_t big = r * (q + 1);
  return p < big ? p / (q + 1) : r + (p - big) / q;
}
__device__ __forceinline__ int64_t run_bin_end(int64_t b, int64_t q, int64_t r) {
  return (b + 1) * q + min(b + 1, r);
}

template <int NKS, int MODE, int BM, int BS, int DT>
__global__ void __launch_bounds__(kThreadsS, 1)
k1_tcs_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmQ,
              const TcsArgs a) {
  using T = StepT<BS>;
  constexpr int kCols = T::kCols, NB = T::kNB, XS = T::kXS, BPW = T::kBPW;
  // elements of one 128-byte K block (the x coordinate of a K block's box)
  constexpr int kElS = DT == KNN_E4M3 ? kSpanS : kSpanS / 2;
  static_assert(MODE == kFused || BS == 16, "the K-loop modes use 16-bin steps");
  // 128-byte K blocks per step
  const int NKB = MODE == kFused ? (NKS + 3) / 4 : a.nkb;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  const int S = a.stages;
  uint8_t* sA = smem;                                      // queries, SW128, [kb][256][128 B]
  uint8_t* sB = sA + a.a_bytes;                            // S stages of one K block
  uint8_t* sAext = sB + (size_t)S * a.stage_bytes;         // ones block (L2)
  uint8_t* sBext = sAext + (a.ext ? kExtAS : 0);           // XS half-norm blocks (L2)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sBext + (a.ext ? XS * T::kExtB : 0));
  // accumulator (h, buf) of query half h: barriers b_accf / b_acce + 8 (h NB + buf),
  // TMEM columns (h NB + buf) kCols
  constexpr int NACC = 2 * NB;
  const uint32_t b_full = smem_u32(bars), b_empty = smem_u32(bars + S);
  const uint32_t b_accf = smem_u32(bars + 2 * S), b_acce = smem_u32(bars + 2 * S + NACC);
  const uint32_t b_xf = smem_u32(bars + 2 * S + 2 * NACC);
  const uint32_t b_xe = smem_u32(bars + 2 * S + 2 * NACC + XS);
  const uint32_t b_q = smem_u32(bars + 2 * S + 2 * NACC + 2 * XS);
  const uint32_t b_done = smem_u32(bars + 2 * S + 2 * NACC + 2 * XS + 1);
  const uint32_t b_qe = smem_u32(bars + 2 * S + 2 * NACC + 2 * XS + 2);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 2 * NACC + 2 * XS + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // CTA = (part, group): the steps [s_begin, s_end) of the database for the
  // query tiles q0 .. q0 + nseg - 1, one after the other (a segment each).
  // The CTAs of one part walk the same rows at the same time, so the rows
  // they share meet in L2; their block indices are adjacent, which keeps
  // them on neighbouring SMs (the same die). Step i of the CTA is step
  // i mod ns of segment i / ns; barrier phases count i across segments.
  const int64_t part = blockIdx.x / a.groups;
  const int64_t q0 = (blockIdx.x % a.groups) * a.kq;
  const int nseg = (int)max((int64_t)0, min(a.kq, a.nqt - q0));
  const int64_t s_begin = part * a.steps_per_part;
  const int64_t s_end = min(a.steps_per_q, s_begin + a.steps_per_part);
  const int ns = (int)max((int64_t)0, s_end - s_begin);
  const int nt = nseg * ns;  // steps of this CTA

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(b_full + 8 * s, 1);
      mbar_init(b_empty + 8 * s, 1);
    }
    for (int c = 0; c < NACC; ++c) {
      mbar_init(b_accf + 8 * c, 1);
      mbar_init(b_acce + 8 * c, 8);  // the 8 warps of the two warpgroups of a half
    }
    for (int e = 0; e < XS; ++e) {
      mbar_init(b_xf + 8 * e, 1);
      mbar_init(b_xe + 8 * e, 1);
    }
    mbar_init(b_q, 1);
    mbar_init(b_done, 1);
    mbar_init(b_qe, 1);
    *abort_flag = 0;
    fence_barrier_init();
  }
  if (a.ext) {
    // the queries' ones block: K index 0..2 = 1, the rest 0; and the second
    // 16-byte piece of every half-norm block is always zero
    const __nv_bfloat16 one = __float2bfloat16_rn(1.0f), zero = __float2bfloat16_rn(0.0f);
    for (int r = threadIdx.x; r < kQH; r += kThreadsS) {
      __nv_bfloat16 v[8] = {one, one, one, zero, zero, zero, zero, zero};
      *reinterpret_cast<uint4*>(sAext + ext_off_s(r, 0)) = *reinterpret_cast<uint4*>(v);
      *reinterpret_cast<uint4*>(sAext + ext_off_s(r, 1)) = make_uint4(0, 0, 0, 0);
    }
    for (int t = threadIdx.x; t < XS * kCols; t += kThreadsS)
      *reinterpret_cast<uint4*>(sBext + (size_t)(t / kCols) * T::kExtB + ext_off_s(t % kCols, 1)) =
          make_uint4(0, 0, 0, 0);
    fence_proxy_async_smem();
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // the prologue above touches no global memory; the queries and the zeroed
  // key array come from the preceding kernel
  pdl_wait();
  pdl_trigger();

  if (warp < 4) asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kCtrlRegsS));
  if (warp == 0) {
    // -------------------------------------------------------------- producer
    int s = 0, issued = 0, q_armed = 0;
    uint32_t ph = 0;
    bool prun = true;
    for (int sg = 0; sg < nseg && prun; ++sg) {
    const int64_t qtile = q0 + sg;
    // the segment's query tile (phase sg of b_q); from the second segment on
    // only after the MMAs of the previous one are done with the old tile
    if (MODE != kKLoopQ && sg > 0 &&
        !warp_all(mbar_wait_sleep(b_qe, (uint32_t)((sg - 1) & 1), abort_flag)))
      break;
    q_armed = sg + 1;
    if (lane == 0) {
      if (MODE == kKLoopQ) {
        mbar_arrive(b_q);  // the queries come with every stage
      } else {
        mbar_expect_tx(b_q, a.a_bytes);
        for (int kb = 0; kb < NKB; ++kb)
          tma_load_2d(smem_u32(sA + (size_t)kb * kQT * kSpanS), &tmQ, b_q, kb * kElS,
                      (int)(qtile * kQT));
      }
    }
    __syncwarp();
    int kb = 0;
    int64_t bg = s_begin / a.ntg, tg = s_begin % a.ntg;
    const int total = ns * NKB;
    for (int g = 0; g < total; ++g) {
      if (issued >= S && !warp_all(mbar_wait_sleep(b_empty + 8 * s, ph ^ 1u, abort_flag))) {
        prun = false;
        break;
      }
      if (lane == 0) {
        mbar_expect_tx(b_full + 8 * s, a.stage_bytes);
        uint32_t dst = smem_u32(sB + (size_t)s * a.stage_bytes);
        if (MODE == kKLoopQ) {
          // the queries' K block first: [256 queries][128 B]
          tma_load_2d(dst, &tmQ, b_full + 8 * s, kb * kElS, (int)(qtile * kQT));
          dst += kQT * kSpanS;
        }
        if constexpr (BM == kBinsRun) {
          // kCols consecutive rows; rows past N read the fill value (zero)
          tma_load_2d(dst, &tmX, b_full + 8 * s, kb * kElS,
                      (int)((s_begin + g / NKB) * kCols));
        } else {
          // one box: K block kb (128 bytes), grid rows tg*16 .. +15, bins
          // bg*BS .. +BS-1, landing as [bin][grid row][128 B]; bins past L,
          // rows past T and elements past the row read the fill value (zero)
          tma_load_3d(dst, &tmX, b_full + 8 * s, kb * kElS, (int)(tg * kRowsBin),
                      (int)(bg * BS));
        }
      }
      __syncwarp();
      ++issued;
      if (++kb == NKB) {
        kb = 0;
        if (++tg == a.ntg) {
          tg = 0;
          ++bg;
        }
      }
      if (++s == S) {
        s = 0;
        ph ^= 1u;
      }
    }
    }
    // the copies still in flight land before the CTA can exit, also after a
    // give-up: the last min(issued, S) stages and the last query tile armed
    for (int k = 0; k < S && k < issued; ++k) {
      if (--s < 0) {
        s = S - 1;
        ph ^= 1u;
      }
      mbar_drain(b_full + 8 * s, ph);
    }
    if (MODE != kKLoopQ && q_armed > 0) mbar_drain(b_q, (uint32_t)((q_armed - 1) & 1));
    return;
  }
  if (warp == 1) {
    // -------------------------------------------------------------- MMA issuer
    // The whole warp runs the loop and the waits; one lane issues. The tensor
    // pipe holds few instructions, so nothing slow sits between the MMAs of a
    // half: every wait of a step (its stages, its L2 block, the accumulator
    // being free) comes before the unrolled run of MMAs it guards, and the
    // commits come after.
    // b_q phase sg: the query tile of segment sg has landed; a commit to b_qe
    // after a segment's last MMAs frees the tile for the next one
    if constexpr (MODE == kFused) {
    {
      const uint64_t a_desc = smem_desc_sw128(smem_u32(sA));
      const uint64_t b_desc = smem_desc_sw128(smem_u32(sB));
      const uint64_t ax_desc = smem_desc_noswz(smem_u32(sAext), 128, 256);
      const uint64_t bx_desc = smem_desc_noswz(smem_u32(sBext), 128, 256);
      int s0 = 0;           // stage of K block 0 of the current step
      uint32_t ph0 = 0;
      bool run = true;
      for (int sg = 0; sg < nseg && run; ++sg) {
      if (!warp_all(mbar_wait(b_q, (uint32_t)(sg & 1), abort_flag))) break;
      for (int li = 0; li < ns && run; ++li) {
        const int i = sg * ns + li;
        const int e = i % XS;
        const int buf = NB == 2 ? (i & 1) : 0;
        // the stages of this step (NKB consecutive ring slots)
        int sk[(NKS + 3) / 4];
        {
          int s = s0;
          uint32_t ph = ph0;
#pragma unroll
          for (int kb = 0; kb < NKB; ++kb) {
            sk[kb] = s;
            if (run && !warp_all(mbar_wait(b_full + 8 * s, ph, abort_flag))) run = false;
            if (++s == S) {
              s = 0;
              ph ^= 1u;
            }
          }
          s0 = s;
          ph0 = ph;
        }
        if (!run) break;
        if (a.ext && !warp_all(mbar_wait(b_xf + 8 * e, (uint32_t)((i / XS) & 1), abort_flag))) {
          run = false;
          break;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          // the accumulator's previous use (step i - NB) has been drained
          const int c = h * NB + buf;
          if (i >= NB &&
              !warp_all(mbar_wait(b_acce + 8 * c, (uint32_t)(((i / NB) & 1) ^ 1), abort_flag))) {
            run = false;
            break;
          }
          tc_fence_after();
          if (lane == 0) {
            const uint32_t d_tmem = tmem_base + (uint32_t)(c * kCols);
            const uint64_t ah = a_desc + (uint64_t)((h * kQH * kSpanS) >> 4);
#pragma unroll
            for (int ks = 0; ks < NKS; ++ks) {
              // descriptors advance by (bytes >> 4) in their address field
              const uint64_t ad = ah + (uint64_t)(((ks >> 2) * kQT * kSpanS + (ks & 3) * 32) >> 4);
              const uint64_t bd =
                  b_desc + (uint64_t)((sk[ks >> 2] * T::kStage + (ks & 3) * 32) >> 4);
              tc_mma<DT>(d_tmem, ad, bd, a.idesc, ks > 0 ? 1u : 0u);
              // half 1 is a K block's last reader: its stage is free once the
              // MMAs so far complete (2-3% faster than freeing all stages of
              // the step after the half's last MMA)
              if (h == 1 && ((ks & 3) == 3 || ks == NKS - 1)) tc_commit(b_empty + 8 * sk[ks >> 2]);
            }
            if (a.ext)
              tc_mma<KNN_BF16>(d_tmem, ax_desc, bx_desc + (uint64_t)((e * T::kExtB) >> 4),
                               a.idesc, 1u);
            tc_commit(b_accf + 8 * c);
            if (h == 1 && a.ext) tc_commit(b_xe + 8 * e);
          }
          __syncwarp();
        }
      }
      if (!run) break;
      if (lane == 0) tc_commit(b_qe);
      __syncwarp();
      }
    }
    }
    if constexpr (MODE != kFused) {
    {
      const uint64_t a_desc = smem_desc_sw128(smem_u32(sA));
      const uint64_t ax_desc = smem_desc_noswz(smem_u32(sAext), 128, 256);
      const uint64_t bx_desc = smem_desc_noswz(smem_u32(sBext), 128, 256);
      int s = 0;
      uint32_t ph = 0;
      bool run = true;
      for (int sg = 0; sg < nseg && run; ++sg) {
      if (!warp_all(mbar_wait(b_q, (uint32_t)(sg & 1), abort_flag))) break;
      for (int li = 0; li < ns && run; ++li) {
        const int i = sg * ns + li;
        const int e = i % XS;
        // both accumulators are written from the first K block on
        if (i >= 1 && (!warp_all(mbar_wait(b_acce, (uint32_t)((i & 1) ^ 1), abort_flag)) ||
                       !warp_all(mbar_wait(b_acce + 8, (uint32_t)((i & 1) ^ 1), abort_flag)))) {
          run = false;
          break;
        }
        for (int kb = 0; kb < NKB; ++kb) {
          if (!warp_all(mbar_wait(b_full + 8 * s, ph, abort_flag))) {
            run = false;
            break;
          }
          tc_fence_after();
          if (lane == 0) {
            const uint32_t st = smem_u32(sB + (size_t)s * a.stage_bytes);
            const uint64_t bd = smem_desc_sw128(MODE == kKLoopQ ? st + kQT * kSpanS : st);
            const int steps = min(4, a.nksteps - kb * 4);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const uint32_t d_tmem = tmem_base + (uint32_t)(h * kCols);
              // descriptors advance by (bytes >> 4) in their address field
              const uint64_t ad =
                  MODE == kKLoopQ
                      ? smem_desc_sw128(st + (uint32_t)(h * kQH * kSpanS))
                      : a_desc + (uint64_t)((kb * kQT * kSpanS + h * kQH * kSpanS) >> 4);
#pragma unroll
              for (int kk = 0; kk < 4; ++kk)
                if (kk < steps)
                  tc_mma<DT>(d_tmem, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), a.idesc,
                             (kb | kk) ? 1u : 0u);
            }
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
          if (!warp_all(mbar_wait(b_xf + 8 * e, (uint32_t)((i / XS) & 1), abort_flag))) {
            run = false;
            break;
          }
          tc_fence_after();
        }
        if (lane == 0) {
          if (a.ext) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
              tc_mma<KNN_BF16>(tmem_base + (uint32_t)(h * kCols), ax_desc,
                               bx_desc + (uint64_t)((e * T::kExtB) >> 4), a.idesc, 1u);
            tc_commit(b_xe + 8 * e);
          }
          tc_commit(b_accf);
          tc_commit(b_accf + 8);
        }
        __syncwarp();
      }
      if (!run) break;
      if (lane == 0) tc_commit(b_qe);
      __syncwarp();
      }
    }
    }
    // all MMAs have completed before tensor memory is released (also after a
    // give-up: the MMAs already issued still write their accumulators)
    if (lane == 0) tc_commit(b_done);
    __syncwarp();
    mbar_drain(b_done, 0);
    asm volatile("bar.sync 1, %0;" ::"n"(32 + 512) : "memory");
    tc_fence_after();
    tmem_dealloc(tmem_base, 512);
    return;
  }
  if (warp == 2) {
    // ---------------------------------------------------------- L2 half norms
    if (!a.ext) return;
    // column n = j*16 + u of a step is bin b0 + j, grid row t0 + u. Lane l
    // writes columns c = l + 32 k (k < HK), i.e. j = c % BS, u = c / BS, so
    // that lanes 0..BS-1 read BS consecutive floats of one grid row. The loads
    // run PD - 1 steps ahead of the step being written (registers hb[PD]), so
    // their latency hides behind that many steps.
    constexpr int HK = kCols / 32;
    constexpr int PD = BS == 8 ? 4 : 2;
    float hb[PD][HK];
    int64_t bg = s_begin / a.ntg, tg = s_begin % a.ntg;
    // (with contiguous bins: column n is row step*kCols + n)
    int64_t rstep = s_begin;  // contiguous bins: the step being loaded
    auto load = [&](int64_t bgx, int64_t tgx, bool live, float (&h)[HK]) {
#pragma unroll
      for (int k = 0; k < HK; ++k) {
        const int c = lane + 32 * k;
        if constexpr (BM == kBinsRun) {
          const int64_t p = rstep * kCols + c;
          h[k] = (live && p < a.N) ? a.hnorm[p] : 0.0f;
        } else {
          const int64_t b = bgx * BS + (c % BS);
          const int64_t t = tgx * kRowsBin + (c / BS);
          h[k] = (live && b < a.L && t < a.T) ? a.hnorm[t * a.L + b] : 0.0f;
        }
      }
      if (++rstep == s_end) rstep = s_begin;  // the next segment repeats the steps
    };
    int64_t bgn = bg, tgn = tg;
    int lsn = 0;  // step within the segment of (bgn, tgn)
    auto advance = [&](int64_t& b, int64_t& t) {
      if (++t == a.ntg) {
        t = 0;
        ++b;
      }
      if (++lsn == ns) {
        lsn = 0;
        b = s_begin / a.ntg;
        t = s_begin % a.ntg;
      }
    };
#pragma unroll
    for (int k = 0; k < PD - 1; ++k) {
      load(bgn, tgn, k < nt, hb[k]);
      advance(bgn, tgn);
    }
    bool run = true;
    for (int i0 = 0; i0 < nt && run; i0 += PD) {
#pragma unroll
      for (int cur = 0; cur < PD; ++cur) {
        const int i = i0 + cur;
        if (i >= nt) break;
        load(bgn, tgn, i + PD - 1 < nt, hb[(cur + PD - 1) % PD]);
        advance(bgn, tgn);
        const int e = i % XS;
        int ok = 1;
        if (lane == 0 && i >= XS)
          ok = mbar_wait_sleep(b_xe + 8 * e, (uint32_t)(((i / XS) & 1) ^ 1), abort_flag) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          run = false;
          break;
        }
        uint8_t* ext = sBext + (size_t)e * T::kExtB;
#pragma unroll
        for (int k = 0; k < HK; ++k) {
          const int c = lane + 32 * k;
          const int n = BM == kBinsRun ? c : (c % BS) * kRowsBin + (c / BS);
          const float hv = hb[cur][k];  // loaded PD - 1 steps ago
          const __nv_bfloat16 hi = __float2bfloat16_rn(hv);
          const float rem1 = hv - __bfloat162float(hi);
          const __nv_bfloat16 mid = __float2bfloat16_rn(rem1);
          const __nv_bfloat16 lo = __float2bfloat16_rn(rem1 - __bfloat162float(mid));
          const __nv_bfloat16 z = __float2bfloat16_rn(0.0f);
          __nv_bfloat16 v[8] = {__hneg(hi), __hneg(mid), __hneg(lo), z, z, z, z, z};
          *reinterpret_cast<uint4*>(ext + ext_off_s(n, 0)) = *reinterpret_cast<uint4*>(v);
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(b_xf + 8 * e);
      }
    }
    return;
  }
  if (warp < 4) return;

  // ---------------------------------------------------------------- epilogue
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kEpiRegsS));
  const int quad = warp & 3;
  const int egrp = (warp - 4) >> 2;  // 0..3
  const int h = egrp >> 1;           // query half
  const int cq = egrp & 1;           // bins cq*BPW .. cq*BPW+BPW-1 of each step
  constexpr int NLD = BPW / 4;       // 64-column loads per step and thread
  // this thread's query in the current segment
  bool q_ok = false;
  unsigned long long* gq = a.G;
  // E4M3: keys hold the raw dot of the codes times the database scale (the
  // per-query scale is left out: it does not change the order in a query)
  const float xs0 = DT == KNN_E4M3 ? a.xscale[0] : 1.0f;
  auto scaled = [&](float v) { return DT == KNN_E4M3 ? __fmul_rn(v, xs0) : v; };
  auto set_query = [&](int sg) {
    const int64_t qi = (q0 + sg) * kQT + h * kQH + quad * 32 + lane;
    q_ok = qi < a.M;
    gq = a.G + (q_ok ? qi : 0) * a.L;
  };
  // TMEM lanes of this warp and this warpgroup's columns of an accumulator
  const uint32_t tlane = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(cq * BPW * 16);
  auto acc_cols = [&](int buf) { return tlane + (uint32_t)((h * NB + buf) * kCols); };
  if constexpr (BM == kBinsRun) {
    // Contiguous bins: this warpgroup sees rows s*kCols + cq*kCols/2 .. + kCols/2 - 1
    // of every step s, in increasing order. A thread follows the current bin
    // (the same for every lane: bins depend on rows only) with its best score
    // and row, and merges it into G when the rows leave the bin.
    const int64_t first = min((s_begin * kCols + cq * (kCols / 2)), a.N - 1);
    int64_t cur = 0, seg_end = 0, brow = -1;
    float bv = __uint_as_float(kNegInfBits);
    auto flush_run = [&]() {
      if (q_ok && brow >= 0)
        atomicMax(&gq[cur], (unsigned long long)make_key(scaled(bv), (int32_t)brow));
    };
    bool erun = true;
    for (int sg = 0; sg < nseg && erun; ++sg) {
    if (sg > 0) flush_run();
    set_query(sg);
    cur = run_bin_of(first, a.bq, a.br);
    seg_end = run_bin_end(cur, a.bq, a.br);
    bv = __uint_as_float(kNegInfBits);
    brow = -1;
    for (int li = 0; li < ns; ++li) {
      const int i = sg * ns + li;
      const int buf = NB == 2 ? (i & 1) : 0;
      if (!warp_all(mbar_wait_sleep(b_accf + 8 * (h * NB + buf), (uint32_t)((i / NB) & 1),
                                    abort_flag))) {
        erun = false;
        break;
      }
      tc_fence_after();
      const int64_t p0 = (s_begin + li) * kCols + cq * (kCols / 2);
      const uint32_t tb = acc_cols(buf);
#pragma unroll
      for (int half64 = 0; half64 < NLD; ++half64) {
        float r[4][16], m[4];
        __syncwarp();
        tmem_ld4x16_max_s(tb + (uint32_t)(half64 * 64), r, m);
        if (half64 == NLD - 1) {
          // everything of this accumulator is in registers: release it
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(b_acce + 8 * (h * NB + buf));
        }
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const int64_t pg = p0 + half64 * 64 + g * 16;
          if (pg + 16 <= seg_end && pg + 16 <= a.N) {
            // the 16 rows lie inside the current bin: one compare
            if (m[g] > bv) {
              int pos = 0;
#pragma unroll
              for (int k = 15; k >= 0; --k) pos = (r[g][k] == m[g]) ? k : pos;
              bv = m[g];
              brow = pg + pos;
            }
          } else {
            // a bin boundary or the end of the rows falls in this run
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const int64_t p = pg + k;
              if (p < a.N) {
                while (p >= seg_end) {
                  flush_run();
                  ++cur;
                  seg_end = run_bin_end(cur, a.bq, a.br);
                  bv = __uint_as_float(kNegInfBits);
                  brow = -1;
                }
                if (r[g][k] > bv) {
                  bv = r[g][k];
                  brow = p;
                }
              }
            }
          }
        }
      }
    }
    }
    tc_fence_before();
    asm volatile("bar.arrive 1, %0;" ::"n"(32 + 512) : "memory");
    flush_run();
    return;
  }
  int64_t bg = 0, tg = 0;
  float best[BPW];
  int32_t bt[BPW];
#pragma unroll
  for (int g = 0; g < BPW; ++g) {
    best[g] = __uint_as_float(kNegInfBits);
    bt[g] = -1;
  }
  auto flush = [&](int64_t bgx) {
#pragma unroll
    for (int g = 0; g < BPW; ++g) {
      const int64_t b = bgx * BS + cq * BPW + g;
      if (q_ok && bt[g] >= 0 && b < a.L)
        atomicMax(&gq[b],
                  (unsigned long long)make_key(scaled(best[g]), (int32_t)(bt[g] * a.L + b)));
      best[g] = __uint_as_float(kNegInfBits);
      bt[g] = -1;
    }
  };
  auto record = [&](float (&r)[4][16], float (&m)[4], int g0, int32_t t0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int g = g0 + q;
      if (m[q] > best[g]) {
        int pos = 0;
#pragma unroll
        for (int k = 15; k >= 0; --k) pos = (r[q][k] == m[q]) ? k : pos;
        best[g] = m[q];
        bt[g] = t0 + pos;
      }
    }
  };
  bool erun = true;
  for (int sg = 0; sg < nseg && erun; ++sg) {
  if (sg > 0) flush(bg);  // the previous segment's last group of bins
  set_query(sg);
  bg = s_begin / a.ntg;
  tg = s_begin % a.ntg;
  for (int li = 0; li < ns; ++li) {
    const int i = sg * ns + li;
    const int buf = NB == 2 ? (i & 1) : 0;
    if (!warp_all(mbar_wait_sleep(b_accf + 8 * (h * NB + buf), (uint32_t)((i / NB) & 1),
                                  abort_flag))) {
      erun = false;
      break;
    }
    tc_fence_after();
    const uint32_t tb = acc_cols(buf);
    const int32_t t0 = (int32_t)(tg * kRowsBin);
    const int64_t bw = bg * BS + cq * BPW;  // first bin of this warpgroup
    if (t0 + kRowsBin <= a.T && bw + BPW <= a.L) {
      // every column valid (warp-uniform): one compare per 16 scores. The
      // accumulator is released as soon as the last run is in registers.
      float r[4][16], m[4];
#pragma unroll
      for (int ld = 0; ld < NLD; ++ld) {
        __syncwarp();
        tmem_ld4x16_max_s(tb + (uint32_t)(ld * 64), r, m);
        if (ld == NLD - 1) {
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(b_acce + 8 * (h * NB + buf));
        }
        record(r, m, 4 * ld, t0);
      }
    } else {
      // past the last full grid row or the last bin: column by column
#pragma unroll
      for (int g = 0; g < BPW; ++g) {
        float r[16];
        __syncwarp();
        tmem_ld16s(tb + (uint32_t)(g * 16), r);
        if (bw + g < a.L) {
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            if (t0 + k < a.T && r[k] > best[g]) {
              best[g] = r[k];
              bt[g] = t0 + k;
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(b_acce + 8 * (h * NB + buf));
    }
    if (++tg == a.ntg) {
      flush(bg);
      tg = 0;
      ++bg;
    }
  }
  }
  tc_fence_before();
  asm volatile("bar.arrive 1, %0;" ::"n"(32 + 512) : "memory");
  flush(bg);
}

// Rows of the ragged last grid row: j = T*L + b for b < r = N - T*L. A CTA
// stages 4 of these rows in shared memory and each of its 128 threads scores
// one query against all 4 (FP32 sum of the BF16 products, minus the half
// norm for L2), merging into G by the same 64-bit atomicMax. (One template
// for both element types, with byte pointers, measured 7 us slower per
// search inside the launch chain than this BF16 kernel; E4M3 has its own.)
constexpr int kTailRows = 4, kTailQ = 128;
__global__ void __launch_bounds__(kTailQ)
k1_tcs_tail(const __nv_bfloat16* __restrict__ X, const __nv_bfloat16* __restrict__ Q,
            const float* __restrict__ hnorm, int64_t N, int64_t M, int64_t L, int64_t T,
            int pitch, int metric, unsigned long long* G) {
  extern __shared__ uint4 tail_smem[];  // kTailRows rows of `pitch` elements
  __nv_bfloat16* rows = reinterpret_cast<__nv_bfloat16*>(tail_smem);
  // Launched behind the contraction, which has already waited for the
  // queries and the zeroed keys: this kernel's atomics merge with the
  // contraction's in any order. It finishes only after the contraction has
  // (the pdl_wait at the end), so the kernel after it sees both.
  pdl_trigger();
  const int64_t r = N - T * L;
  const int64_t b0 = (int64_t)blockIdx.x * kTailRows;
  const int nr = (int)min((int64_t)kTailRows, r - b0);
  const int chunks = pitch / 8;  // 16-byte pieces of a row
  for (int c = threadIdx.x; c < kTailRows * chunks; c += kTailQ) {
    const int k = c / chunks, part = c % chunks;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (k < nr) v = reinterpret_cast<const uint4*>(X + (T * L + b0 + k) * pitch)[part];
    reinterpret_cast<uint4*>(rows + k * pitch)[part] = v;
  }
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.y * kTailQ + threadIdx.x;
  if (i < M) {
  float acc[kTailRows];
#pragma unroll
  for (int k = 0; k < kTailRows; ++k) acc[k] = 0.0f;
  const uint4* qrow = reinterpret_cast<const uint4*>(Q + i * pitch);
  // eight 16-byte pieces of the query row in flight at a time
  for (int p0 = 0; p0 < chunks; p0 += 8) {
    uint4 qv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) qv[u] = p0 + u < chunks ? qrow[p0 + u] : make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (p0 + u >= chunks) break;
      const __nv_bfloat16* qe = reinterpret_cast<const __nv_bfloat16*>(&qv[u]);
      float qf[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) qf[e] = __bfloat162float(qe[e]);
#pragma unroll
      for (int k = 0; k < kTailRows; ++k) {
        const uint4 xv = reinterpret_cast<const uint4*>(rows + k * pitch)[p0 + u];
        const __nv_bfloat16* xe = reinterpret_cast<const __nv_bfloat16*>(&xv);
#pragma unroll
        for (int e = 0; e < 8; ++e) acc[k] = fmaf(qf[e], __bfloat162float(xe[e]), acc[k]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kTailRows; ++k) {
    if (k < nr) {
      const int64_t j = T * L + b0 + k;
      const float sc = metric == KNN_L2 ? acc[k] - hnorm[j] : acc[k];
      atomicMax(&G[i * L + b0 + k], (unsigned long long)make_key(sc, (int32_t)j));
    }
  }
  }
  pdl_wait();
}

// The same for E4M3 codes (16 per 16-byte piece), the FP32 sum times the
// database scale as in the main kernel (IP and COS only).
__global__ void __launch_bounds__(kTailQ)
k1_tcs_tail_e4m3(const uint8_t* __restrict__ X, const uint8_t* __restrict__ Q,
                 const float* __restrict__ xscale, int64_t N, int64_t M, int64_t L, int64_t T,
                 int pitch, unsigned long long* G) {
  extern __shared__ uint4 tail_smem[];  // kTailRows rows of `pitch` bytes
  uint8_t* rows = reinterpret_cast<uint8_t*>(tail_smem);
  pdl_trigger();
  const int64_t r = N - T * L;
  const int64_t b0 = (int64_t)blockIdx.x * kTailRows;
  const int nr = (int)min((int64_t)kTailRows, r - b0);
  const int chunks = pitch / 16;  // 16-byte pieces of a row
  for (int c = threadIdx.x; c < kTailRows * chunks; c += kTailQ) {
    const int k = c / chunks, part = c % chunks;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (k < nr) v = reinterpret_cast<const uint4*>(X + (T * L + b0 + k) * pitch)[part];
    reinterpret_cast<uint4*>(rows + k * pitch)[part] = v;
  }
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.y * kTailQ + threadIdx.x;
  if (i < M) {
  float acc[kTailRows];
#pragma unroll
  for (int k = 0; k < kTailRows; ++k) acc[k] = 0.0f;
  const uint4* qrow = reinterpret_cast<const uint4*>(Q + i * pitch);
  for (int p0 = 0; p0 < chunks; p0 += 4) {
    uint4 qv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) qv[u] = p0 + u < chunks ? qrow[p0 + u] : make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (p0 + u >= chunks) break;
      const uint8_t* qc = reinterpret_cast<const uint8_t*>(&qv[u]);
      float qf[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) qf[e] = e4m3_code_to_float(qc[e]);
#pragma unroll
      for (int k = 0; k < kTailRows; ++k) {
        const uint4 xv = reinterpret_cast<const uint4*>(rows + k * pitch)[p0 + u];
        const uint8_t* xc = reinterpret_cast<const uint8_t*>(&xv);
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[k] = fmaf(qf[e], e4m3_code_to_float(xc[e]), acc[k]);
      }
    }
  }
  const float xs0 = xscale[0];
#pragma unroll
  for (int k = 0; k < kTailRows; ++k) {
    if (k < nr) {
      const int64_t j = T * L + b0 + k;
      atomicMax(&G[i * L + b0 + k], (unsigned long long)make_key(__fmul_rn(acc[k], xs0), (int32_t)j));
    }
  }
  }
  pdl_wait();
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode_s() {
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

CUtensorMapDataType map_type(int esz) {
  return esz == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
}

// 2-D map of BF16 (esz 2) or E4M3 codes (esz 1): inner extent `inner`
// elements, `rows` rows `stride_el` elements apart, box of 128 bytes x
// box_rows, 128-byte swizzle.
bool make_map_s(CUtensorMap* m, const void* base, int64_t inner, int64_t rows, int64_t stride_el,
                int box_rows, int esz) {
  auto enc = get_encode_s();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)stride_el * esz};
  cuuint32_t box[2] = {(cuuint32_t)(kSpanS / esz), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(m, map_type(esz), 2, const_cast<void*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 3-D view of the database for the step boxes: element d of grid row t,
// bin b is row t*L + b. Dimensions (d, t, b) with the bin outermost, so a
// box of (128 bytes, 16, bs) lands as [bin][grid row][128 B]: each bin's 16
// rows are consecutive accumulator columns.
bool make_map_grid(CUtensorMap* m, const void* base, int64_t pitch, int64_t L, int64_t T, int bs,
                   int esz) {
  auto enc = get_encode_s();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)T, (cuuint64_t)L};
  cuuint64_t strides[2] = {(cuuint64_t)(L * pitch * esz), (cuuint64_t)(pitch * esz)};
  cuuint32_t box[3] = {(cuuint32_t)(kSpanS / esz), (cuuint32_t)kRowsBin, (cuuint32_t)bs};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(m, map_type(esz), 3, const_cast<void*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// One CTA per SM at most: the database steps split into `parts` ranges and
// the query tiles into groups of kq; CTA (group, part) runs the tiles of its
// group one after the other over its range. Picks the kq (and the parts it
// allows) with the least work per CTA, counting a query-tile reload as one
// step; ties go to the smaller kq (fewer reloads, fewer database passes).
void tcs_schedule(int64_t nqt, int64_t steps, int64_t sms, int64_t* kq_out, int64_t* parts_out,
                  int64_t* spp_out, int64_t* groups_out) {
  if (sms < 1) sms = 1;
  const int64_t kq_min = cdiv(nqt, sms);
  int64_t best = -1;
  for (int64_t kq = kq_min; kq <= min(nqt, kq_min + 16); ++kq) {
    const int64_t groups = cdiv(nqt, kq);
    if (groups > sms) continue;
    int64_t parts = min(sms / groups, steps);
    const int64_t spp = cdiv(steps, parts);
    parts = cdiv(steps, spp);
    const int64_t work = kq * (spp + 1);
    if (best < 0 || work < best) {
      best = work;
      *kq_out = kq;
      *parts_out = parts;
      *spp_out = spp;
      *groups_out = groups;
    }
  }
}

struct TcsShape {
  int mode, nkb, nksteps, stages, bs;
  uint32_t a_bytes, stage_bytes;
  size_t smem;
};

// Bins per step of the fused mode (rows up to 128 elements): 16 (N = 256,
// 32 KB stages) or 8 (N = 128, double-buffered accumulators, 16 KB stages).
// Measured on the 1M x 128 workloads: 16 bins 0.195 ms (L2) / 0.185 ms (IP),
// 8 bins 0.320 / 0.302 ms -- the N = 128 MMAs read 1.5x the shared-memory
// operand bytes per FLOP (A and B 4 KB each per 0.5 MFLOP) and are limited by
// shared-memory bandwidth, which outweighs the deeper ring.
constexpr int kFusedBins = 16;

template <int BS>
size_t tcs_fixed_smem(int ext) {
  return 1024 + (ext ? kExtAS + StepT<BS>::kXS * StepT<BS>::kExtB : 0) + 512;
}

// The first mode whose shared memory fits: kFused (resident query tile, the
// whole step's K blocks plus one of look-ahead), kKLoopA (resident query
// tile, at least 2 stages of one K block), kKLoopQ (query K block streamed in
// every stage). The K-loop modes use 16-bin steps.
bool tcs_shape(int D, int metric, int esz, TcsShape* sh) {
  const int pitch = (int)round_up(D, 16);
  const size_t budget = 227 * 1024;
  const int ext = metric == KNN_L2;
  // 128-byte K blocks and 32-byte MMA K-steps (16 BF16 or 32 E4M3 elements)
  sh->nkb = (int)cdiv((int64_t)pitch * esz, kSpanS);
  const int nks = (int)cdiv((int64_t)pitch * esz, 32);
  const uint32_t a_res = (uint32_t)(sh->nkb * kQT * kSpanS);
  // kFused: K-steps rounded up to an even count (the extra step multiplies
  // zero query columns: the query box reads zeros past the row)
  const int nks_even = (int)round_up(nks, 2);
  if (nks_even <= 8) {
    const size_t stage = (size_t)StepT<kFusedBins>::kStage;
    const size_t fixed = tcs_fixed_smem<kFusedBins>(ext) + a_res;
    const int need = sh->nkb + 1 > 3 ? sh->nkb + 1 : 3;
    if (fixed + (size_t)need * stage <= budget) {
      sh->mode = kFused;
      sh->bs = kFusedBins;
      sh->nksteps = nks_even;
      sh->a_bytes = a_res;
      sh->stage_bytes = (uint32_t)stage;
      sh->stages = (int)std::min<size_t>(16, (budget - fixed) / stage);
      sh->smem = fixed + (size_t)sh->stages * stage;
      return true;
    }
  }
  const size_t fixed0 = tcs_fixed_smem<16>(ext);
  const size_t stage16 = (size_t)StepT<16>::kStage;
  sh->bs = 16;
  sh->nksteps = nks;
  if (fixed0 + a_res + 2 * stage16 <= budget) {
    sh->mode = kKLoopA;
    sh->a_bytes = a_res;
    sh->stage_bytes = (uint32_t)stage16;
    sh->stages = (int)std::min<size_t>(8, (budget - fixed0 - a_res) / stage16);
  } else {
    sh->mode = kKLoopQ;
    sh->a_bytes = 0;
    sh->stage_bytes = (uint32_t)(kQT * kSpanS + stage16);
    sh->stages = (int)std::min<size_t>(4, (budget - fixed0) / sh->stage_bytes);
    if (sh->stages < 2) return false;
  }
  sh->smem = fixed0 + sh->a_bytes + (size_t)sh->stages * sh->stage_bytes;
  return true;
}

template <int NKS, int MODE, int BM, int BS, int DT>
cudaError_t launch_tcs(const CUtensorMap& mx, const CUtensorMap& mq, const TcsArgs& a, size_t smem,
                       int64_t blocks, cudaStream_t st) {
  // setmaxnreg.inc waits until the registers it asks for are free: refuse to
  // launch unless the launch-time allocation covers the split.
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k1_tcs_kernel<NKS, MODE, BM, BS, DT>);
  if (e != cudaSuccess) return e;
  if ((int64_t)round_up(fa.numRegs, 8) * kThreadsS < 128 * kCtrlRegsS + 512 * kEpiRegsS)
    return cudaErrorNotSupported;
  e = cudaFuncSetAttribute(k1_tcs_kernel<NKS, MODE, BM, BS, DT>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if constexpr (BM == kBinsRun) {
    // Contiguous bins: a plain launch. Started early behind the query prep,
    // the CTAs land on SMs in the order those free up, and the sharers of a
    // part end up far apart (measured: 0.244 -> 0.284 ms per search).
    k1_tcs_kernel<NKS, MODE, BM, BS, DT><<<(unsigned)blocks, kThreadsS, smem, st>>>(mx, mq, a);
    return cudaGetLastError();
  } else {
    return launch_pdl(k1_tcs_kernel<NKS, MODE, BM, BS, DT>, dim3((unsigned)blocks), dim3(kThreadsS),
                      smem, st, mx, mq, a);
  }
}

}  // namespace

// KNN_BF16 with any metric; KNN_E4M3_T (one database-wide scale) with IP
// and COS (the L2 half norm enters the BF16 contraction as an extra K block,
// which the E4M3 MMAs do not take).
bool k1_tcs_supported(int dtype, int D, int metric, int64_t N, int64_t L) {
  TcsShape sh;
  if (metric < KNN_IP || metric > KNN_COS) return false;
  if (dtype != KNN_BF16 && !(dtype == KNN_E4M3_T && metric != KNN_L2)) return false;
  const int esz = dtype == KNN_BF16 ? 2 : 1;
  if (!tcs_shape(D, metric, esz, &sh)) return false;
  if (L < 1 || L > N || N >= ((int64_t)1 << 31)) return false;
  // the grid view's row stride (L rows) must stay below 2^40 bytes
  return L * round_up(D, 16) * esz < ((int64_t)1 << 40);
}

template <int BM, int DT>
cudaError_t launch_tcs_mode(const TcsShape& sh, const CUtensorMap& mx, const CUtensorMap& mq,
                            const TcsArgs& a, int64_t blocks, cudaStream_t st) {
  if (sh.mode == kKLoopA) return launch_tcs<4, kKLoopA, BM, 16, DT>(mx, mq, a, sh.smem, blocks, st);
  if (sh.mode == kKLoopQ) return launch_tcs<4, kKLoopQ, BM, 16, DT>(mx, mq, a, sh.smem, blocks, st);
  constexpr int FB = kFusedBins;
  switch (sh.nksteps) {
    case 2: return launch_tcs<2, kFused, BM, FB, DT>(mx, mq, a, sh.smem, blocks, st);
    case 4: return launch_tcs<4, kFused, BM, FB, DT>(mx, mq, a, sh.smem, blocks, st);
    case 6: return launch_tcs<6, kFused, BM, FB, DT>(mx, mq, a, sh.smem, blocks, st);
    case 8: return launch_tcs<8, kFused, BM, FB, DT>(mx, mq, a, sh.smem, blocks, st);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t launch_k1_tcs(int64_t N, int64_t M, int64_t L, int D, int metric, int dtype,
                          int bin_map, const void* X, const float* xscale, const float* hnorm,
                          const void* Qp, unsigned long long* G, cudaStream_t st) {
  TcsShape sh;
  const bool e4 = dtype == KNN_E4M3_T;
  const int esz = e4 ? 1 : 2;
  if (!k1_tcs_supported(dtype, D, metric, N, L) || !tcs_shape(D, metric, esz, &sh))
    return cudaErrorNotSupported;
  if (metric == KNN_L2 && !hnorm) return cudaErrorInvalidValue;
  if (e4 && !xscale) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (reinterpret_cast<uintptr_t>(Qp) & 15))
    return cudaErrorInvalidValue;
  if (M <= 0) return cudaSuccess;
  const bool runs = bin_map == KNN_BINS_CONTIGUOUS;
  const int pitch = (int)round_up(D, 16);
  TcsArgs a{};
  a.N = N;
  a.M = M;
  a.L = L;
  a.T = N / L;
  a.ntg = cdiv(a.T, kRowsBin);
  const int cols = sh.bs * kRowsBin;  // MMA N: database rows per step
  a.nbg = cdiv(L, sh.bs);
  a.bq = N / L;
  a.br = N % L;
  a.nqt = cdiv(M, kQT);
  // a step: bs bins x 16 grid rows (j mod L), or 16 bs consecutive rows
  a.steps_per_q = runs ? cdiv(N, cols) : a.ntg * a.nbg;
  const int64_t sms = device_sm_count();
  tcs_schedule(a.nqt, a.steps_per_q, sms, &a.kq, &a.parts, &a.steps_per_part, &a.groups);
  // step counters of a CTA are 32-bit
  if (a.kq * a.steps_per_part * sh.nkb >= ((int64_t)1 << 31)) return cudaErrorNotSupported;
  a.pitch = pitch;
  a.nkb = sh.nkb;
  a.nksteps = sh.nksteps;
  a.stages = sh.stages;
  a.a_bytes = sh.a_bytes;
  a.stage_bytes = sh.stage_bytes;
  a.ext = metric == KNN_L2 ? 1 : 0;
  // D = F32, A = B = BF16 (kind::f16) or E4M3 (kind::f8f6f4, format 0), both
  // K-major, N = cols, M = 128
  a.idesc = (1u << 4) | (e4 ? 0u : (1u << 7) | (1u << 10)) | ((uint32_t)(cols >> 3) << 17) |
            ((uint32_t)(kQH >> 4) << 24);
  a.hnorm = hnorm;
  a.xscale = xscale;
  a.G = G;
  CUtensorMap mx, mq;
  const bool mapped = runs ? make_map_s(&mx, X, pitch, N, pitch, cols, esz)
                           : make_map_grid(&mx, X, pitch, L, a.T, sh.bs, esz);
  if (!mapped) return cudaErrorInvalidValue;
  if (!make_map_s(&mq, Qp, pitch, M, pitch, kQT, esz)) return cudaErrorInvalidValue;
  const int64_t blocks = a.groups * a.parts;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  cudaError_t e;
  if (e4)
    e = runs ? launch_tcs_mode<kBinsRun, KNN_E4M3>(sh, mx, mq, a, blocks, st)
             : launch_tcs_mode<kBinsMod, KNN_E4M3>(sh, mx, mq, a, blocks, st);
  else
    e = runs ? launch_tcs_mode<kBinsRun, KNN_BF16>(sh, mx, mq, a, blocks, st)
             : launch_tcs_mode<kBinsMod, KNN_BF16>(sh, mx, mq, a, blocks, st);
  if (e != cudaSuccess) return e;
  const int64_t r = N - a.T * L;
  if (!runs && r > 0) {
    dim3 grid((unsigned)cdiv(r, kTailRows), (unsigned)cdiv(M, kTailQ));
    const size_t tsmem = (size_t)kTailRows * pitch * esz;  // <= 32 KB (pitch <= 4096)
    if (e4)
      e = launch_pdl(k1_tcs_tail_e4m3, grid, dim3(kTailQ), tsmem, st,
                     reinterpret_cast<const uint8_t*>(X), reinterpret_cast<const uint8_t*>(Qp),
                     xscale, N, M, L, a.T, pitch, G);
    else
      e = launch_pdl(k1_tcs_tail, grid, dim3(kTailQ), tsmem, st,
                     reinterpret_cast<const __nv_bfloat16*>(X),
                     reinterpret_cast<const __nv_bfloat16*>(Qp), hnorm, N, M, L, a.T, pitch,
                     metric, G);
  }
  return e;
}

bool k1_tcs_take_timeout() { return tc_take_timeout_local(); }
bool k1_tcs_set_wait_limit(unsigned long long ns) { return tc_set_wait_limit_local(ns); }

}  // namespace tpuknn
