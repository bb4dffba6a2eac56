// k2_topk.cu -- ExactRescoring (Sec. 5): per query, merge the partial bin
// winners of every split (and fold) and select the best Kp (score, index)
// pairs, sorted best first.
//
// One CTA per query. Candidates stream through shared memory against a
// threshold (the current Kp-th best key): only keys above it are appended to
// a buffer, and when the buffer could overflow it is sorted together with
// the running best Kp (bitonic, descending) and truncated. With the L bin
// winners of one query this is a single bitonic sort of O(L log^2 L) work, the
// paper's ExactRescoring; the same code streams the N scores of a chunked
// exact search.
#include "common.cuh"
#include "kernels.h"

namespace tpuknn {

namespace {

// Candidate b (an output bin, 0 <= b < L) of query i: the best partial over
// every split s and fold f (K1 bins b + f*L).
struct PairSource {
  const float* v;
  const int32_t* a;
  int64_t M, Lk, L, nsplits, index_offset;
  int g;
  // The splits' entries are read four at a time, value and index together
  // (both arrays are written for every entry), so with few queries a warp
  // still has many loads in flight.
  __device__ __forceinline__ uint64_t key(int64_t i, int64_t b) const {
    uint64_t best = 0;
    for (int f = 0; f < g; ++f) {
      const int64_t b0 = i * Lk + b + (int64_t)f * L;
      for (int64_t s0 = 0; s0 < nsplits; s0 += 4) {
        int32_t jj[4];
        float vv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool in = s0 + u < nsplits;
          const int64_t e = b0 + (s0 + u) * M * Lk;
          jj[u] = in ? a[e] : -1;
          vv[u] = in ? v[e] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (jj[u] >= 0) {
            const uint64_t k = make_key(vv[u], (int32_t)(jj[u] + index_offset));
            best = k > best ? k : best;
          }
        }
      }
    }
    return best;
  }
};

// Packed partials: a float whose low `bits` bits hold (2^bits - 1 - t_local),
// t_local the tile ordinal inside the split; the bin's row is then
// j = (s * tiles_per_split + t_local) * Lk + bin.
struct PackedSource {
  const uint32_t* p;
  int64_t M, Lk, L, nsplits, tiles_per_split, index_offset;
  int g, bits;
  __device__ __forceinline__ uint64_t key(int64_t i, int64_t b) const {
    const uint32_t mask = bits ? ((1u << bits) - 1u) : 0u;
    uint64_t best = 0;
#pragma unroll 4
    for (int64_t s = 0; s < nsplits; ++s) {
      const int64_t base = (s * M + i) * Lk + b;
      for (int f = 0; f < g; ++f) {
        const uint32_t w = p[base + (int64_t)f * L];
        if (w == kNegInfBits) continue;  // no row reached this (split, bin)
        const int64_t tl = (int64_t)(mask - (w & mask));
        const int64_t bin = b + (int64_t)f * L;
        const int64_t j = (s * tiles_per_split + tl) * Lk + bin + index_offset;
        const uint64_t k = make_key(__uint_as_float(w & ~mask), (int32_t)j);
        best = k > best ? k : best;
      }
    }
    return best;
  }
};

// Merged partials: G[i][bin] = order-mapped packed key (0 = empty) whose
// low `bits` bits hold (2^bits - 1 - t), t the global tile ordinal; the row is
// j = t * Lk + bin.
struct MergedSource {
  const uint32_t* G;
  int64_t M, Lk, L, index_offset;
  int g, bits;
  __device__ __forceinline__ uint64_t key(int64_t i, int64_t b) const {
    const uint32_t mask = bits ? ((1u << bits) - 1u) : 0u;
    uint64_t best = 0;
    for (int f = 0; f < g; ++f) {
      const int64_t bin = b + (int64_t)f * L;
      const uint32_t u = G[i * Lk + bin];
      if (u == 0u) continue;
      const uint32_t w = __float_as_uint(ordered_to_float(u));
      const int64_t t = (int64_t)(mask - (w & mask));
      const int64_t j = t * Lk + bin + index_offset;
      const uint64_t k = make_key(__uint_as_float(w & ~mask), (int32_t)j);
      best = k > best ? k : best;
    }
    return best;
  }
};

// 64-bit keys already merged per (query, bin).
struct KeySource {
  const uint64_t* G;
  int64_t L;
  __device__ __forceinline__ uint64_t key(int64_t i, int64_t b) const { return G[i * L + b]; }
};

// Descending sort of KPL keys held in registers (bitonic network).
template <int KPL>
__device__ __forceinline__ void reg_sort_desc(uint64_t (&k)[KPL]) {
#pragma unroll
  for (int size = 2; size <= KPL; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
      for (int t = 0; t < KPL / 2; ++t) {
        const int lo = 2 * t - (t & (stride - 1));
        const int hi = lo + stride;
        const bool desc = (lo & size) == 0;
        const uint64_t x = k[lo], y = k[hi];
        const bool sw = desc ? (x < y) : (x > y);
        k[lo] = sw ? y : x;
        k[hi] = sw ? x : y;
      }
    }
  }
}

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int o) {
  const uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, o);
  const uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), o);
  return ((uint64_t)hi << 32) | lo;
}

// Lane `lane`'s candidates b = lane + 32 r (r < KPL) of query i, 0 past L.
template <class Src, int KPL>
__device__ __forceinline__ void lane_keys(const Src& src, int64_t i, int lane, int64_t L,
                                          uint64_t (&k)[KPL]) {
#pragma unroll
  for (int r = 0; r < KPL; ++r) {
    const int64_t b = lane + 32 * r;
    k[r] = b < L ? src.key(i, b) : 0;
  }
}
// The same from per-split (value, index) partials: the splits are the outer
// loop, so a lane has the loads of all its candidates of one split in flight
// at once (with few queries the per-candidate loop over the splits left each
// warp waiting on one load at a time).
template <int KPL>
__device__ __forceinline__ void lane_keys(const PairSource& src, int64_t i, int lane, int64_t L,
                                          uint64_t (&k)[KPL]) {
#pragma unroll
  for (int r = 0; r < KPL; ++r) k[r] = 0;
  for (int f = 0; f < src.g; ++f) {
    for (int64_t s = 0; s < src.nsplits; ++s) {
      const int64_t base = (s * src.M + i) * src.Lk + (int64_t)f * src.L + lane;
#pragma unroll
      for (int r0 = 0; r0 < KPL; r0 += 8) {
        int32_t jj[8];
        float vv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const bool in = r0 + u < KPL && lane + 32 * (r0 + u) < L;
          jj[u] = in ? src.a[base + 32 * (r0 + u)] : -1;
          vv[u] = in ? src.v[base + 32 * (r0 + u)] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (r0 + u < KPL && jj[u] >= 0) {
            const uint64_t key = make_key(vv[u], (int32_t)(jj[u] + src.index_offset));
            k[r0 + u] = key > k[r0 + u] ? key : k[r0 + u];
          }
        }
      }
    }
  }
}

// One warp per query: lane l holds candidates l, l+32, ... (KPL of them),
// sorted; Kp rounds each take the warp-wide maximum of the lane heads and pop
// it from its lane. Keys are unique (distinct indices), so one lane pops.
template <class Src, int KPL>
__global__ void __launch_bounds__(256)
k2_warp_kernel(Src src, int64_t M, int64_t L, int Kp, uint64_t* __restrict__ out_keys) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= M) return;
  uint64_t k[KPL];
  lane_keys(src, i, lane, L, k);
  reg_sort_desc<KPL>(k);
  for (int r = 0; r < Kp; ++r) {
    uint64_t m = k[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t y = shfl_xor_u64(m, o);
      m = y > m ? y : m;
    }
    if (lane == 0) out_keys[i * Kp + r] = m;
    if (m != 0 && k[0] == m) {
#pragma unroll
      for (int t = 0; t + 1 < KPL; ++t) k[t] = k[t + 1];
      k[KPL - 1] = 0;
    }
  }
}

template <class Src>
cudaError_t run_k2_warp(const Src& src, int64_t M, int64_t L, int Kp, uint64_t* out,
                        cudaStream_t st) {
  const int kpl = next_pow2((int)cdiv(L, 32));
  const unsigned blocks = (unsigned)cdiv(M * 32, 256);
  switch (kpl) {
    case 1: k2_warp_kernel<Src, 1><<<blocks, 256, 0, st>>>(src, M, L, Kp, out); break;
    case 2: k2_warp_kernel<Src, 2><<<blocks, 256, 0, st>>>(src, M, L, Kp, out); break;
    case 4: k2_warp_kernel<Src, 4><<<blocks, 256, 0, st>>>(src, M, L, Kp, out); break;
    case 8: k2_warp_kernel<Src, 8><<<blocks, 256, 0, st>>>(src, M, L, Kp, out); break;
    case 16: k2_warp_kernel<Src, 16><<<blocks, 256, 0, st>>>(src, M, L, Kp, out); break;
    default: k2_warp_kernel<Src, 32><<<blocks, 256, 0, st>>>(src, M, L, Kp, out); break;
  }
  return cudaGetLastError();
}

template <class Src>
__global__ void __launch_bounds__(256)
k2_topk_kernel(Src src, int64_t nelem, int Kp, int CH, int CAP, const uint64_t* __restrict__ run_in,
               uint64_t* __restrict__ out_keys) {
  extern __shared__ uint64_t sk[];
  __shared__ int cnt;
  __shared__ uint64_t thr;
  const int64_t i = blockIdx.x;
  for (int t = threadIdx.x; t < Kp; t += blockDim.x) sk[t] = run_in ? run_in[i * Kp + t] : 0;
  if (threadIdx.x == 0) {
    cnt = 0;
    thr = run_in ? run_in[i * Kp + Kp - 1] : 0;
  }
  __syncthreads();
  auto flush = [&]() {
    const int used = Kp + cnt;
    for (int t = used + threadIdx.x; t < CAP; t += blockDim.x) sk[t] = 0;
    bitonic_sort_desc(sk, CAP);
    if (threadIdx.x == 0) {
      thr = sk[Kp - 1];
      cnt = 0;
    }
    __syncthreads();
  };
  for (int64_t base = 0; base < nelem; base += blockDim.x) {
    // every thread reads the count before any thread appends again, so the
    // flush decision (which contains barriers) is the same in every thread
    const int c = cnt;
    __syncthreads();
    if (c + (int)blockDim.x > CH) flush();
    const int64_t e = base + threadIdx.x;
    if (e < nelem) {
      const uint64_t k = src.key(i, e);
      if (k > thr) {
        const int pos = atomicAdd(&cnt, 1);
        sk[Kp + pos] = k;
      }
    }
    __syncthreads();
  }
  if (cnt > 0 || run_in == nullptr) flush();
  for (int t = threadIdx.x; t < Kp; t += blockDim.x) out_keys[i * Kp + t] = sk[t];
}

template <class Src>
__global__ void merge_bins_kernel(Src src, int64_t M, int64_t L, float* __restrict__ out_v,
                                  int32_t* __restrict__ out_a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= M * L) return;
  const uint64_t k = src.key(t / L, t % L);
  out_v[t] = k ? key_score(k) : neg_inf();
  out_a[t] = k ? key_index(k) : -1;
}

template <class Src>
cudaError_t run_k2(const Src& src, int64_t M, int64_t nelem, int Kp, const uint64_t* run_in,
                   uint64_t* out, cudaStream_t st) {
  const int threads = 256;
  const int64_t ch64 = round_up(nelem, threads);
  int CH = (int)(ch64 < 4 * threads ? ch64 : 4 * threads);
  if (CH < threads) CH = threads;
  const int CAP = next_pow2(Kp + CH);
  const size_t smem = (size_t)CAP * sizeof(uint64_t);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  auto kern = k2_topk_kernel<Src>;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (M <= 0) return cudaSuccess;
  kern<<<(unsigned)M, threads, smem, st>>>(src, nelem, Kp, CH, CAP, run_in, out);
  return cudaGetLastError();
}

// ExactRescoring and the FP32 re-rank in one CTA of 4 warps per query, for
// the merged 64-bit keys of K1 (L <= 1024, Kp <= 32, K <= 32, 16-byte
// aligned FP32 rows with D % 4 == 0). Warp 0 takes the best Kp of the L keys:
// each lane sorts its KPL keys, then every round the warp's maximum key
// comes from two 32-bit max-reductions (high word, then the low word among
// the lanes that hold the high maximum) and the lane that holds it shifts
// its list. The 4 warps then score the Kp candidates against the FP32 rows
// (a lane reads 4 consecutive elements; a warp has up to 8 rows in flight),
// and warp 0 sorts the Kp exact keys across its lanes and writes the best K.
// Same results as the two-kernel path: the candidates are the Kp largest
// keys, and the re-rank scores and orders them the same way.
template <int METRIC, int KPL>
__global__ void __launch_bounds__(128)
k23_kernel(const uint64_t* __restrict__ G, int64_t L, int Kp, int K, int D,
           const float* __restrict__ qf32, int64_t q_stride, const float* __restrict__ xf32,
           int64_t N, float* __restrict__ out_val, int32_t* __restrict__ out_idx) {
  constexpr int kWarps = 4, kPerWarp = 8;  // 4 x 8 = 32 candidates at most
  __shared__ uint64_t s_cand[32];
  __shared__ uint64_t s_key[32];
  const int64_t i = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  pdl_wait();  // the keys come from the contraction (and the ragged-row kernel)
  pdl_trigger();  // the next call's query prep may launch (it waits for this kernel)
  if (warp == 0) {
    uint64_t k[KPL];
#pragma unroll
    for (int r = 0; r < KPL; ++r) {
      const int64_t b = lane + 32 * r;
      k[r] = b < L ? G[i * L + b] : 0;
    }
    reg_sort_desc<KPL>(k);
    uint64_t mine = 0;
    for (int r = 0; r < Kp; ++r) {
      const uint32_t hi = (uint32_t)(k[0] >> 32);
      const uint32_t mh = __reduce_max_sync(0xffffffffu, hi);
      const uint32_t ml = __reduce_max_sync(0xffffffffu, hi == mh ? (uint32_t)k[0] : 0u);
      const uint64_t m = ((uint64_t)mh << 32) | ml;
      if (lane == r) mine = m;
      // keys are unique (distinct rows), so one lane pops
      if (m != 0 && k[0] == m) {
#pragma unroll
        for (int t = 0; t + 1 < KPL; ++t) k[t] = k[t + 1];
        k[KPL - 1] = 0;
      }
    }
    s_cand[lane] = mine;
  }
  __syncthreads();
  const float* q = qf32 + i * q_stride;
  {
    int32_t js[kPerWarp];
    float acc[kPerWarp];
#pragma unroll
    for (int u = 0; u < kPerWarp; ++u) {
      const int c = warp + kWarps * u;
      const uint64_t key = c < Kp ? s_cand[c] : 0;
      const int32_t j = key ? key_index(key) : -1;
      js[u] = (j >= 0 && j < N) ? j : -1;
      acc[u] = 0.0f;
    }
    for (int d0 = 0; d0 < D; d0 += 128) {
      const int d = d0 + lane * 4;
      const bool in = d < D;
      const float4 qv = in ? *reinterpret_cast<const float4*>(q + d) : make_float4(0, 0, 0, 0);
      float4 xv[kPerWarp];
#pragma unroll
      for (int u = 0; u < kPerWarp; ++u)
        xv[u] = (in && js[u] >= 0)
                    ? __ldg(reinterpret_cast<const float4*>(xf32 + (int64_t)js[u] * D + d))
                    : make_float4(0, 0, 0, 0);
#pragma unroll
      for (int u = 0; u < kPerWarp; ++u) {
        if (METRIC == KNN_L2) {
          // elements past D contribute 0: both sides are zero there
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
    for (int u = 0; u < kPerWarp; ++u) {
      float v = acc[u];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      const int c = warp + kWarps * u;
      if (lane == 0 && c < 32)
        s_key[c] = js[u] >= 0 ? make_key(METRIC == KNN_L2 ? -v : v, js[u]) : 0;
    }
  }
  __syncthreads();
  if (warp != 0) return;
  uint64_t mine = s_key[lane];
#pragma unroll
  for (int k2 = 2; k2 <= 32; k2 <<= 1) {
#pragma unroll
    for (int jj = k2 >> 1; jj > 0; jj >>= 1) {
      const uint64_t other = shfl_xor_u64(mine, jj);
      const bool up = (lane & k2) == 0, lower = (lane & jj) == 0;
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

template <int METRIC>
cudaError_t run_k23(const uint64_t* G, int64_t M, int64_t L, int Kp, int K, int D,
                    const float* qf32, int64_t q_stride, const float* xf32, int64_t N,
                    float* out_val, int32_t* out_idx, cudaStream_t st) {
  const int kpl = next_pow2((int)cdiv(L, 32));
  const unsigned blocks = (unsigned)M;
#define K23_CASE(P)                                                                          \
  case P:                                                                                    \
    return launch_pdl(k23_kernel<METRIC, P>, dim3(blocks), dim3(128), 0, st, G, L, Kp, K, D, \
                      qf32, q_stride, xf32, N, out_val, out_idx);
  switch (kpl) {
    K23_CASE(1)
    K23_CASE(2)
    K23_CASE(4)
    K23_CASE(8)
    K23_CASE(16)
    K23_CASE(32)
    default: return cudaErrorNotSupported;
  }
#undef K23_CASE
}


// Up to 2048 candidates and 256 selected per query (no running input): a CTA
// of 8 warps per query. Warp w sorts candidates [256 w, 256 w + 256) held in
// registers, element e = 32 r + lane in register r, by a bitonic network
// (partners within a lane swap registers, partners across lanes exchange by
// shuffle). Three merge rounds then halve the sorted lists: the top 256 of two
// descending lists A and B are max(A[e], B[255 - e]), a bitonic sequence that
// eight more bitonic steps sort. The result is the best Kp keys in order, as
// from the CTA kernel, at O(L log^2 256) compare-exchanges instead of full
// sorts of the whole buffer.
__device__ __forceinline__ void wsort_step(uint64_t (&k)[8], int lane, int size, int stride,
                                           bool all_desc) {
  if (stride >= 32) {
    const int rs = stride >> 5;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      if ((r & rs) == 0) {
        const int e = r * 32 + lane;
        const bool desc = all_desc || (e & size) == 0;
        const uint64_t a = k[r], b = k[r | rs];
        const bool sw = desc ? (a < b) : (a > b);
        k[r] = sw ? b : a;
        k[r | rs] = sw ? a : b;
      }
    }
  } else {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int e = r * 32 + lane;
      const bool desc = all_desc || (e & size) == 0;
      const uint64_t o = shfl_xor_u64(k[r], stride);
      const bool lower = (lane & stride) == 0;
      const bool keep_max = (lower == desc);
      k[r] = keep_max ? (o > k[r] ? o : k[r]) : (o < k[r] ? o : k[r]);
    }
  }
}

template <class Src>
__global__ void __launch_bounds__(256)
k2_wsort_kernel(Src src, int64_t L, int Kp, uint64_t* __restrict__ out_keys) {
  __shared__ uint64_t lists[8][256];
  const int64_t i = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t k[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t b = (int64_t)warp * 256 + r * 32 + lane;
    k[r] = b < L ? src.key(i, b) : 0;
  }
#pragma unroll
  for (int size = 2; size <= 256; size <<= 1)
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) wsort_step(k, lane, size, stride, false);
#pragma unroll
  for (int r = 0; r < 8; ++r) lists[warp][r * 32 + lane] = k[r];
  for (int level = 1; level < 8; level <<= 1) {
    __syncthreads();
    if ((warp & (2 * level - 1)) == 0) {
      const uint64_t* B = lists[warp + level];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int e = r * 32 + lane;
        const uint64_t a = lists[warp][e], b = B[255 - e];
        k[r] = a > b ? a : b;
      }
#pragma unroll
      for (int stride = 128; stride > 0; stride >>= 1) wsort_step(k, lane, 256, stride, true);
      __syncwarp();
#pragma unroll
      for (int r = 0; r < 8; ++r) lists[warp][r * 32 + lane] = k[r];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < Kp; t += blockDim.x) out_keys[i * Kp + t] = lists[0][t];
}

template <class Src>
cudaError_t run_k2_wsort(const Src& src, int64_t M, int64_t L, int Kp, uint64_t* out,
                         cudaStream_t st) {
  k2_wsort_kernel<Src><<<(unsigned)M, 256, 0, st>>>(src, L, Kp, out);
  return cudaGetLastError();
}

// The best Kp of a query's L keys as a set, in no particular order (for the
// re-rank, which orders its candidates itself): one CTA of 256 threads per
// query holds the L keys in registers (KPT per thread, L <= 256 KPT) and
// finds the Kp-th largest key T by a radix select over the 64 key bits, 8 per
// pass from the most significant: per pass a 256-bin histogram in shared
// memory of the keys that match the digits chosen so far, and warp 0 picks
// the digit where the count from the top reaches Kp. It stops once every key
// matching the chosen digits is needed. Output: the keys above the chosen
// digits, then as many matching keys as still needed (all of them but for
// repeated empty keys, 0). Keys are distinct otherwise, so this is the set
// of the Kp largest, the same set a sort would keep.
template <class Src, int KPT>
__global__ void __launch_bounds__(256)
k2_select_kernel(Src src, int64_t L, int Kp, uint64_t* __restrict__ out_keys) {
  __shared__ uint32_t hist[256];
  __shared__ int s_digit, s_above, s_stop, s_hi, s_eq;
  const int64_t i = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31;
  uint64_t k[KPT];
#pragma unroll
  for (int u = 0; u < KPT; ++u) {
    const int64_t b = (int64_t)u * 256 + tid;
    k[u] = b < L ? src.key(i, b) : 0;
  }
  uint64_t prefix = 0, mask = 0;
  int need = Kp;  // keys still to take among those matching the prefix
  for (int shift = 56; shift >= 0; shift -= 8) {
    hist[tid] = 0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < KPT; ++u)
      if ((int64_t)u * 256 + tid < L && (k[u] & mask) == prefix)
        atomicAdd(&hist[(uint32_t)(k[u] >> shift) & 255u], 1u);
    __syncthreads();
    if (tid < 32) {
      // lane l sums bins 255-8l .. 248-8l; counts from the top by a warp scan
      uint32_t c[8], sum = 0;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        c[t] = hist[255 - 8 * lane - t];
        sum += c[t];
      }
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      const uint32_t excl = incl - sum;  // keys matching the prefix in higher bins
      const bool mine = excl < (uint32_t)need && (uint32_t)need <= incl;
      const unsigned who = __ballot_sync(0xffffffffu, mine);
      if (who == 0) {
        // fewer matching keys than needed cannot happen for need <= L
        if (lane == 0) {
          s_digit = 0;
          s_above = 0;
          s_stop = 1;
        }
      } else if (mine) {
        uint32_t above = excl, ct = 0;
        int tf = 7;
        bool found = false;
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          if (!found) {
            if (above + c[t] >= (uint32_t)need) {
              tf = t;
              ct = c[t];
              found = true;
            } else {
              above += c[t];
            }
          }
        }
        s_digit = 255 - 8 * lane - tf;
        s_above = (int)above;
        s_stop = (above + ct == (uint32_t)need) ? 1 : 0;
      }
    }
    __syncthreads();
    prefix |= (uint64_t)s_digit << shift;
    mask |= (uint64_t)0xFF << shift;
    need -= s_above;
    const bool stop = s_stop != 0;
    __syncthreads();  // s_* are rewritten by the next pass
    if (stop) break;
  }
  // the keys above the prefix (masked), then `need` of those matching it
  if (tid == 0) {
    s_hi = 0;
    s_eq = 0;
  }
  __syncthreads();
  uint64_t* out = out_keys + i * Kp;
  const int n_hi = Kp - need;
#pragma unroll
  for (int u = 0; u < KPT; ++u) {
    if ((int64_t)u * 256 + tid >= L) continue;
    const uint64_t m = k[u] & mask;
    if (m > prefix) {
      out[atomicAdd(&s_hi, 1)] = k[u];
    } else if (m == prefix) {
      const int p = atomicAdd(&s_eq, 1);
      if (p < need) out[n_hi + p] = k[u];
    }
  }
}

template <class Src>
cudaError_t run_k2_select(const Src& src, int64_t M, int64_t L, int Kp, uint64_t* out,
                          cudaStream_t st) {
  if (L <= 2048)
    k2_select_kernel<Src, 8><<<(unsigned)M, 256, 0, st>>>(src, L, Kp, out);
  else if (L <= 4096)
    k2_select_kernel<Src, 16><<<(unsigned)M, 256, 0, st>>>(src, L, Kp, out);
  else
    k2_select_kernel<Src, 32><<<(unsigned)M, 256, 0, st>>>(src, L, Kp, out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_merge_bins(const K1Plan& p, Partials parts, float* out_v, int32_t* out_a,
                              cudaStream_t st) {
  const int64_t n = p.M * p.L;
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)cdiv(n, 256);
  if (parts.keys64) {
    KeySource s{reinterpret_cast<const uint64_t*>(parts.v), p.L};
    merge_bins_kernel<<<blocks, 256, 0, st>>>(s, p.M, p.L, out_v, out_a);
  } else if (parts.a) {
    PairSource s{parts.v, parts.a, p.M, p.Lk, p.L, p.nsplits, parts.index_offset, p.g};
    merge_bins_kernel<<<blocks, 256, 0, st>>>(s, p.M, p.L, out_v, out_a);
  } else if (parts.merged) {
    MergedSource s{reinterpret_cast<const uint32_t*>(parts.v), p.M, p.Lk, p.L,
                   parts.index_offset, p.g, p.code_bits};
    merge_bins_kernel<<<blocks, 256, 0, st>>>(s, p.M, p.L, out_v, out_a);
  } else {
    PackedSource s{reinterpret_cast<const uint32_t*>(parts.v), p.M, p.Lk, p.L, p.nsplits,
                   p.tiles_per_split, parts.index_offset, p.g, p.code_bits};
    merge_bins_kernel<<<blocks, 256, 0, st>>>(s, p.M, p.L, out_v, out_a);
  }
  return cudaGetLastError();
}

// Per query: the warp kernel serves up to 1024 candidates and 64 selected,
// the sorting CTA kernel up to 2048 candidates and 256 selected (both with
// no running input); beyond those, when an unordered set will do, the radix
// select up to 8192 candidates; the streaming CTA kernel everything else.
template <class Src>
cudaError_t dispatch_k2(const Src& s, const K1Plan& p, int Kp, const uint64_t* run_in,
                        uint64_t* out_keys, bool sorted, cudaStream_t st) {
  if (run_in == nullptr && p.L <= 1024 && Kp <= 64) return run_k2_warp(s, p.M, p.L, Kp, out_keys, st);
  if (run_in == nullptr && p.L <= 2048 && Kp <= 256 && p.M <= 0x7fffffffLL)
    return run_k2_wsort(s, p.M, p.L, Kp, out_keys, st);
  // a set is enough (the re-rank orders it): radix select instead of sorts
  if (!sorted && run_in == nullptr && p.L <= 8192 && p.M <= 0x7fffffffLL)
    return run_k2_select(s, p.M, p.L, Kp, out_keys, st);
  return run_k2(s, p.M, p.L, Kp, run_in, out_keys, st);
}

cudaError_t launch_k2(const K1Plan& p, Partials parts, int Kp, const uint64_t* run_in,
                      uint64_t* out_keys, cudaStream_t st, bool sorted) {
  if (p.M <= 0) return cudaSuccess;
  if (parts.keys64) {
    KeySource s{reinterpret_cast<const uint64_t*>(parts.v), p.L};
    return dispatch_k2(s, p, Kp, run_in, out_keys, sorted, st);
  }
  if (parts.a) {
    PairSource s{parts.v, parts.a, p.M, p.Lk, p.L, p.nsplits, parts.index_offset, p.g};
    return dispatch_k2(s, p, Kp, run_in, out_keys, sorted, st);
  }
  if (parts.merged) {
    MergedSource s{reinterpret_cast<const uint32_t*>(parts.v), p.M, p.Lk, p.L,
                   parts.index_offset, p.g, p.code_bits};
    return dispatch_k2(s, p, Kp, run_in, out_keys, sorted, st);
  }
  PackedSource s{reinterpret_cast<const uint32_t*>(parts.v), p.M, p.Lk, p.L, p.nsplits,
                 p.tiles_per_split, parts.index_offset, p.g, p.code_bits};
  return dispatch_k2(s, p, Kp, run_in, out_keys, sorted, st);
}

bool k23_supported(int64_t M, int64_t L, int Kp, int K, int D, const float* qf32,
                   int64_t q_stride, const float* xf32) {
  return M > 0 && M <= 0x7fffffffLL && L >= 1 && L <= 1024 && Kp >= 1 && Kp <= 32 &&
         K >= 1 && K <= 32 && xf32 && D % 4 == 0 && q_stride % 4 == 0 &&
         (reinterpret_cast<uintptr_t>(xf32) & 15) == 0 &&
         (reinterpret_cast<uintptr_t>(qf32) & 15) == 0;
}

cudaError_t launch_k23(const uint64_t* G, int64_t M, int64_t L, int Kp, int K, int D, int metric,
                       const float* qf32, int64_t q_stride, const float* xf32, int64_t N,
                       float* out_val, int32_t* out_idx, cudaStream_t st) {
  if (M <= 0) return cudaSuccess;
  if (!k23_supported(M, L, Kp, K, D, qf32, q_stride, xf32)) return cudaErrorNotSupported;
  return metric == KNN_L2 ? run_k23<KNN_L2>(G, M, L, Kp, K, D, qf32, q_stride, xf32, N, out_val,
                                            out_idx, st)
                          : run_k23<KNN_IP>(G, M, L, Kp, K, D, qf32, q_stride, xf32, N, out_val,
                                            out_idx, st);
}

}  // namespace tpuknn
