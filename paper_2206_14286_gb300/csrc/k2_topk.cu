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
  __device__ __forceinline__ uint64_t key(int64_t i, int64_t b) const {
    uint64_t best = 0;
    for (int64_t s = 0; s < nsplits; ++s) {
      const int64_t base = (s * M + i) * Lk + b;
      for (int f = 0; f < g; ++f) {
        const int32_t j = a[base + (int64_t)f * L];
        if (j < 0) continue;
        const uint64_t k = make_key(v[base + (int64_t)f * L], (int32_t)(j + index_offset));
        best = k > best ? k : best;
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
    if (cnt + (int)blockDim.x > CH) flush();
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
}  // namespace

cudaError_t launch_merge_bins(const K1Plan& p, Partials parts, float* out_v, int32_t* out_a,
                              cudaStream_t st) {
  const int64_t n = p.M * p.L;
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)cdiv(n, 256);
  if (parts.a) {
    PairSource s{parts.v, parts.a, p.M, p.Lk, p.L, p.nsplits, parts.index_offset, p.g};
    merge_bins_kernel<<<blocks, 256, 0, st>>>(s, p.M, p.L, out_v, out_a);
  } else {
    PackedSource s{reinterpret_cast<const uint32_t*>(parts.v), p.M, p.Lk, p.L, p.nsplits,
                   p.tiles_per_split, parts.index_offset, p.g, p.code_bits};
    merge_bins_kernel<<<blocks, 256, 0, st>>>(s, p.M, p.L, out_v, out_a);
  }
  return cudaGetLastError();
}

cudaError_t launch_k2(const K1Plan& p, Partials parts, int Kp, const uint64_t* run_in,
                      uint64_t* out_keys, cudaStream_t st) {
  if (parts.a) {
    PairSource s{parts.v, parts.a, p.M, p.Lk, p.L, p.nsplits, parts.index_offset, p.g};
    return run_k2(s, p.M, p.L, Kp, run_in, out_keys, st);
  }
  PackedSource s{reinterpret_cast<const uint32_t*>(parts.v), p.M, p.Lk, p.L, p.nsplits,
                 p.tiles_per_split, parts.index_offset, p.g, p.code_bits};
  return run_k2(s, p.M, p.L, Kp, run_in, out_keys, st);
}

}  // namespace tpuknn
