// kernels.h -- host-side launchers of the library's kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tpuknn {

// ----------------------------------------------------------------------------
// Work decomposition of PartialReduce (K1), shared by every K1 variant.
//
// Bins: row j belongs to bin j mod L. K1 runs with Lk = g*L bins (g >= 1 a
// fold factor so that a strip of BW tile rows is filled when L < BW); K2 then
// merges bins b, b+L, ..., b+(g-1)L, which together hold exactly the rows of
// bin b. Viewing the database as a [ntiles x Lk] grid (row j = t*Lk + b), a
// "strip" is BW consecutive bins and a "tile" is one strip of one grid row t:
// BW consecutive database rows whose bins are fixed per lane. Every CTA owns
// (strip, query tile, split) and walks tiles t in its split's range, keeping
// the running best of each (query, bin) it owns in registers.
// ----------------------------------------------------------------------------
struct K1Plan {
  int64_t N, M, L, Lk;
  int g;
  int D, pitch;
  int metric, dtype;
  int BW, BQ;               // tile rows (bins per strip), queries per tile
  int64_t nstrips, nqtiles, ntiles, tiles_per_split, nsplits;
  int code_bits;            // packed partials: bits of the tile ordinal
  bool atomic_merge;        // packed partials merged in K1 into one [M][Lk] array
};

// Partial results of K1:
//   pair form   : per (split, query, bin) a float value + int32 index (exact;
//                 FP32 path);
//   packed form : per (split, query, bin) one 32-bit float whose low
//                 code_bits bits encode the tile ordinal inside the split;
//   merged form : per (query, bin) the maximum over splits of the packed keys
//                 (code = global tile ordinal), stored order-mapped (see
//                 float_to_ordered) so that unsigned atomicMax merges them;
//                 0 marks a bin no row reached. The array must start at zero.
struct Partials {
  float* v;         // pair form values, or packed / merged keys
  int32_t* a;       // pair form indices (nullptr otherwise)
  int64_t index_offset;  // added to every decoded index (chunked exact search)
  bool merged;
  bool keys64;      // v holds [M][L] 64-bit (score, ~index) keys, 0 = empty
};

// Row preparation; optionally also zeroes zero_n 32-bit words of zero_buf.
cudaError_t launch_prep(const float* x, int64_t rows, int D, int pitch, int metric, int dtype,
                        void* out_lp, float* out_scale, float* out_hnorm, float* out_f32,
                        cudaStream_t st, uint32_t* zero_buf = nullptr, int64_t zero_n = 0);

cudaError_t launch_k1_simt(const K1Plan& p, const float* X, const float* hnorm, const float* Qp,
                           Partials out, cudaStream_t st);

// Tensor-core K1 (BF16 / E4M3). Returns cudaErrorNotSupported when the shape is
// outside what the kernel handles.
cudaError_t launch_k1_tc(const K1Plan& p, const void* X, const float* xscale, const float* hnorm,
                         const void* Qp, const float* qscale, Partials out, cudaStream_t st);

// Tensor-core K1 (BF16, rows up to 4096 elements; or E4M3 codes with one
// database-wide scale xscale[0], IP and COS), queries on TMEM lanes;
// with bin_map KNN_BINS_MOD each bin's rows sit side by side in the
// accumulator (the ragged last grid row is scored by a small extra kernel),
// with KNN_BINS_CONTIGUOUS a step is 256 consecutive rows. G[M][L] receives
// ordered 64-bit (score, ~index) keys by atomicMax and must be zero on entry.
bool k1_tcs_supported(int dtype, int D, int metric, int64_t N, int64_t L);
cudaError_t launch_k1_tcs(int64_t N, int64_t M, int64_t L, int D, int metric, int dtype,
                          int bin_map, const void* X, const float* xscale, const float* hnorm,
                          const void* Qp, unsigned long long* G, cudaStream_t st);
bool k1_tcs_take_timeout();
bool k1_tcs_set_wait_limit(unsigned long long ns);

// approx_max_k on a caller's score matrix (FP32 or BF16, M x N): the bin
// winners merged as ordered 64-bit keys into G[M][L] (zero on entry), scores
// negated first when neg != 0; and the keys turned back into (value, index).
cudaError_t launch_bin_max(const void* S, int dtype, int64_t M, int64_t N, int64_t L, int bin_map,
                           int neg, unsigned long long* G, cudaStream_t st);
cudaError_t launch_keys_to_pairs(const uint64_t* keys, int64_t n, int neg, float* out_v,
                                 int32_t* out_a, cudaStream_t st);

// K2: per query, merge the partials of every split and fold and select the
// best Kp (score, index) keys, sorted. If run_in is given its Kp keys per
// query join the selection (running top-K of a chunked search). With
// sorted = false the keys may come in any order (for the re-rank, which
// orders its candidates itself).
cudaError_t launch_k2(const K1Plan& p, Partials parts, int Kp, const uint64_t* run_in,
                      uint64_t* out_keys, cudaStream_t st, bool sorted = true);

// PartialReduce output alone: per (query, bin) the merged best value and
// index (index -1 and value -inf for a bin no row reached).
cudaError_t launch_merge_bins(const K1Plan& p, Partials parts, float* out_v, int32_t* out_a,
                              cudaStream_t st);

// K3: score the Kp candidates of each query in FP32 and keep the best K.
// Rows come from xf32 (N x D) when given, else from the stored rows.
// ExactRescoring and the FP32 re-rank fused (one CTA of 4 warps per query)
// for K1's merged [M][L] keys; the same results as launch_k2 followed by
// launch_k3. Supported when k23_supported(...) holds (L <= 1024, Kp <= 32,
// K <= 32, 16-byte aligned FP32 rows and queries with D % 4 == 0);
// otherwise returns cudaErrorNotSupported.
bool k23_supported(int64_t M, int64_t L, int Kp, int K, int D, const float* qf32,
                   int64_t q_stride, const float* xf32);
cudaError_t launch_k23(const uint64_t* G, int64_t M, int64_t L, int Kp, int K, int D, int metric,
                       const float* qf32, int64_t q_stride, const float* xf32, int64_t N,
                       float* out_val, int32_t* out_idx, cudaStream_t st);

cudaError_t launch_k3(int64_t M, int D, int metric, const uint64_t* cand, int Kp, int K,
                      const float* qf32, int64_t q_stride, const float* xf32, const void* xlp,
                      int dtype, int pitch, const float* xscale, int64_t N, float* out_val,
                      int32_t* out_idx, cudaStream_t st);

cudaError_t launch_backward(int64_t M, int D, int K, int metric, const float* q,
                            const float* xf32, const void* xlp, int dtype, int pitch,
                            const float* xscale, int64_t N, const int32_t* idx,
                            const float* g, float* dq, float* dx, int zero_dx, int deterministic,
                            void* ws, cudaStream_t st);
size_t backward_ws_bytes(int64_t N, int64_t M, int K);

// Largest resident query tile of the tensor-core K1 for this row length
// (256 or 128), or 0 if the rows are too long.
int k1_tc_query_tile(int dtype, int D);

// N-sharded search (shard.cu): PartialReduce pairs -> signed-order keys with
// global indices; signed keys -> keys; FP32 scores of the candidates a shard
// holds, as signed keys (empty for the others).
cudaError_t launch_pairs_to_signed_keys(const float* v, const int32_t* a, int64_t n, int64_t add,
                                        int64_t* out, cudaStream_t st);
cudaError_t launch_signed_to_keys(const int64_t* in, int64_t n, uint64_t* out, cudaStream_t st);
cudaError_t launch_score_owned(const uint64_t* cand, int64_t M, int Kp, const float* q,
                               int64_t q_stride, const float* x, int64_t n_local, int64_t row0,
                               int D, int metric, int64_t* out, cudaStream_t st);

// Issue-rate microbenchmark (knn_measure_rate): operations per second of one
// instruction kind over a grid that fills every SM.
cudaError_t measure_rate(int kind, int64_t iters, double* ops_per_s, double* ms,
                         cudaStream_t st);

// Number of SMs of the current device (cached).
int device_sm_count();
// Take and clear the tensor-core kernels' timeout flag (synchronous).
bool k1_tc_take_timeout();
// Set the limit of the tensor-core kernels' pipeline waits on the current
// device (ns = 0: the default 2 s).
bool k1_tc_set_wait_limit(unsigned long long ns);

}  // namespace tpuknn
