/*
 * tpuknn.h -- C ABI of the GB300 (sm_103a) K-nearest-neighbour search library.
 *
 * The library implements the search of arXiv 2206.14286 ("TPU-KNN"):
 *   1. a distance contraction between the queries Q (M x D) and the database
 *      X (N x D) fused with PartialReduce (Alg. 1): for every query and every
 *      bin l in [0, L) keep the best score and its index over the rows
 *      j with j mod L == l, so the M x N score matrix never reaches memory;
 *   2. ExactRescoring (Sec. 5): an exact top-K' over the L bin winners;
 *   3. a re-rank of the K' candidates with FP32 scores, returning the top K.
 * The problem statement is Sec. 2 (Eq. 1 K-argmin of a distance, Eq. 2 MIPS).
 *
 * Conventions for every entry point
 *   - All array arguments are DEVICE pointers unless stated otherwise; the
 *     caller owns every buffer. Matrices are row-major.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Work is enqueued asynchronously; nothing synchronises unless
 *     stated. A non-OK return means nothing was enqueued, except
 *     KNN_ECUDA (a launch failed; see knn_last_cuda_error).
 *   - A search's kernels are chained by programmatic dependent launch: each
 *     waits on the device for the kernel before it. Its last kernel lets a
 *     following kernel that the caller launches WITH programmatic stream
 *     serialization start early. Such a kernel must call
 *     cudaGridDependencySynchronize() before it reads the outputs. Plain
 *     launches, copies and events are ordered as usual.
 *   - Device-side waits are bounded. A kernel that gives up sets a sticky
 *     device flag; knn_sync_status() synchronises the device and returns
 *     KNN_ETIMEOUT once, then clears it.
 *   - Scores are "larger is better" internally: IP <q,x>; L2 the relaxed
 *     <q,x> - ||x||^2/2 (App. A.2, Eq. 19, negated); COS <q,x> of rows
 *     scaled to unit length (Sec. 2). Equal scores rank the smaller index
 *     first. Returned values: IP <q,x>, L2 ||q-x||^2, COS cosine similarity,
 *     each computed in FP32 (best first: IP/COS descending, L2 ascending).
 *   - Inputs must be finite. Indices are int32 (N < 2^31).
 *   - No C++ exception crosses this boundary.
 */
#ifndef TPUKNN_H_
#define TPUKNN_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KNN_OK = 0,
  KNN_EINVAL = 1,        /* an argument is out of range, NULL or misaligned */
  KNN_ENOMEM = 2,        /* the caller's workspace is smaller than required */
  KNN_ECUDA = 3,         /* a CUDA call or launch failed */
  KNN_ETIMEOUT = 4,      /* a device-side wait ran out (see knn_sync_status) */
  KNN_EUNSUPPORTED = 5   /* valid request this build does not handle */
} knn_status;

typedef enum { KNN_IP = 0, KNN_L2 = 1, KNN_COS = 2 } knn_metric;

/* Element type the contraction runs in. The database and the queries are
 * stored in it; products accumulate in FP32. E4M3 uses one FP32 scale per
 * row: value = code * scale. KNN_E4M3_T stores the database the same way
 * (codes and a per-row scale array) with ONE scale for every row, the
 * database-wide max|x| / 448; queries of a KNN_E4M3_T search keep their own
 * per-row scales. E4M3 being a floating-point code, the shared scale costs
 * precision only where a value falls below 2^-6 of the scale (subnormal
 * codes); it lets the contraction compare raw dot products of different rows
 * directly (the KNN_BF16 kernel's one compare per 16 rows, with IP and COS). */
typedef enum { KNN_F32 = 0, KNN_BF16 = 1, KNN_E4M3 = 2, KNN_E4M3_T = 3 } knn_dtype;

/* Map from database row j to its bin l (Alg. 1, Sec. 5):
 *   KNN_BINS_MOD        l = j mod L;
 *   KNN_BINS_CONTIGUOUS runs of consecutive rows (Alg. 1's l = ShiftRight(j, W)),
 *                       balanced for any L: with q = N / L and r = N mod L, bin l
 *                       holds rows [l*q + min(l, r), (l+1)*q + min(l+1, r)).
 * Both give every bin N/L rows (up to one), so the recall law of Sec. 5.1 is the
 * same for exchangeable rows. KNN_BINS_CONTIGUOUS is implemented for KNN_BF16, and
 * for KNN_E4M3_T with KNN_IP and KNN_COS. */
typedef enum { KNN_BINS_MOD = 0, KNN_BINS_CONTIGUOUS = 1 } knn_bin_map;

const char* knn_status_string(int status);
/* The last CUDA error code seen by the library on this thread (0 = none). */
int knn_last_cuda_error(void);

/* Bytes per element of `dtype` (4, 2, 1), or 0 for an unknown dtype. */
int32_t knn_dtype_bytes(int32_t dtype);

/* Row pitch, in elements, of a prepared database or query buffer: D rounded
 * up to a multiple of 16 (so every row starts on a 16-byte boundary for the
 * tensor-memory copies). Returns -1 if D < 1. */
int32_t knn_row_pitch(int32_t D);

/*
 * Number of bins L for a recall target (Sec. 5.1, Eq. 13-14): the smallest
 * L >= 1 with ((L-1)/L)^(K-1) >= recall_target, rounded up to a multiple of
 * `round_to` (if round_to > 1), then clamped to N. K = 1 gives 1.
 * Returns L, or -1 if N < 1, K < 1, K > N or recall_target is not in (0, 1).
 * Host-only; needs no GPU.
 */
int64_t knn_plan_bins(int64_t N, int32_t K, double recall_target, int32_t round_to);

/*
 * Preparation of rows for the contraction (the database once, or queries).
 *   x        : rows x D FP32 input rows (device).
 *   out_lp   : rows x knn_row_pitch(D) elements of `dtype` (device). Columns
 *              D..pitch-1 are written as zero. For KNN_F32 the rows are
 *              copied (and normalised for KNN_COS).
 *   out_scale: rows FP32 scales, required for KNN_E4M3 (scale = max|x|/448,
 *              code = E4M3(x/scale), round-to-nearest-even, saturating; a
 *              zero row gets scale 1) and KNN_E4M3_T (every row gets the
 *              scale of all `rows` together: max over them of |x| / 448, 1
 *              if all are zero), else ignored (may be NULL).
 *   out_hnorm: rows FP32 values ||x^||^2/2 of the stored (rounded) rows,
 *              required for KNN_L2 (the half-norm of App. A.2, Eq. 19), else
 *              ignored (may be NULL).
 *   out_f32  : rows x D FP32 unit-length rows, required for KNN_COS (the
 *              FP32 source of the re-rank; normalisation sums squares in
 *              FP64 in index order), else ignored (may be NULL).
 * For KNN_COS every row is first scaled to unit length (Sec. 2: cosine
 * search is MIPS on normalised rows) and the stored form is made from that.
 * Errors: KNN_EINVAL for rows < 0, D < 1, a required pointer NULL, or a
 * pointer not 16-byte aligned.
 */
knn_status knn_prepare(const float* x, int64_t rows, int32_t D, int32_t metric, int32_t dtype,
                       void* out_lp, float* out_scale, float* out_hnorm, float* out_f32,
                       void* stream);

/*
 * Approximate K-NN search: PartialReduce (Alg. 1) + ExactRescoring (Sec. 5)
 * + FP32 re-rank.
 *   db_lp, db_scale, db_hnorm : the prepared database (knn_prepare), N rows.
 *   db_f32    : N x D FP32 rows used to score the final candidates (for COS
 *               the unit-length rows from knn_prepare). NULL = score the
 *               candidates from db_lp (dequantised).
 *   q         : M x D FP32 queries (device); prepared inside the call.
 *   K         : neighbours per query, 1 <= K <= min(L, 4096).
 *   L         : number of bins, 1 <= L <= N; if L <= 0,
 *               L = knn_plan_bins(N, K, recall_target, 1).
 *   bin_map   : knn_bin_map (which rows share a bin).
 *   rerank_mult: K' = max(1, rerank_mult) * K candidates (capped at L) leave
 *               ExactRescoring and are scored in FP32; the best K are kept.
 *   out_val   : M x K FP32 values (reported form), best first.
 *   out_idx   : M x K int32 database indices.
 *   workspace : device scratch of at least knn_search_workspace(...) bytes,
 *               256-byte aligned. Its contents on entry do not matter.
 * M = 0 is a valid no-op. Errors: KNN_EINVAL (sizes, NULL, alignment),
 * KNN_ENOMEM (workspace too small), KNN_EUNSUPPORTED (D > 4096; with E4M3
 * D > 256, except KNN_E4M3_T with KNN_IP or KNN_COS).
 */
knn_status knn_search(const void* db_lp, const float* db_scale, const float* db_hnorm,
                      const float* db_f32, int64_t N, int32_t D, int32_t dtype, int32_t metric,
                      const float* q, int64_t M, int32_t K, int64_t L, int32_t bin_map,
                      double recall_target, int32_t rerank_mult, float* out_val,
                      int32_t* out_idx, void* workspace, size_t ws_bytes, void* stream);

size_t knn_search_workspace(int64_t N, int32_t D, int32_t dtype, int32_t metric, int64_t M,
                            int32_t K, int64_t L, int32_t bin_map, double recall_target,
                            int32_t rerank_mult);

/*
 * The same search with HOST queries and HOST outputs: copies q (M x D FP32)
 * to the device, searches, copies the results back and synchronises
 * `stream` before returning. The database and the workspace stay on the
 * device; the workspace must also hold the staged queries and results
 * (knn_search_host_workspace bytes). Pinned host memory makes the copies
 * asynchronous DMA; pageable memory works but is slower.
 */
knn_status knn_search_host(const void* db_lp, const float* db_scale, const float* db_hnorm,
                           const float* db_f32, int64_t N, int32_t D, int32_t dtype,
                           int32_t metric, const float* q_host, int64_t M, int32_t K, int64_t L,
                           int32_t bin_map, double recall_target, int32_t rerank_mult,
                           float* out_val_host, int32_t* out_idx_host, void* workspace,
                           size_t ws_bytes, void* stream);

size_t knn_search_host_workspace(int64_t N, int32_t D, int32_t dtype, int32_t metric, int64_t M,
                                 int32_t K, int64_t L, int32_t bin_map, double recall_target,
                                 int32_t rerank_mult);

/*
 * knn_search_host without the final synchronisation: the copy of q, the
 * search and the copies of the results are enqueued on `stream` and the call
 * returns. The outputs hold the results, and q_host, the outputs and the
 * workspace may be reused, only once that work has completed (synchronise
 * the stream or an event recorded after the call). With pinned host buffers
 * the copies are asynchronous DMA, so searches in flight on two streams (each
 * with its own workspace and outputs) overlap one search's copies with the
 * other's kernels. Arguments, workspace size and errors as knn_search_host;
 * errors of the enqueued work are reported by knn_sync_status.
 */
knn_status knn_search_host_async(const void* db_lp, const float* db_scale,
                                 const float* db_hnorm, const float* db_f32, int64_t N,
                                 int32_t D, int32_t dtype, int32_t metric, const float* q_host,
                                 int64_t M, int32_t K, int64_t L, int32_t bin_map,
                                 double recall_target, int32_t rerank_mult, float* out_val_host,
                                 int32_t* out_idx_host, void* workspace, size_t ws_bytes,
                                 void* stream);

/*
 * knn_search without a caller workspace: the search runs in a scratch buffer
 * of KNN_STATIC_WORKSPACE_BYTES that the library reserves in device memory
 * when the module loads (a file-scope __device__ array, one per device). The
 * paper has no counterpart; this is a library convenience.
 *
 * Who needs it: callers that cannot allocate device memory at the moment
 * they search -- code running inside an allocator's own callbacks or
 * out-of-memory handler, a serving thread that must not take the caching
 * allocator's lock or grow its pool, or a plugin whose host framework hands
 * it no scratch. This call allocates nothing: no cudaMalloc, no cudaFree, no
 * allocating library routine.
 *
 * Arguments, results and errors are those of knn_search, minus workspace and
 * ws_bytes. In addition:
 *   - KNN_ENOMEM when knn_search_workspace(...) for the same arguments
 *     exceeds KNN_STATIC_WORKSPACE_BYTES (checked before any CUDA call);
 *     use knn_search with a workspace of your own for larger batches.
 *   - The first call in each CUDA context looks up the buffer's address
 *     (cudaGetSymbolAddress with the device current, which can load the
 *     module); later calls in the same context reuse it. The address is
 *     cached per device with the context's unique id, so after
 *     cudaDeviceReset (which replaces the device's primary context) the next
 *     call looks it up again. Make the first call in a context before any
 *     stream capture begins. A failed lookup returns KNN_ECUDA.
 *   - Nothing in the buffer has to start at zero: each call clears what it
 *     accumulates into (the merged bin winners) in its first kernel.
 *   - One buffer serves every call on a device. Calls that overlap in time
 *     (on different streams, or from several host threads without ordering)
 *     race on it and give wrong results; calls on one stream are ordered and
 *     safe.
 */
#define KNN_STATIC_WORKSPACE_BYTES (16u << 20)

knn_status knn_search_static(const void* db_lp, const float* db_scale, const float* db_hnorm,
                             const float* db_f32, int64_t N, int32_t D, int32_t dtype,
                             int32_t metric, const float* q, int64_t M, int32_t K, int64_t L,
                             int32_t bin_map, double recall_target, int32_t rerank_mult,
                             float* out_val, int32_t* out_idx, void* stream);

/*
 * N-sharded search (Sec. 7: the search runs on pods of chips that each hold
 * part of the database; App. A.1: reduction_input_size_override plans the
 * bins for the whole input when an operand holds one shard). A database of
 * N_global rows is split by rows; a shard holds the global rows
 * [row0, row0 + n_local), prepared as knn_prepare does. Bins are j mod L of
 * the GLOBAL row index j, L planned for N_global (knn_plan_bins); row0 must be
 * a multiple of L, so every shard's rows keep their global bins, and
 * L <= n_local. Only the j mod L bin map is supported.
 *
 * The shards exchange two arrays between three calls, each merged by an
 * element-wise maximum over the shards (e.g. an all-reduce MAX over int64):
 *   1. knn_shard_partial_reduce: PartialReduce (Alg. 1) of the shard's rows,
 *      keys[M x L] (int64, device): per query and bin the best (score, global
 *      row) as a signed-order key, or INT64_MIN for a bin with no row here.
 *      Workspace: knn_shard_partial_reduce_workspace bytes (0 = invalid).
 *   2. knn_shard_rescore: on the merged keys, ExactRescoring's top
 *      Kp = knn_rescore_count(K, rerank_mult, L) bin winners per query
 *      (every shard gets the same ones), and for those whose row this shard
 *      holds the FP32 score from x_f32 (n_local x D, the shard's FP32 rows;
 *      for COS its unit rows) against the FP32 queries q (M x D); the others
 *      stay INT64_MIN. Output cand_keys[M x Kp] (int64, device).
 *      Workspace: knn_shard_rescore_workspace bytes.
 *   3. knn_shard_finish: on the merged cand_keys, the best K per query, best
 *      first, in the reported form (as knn_search's outputs).
 *      Workspace: knn_shard_finish_workspace bytes.
 * A key orders (score, row) like the library's 64-bit keys (larger score
 * first, then the smaller row), XOR 2^63 so that signed int64 comparison
 * gives that order; a MAX reduction therefore keeps, per bin, the best row of
 * all shards (ties to the smaller global row), exactly PartialReduce over
 * the whole database. With one shard (row0 = 0, n_local = N_global) the three
 * calls are the search.
 * Errors: KNN_EINVAL (sizes, row0 not a multiple of L, L > n_local, NULL,
 * alignment), KNN_ENOMEM (workspace), KNN_EUNSUPPORTED, KNN_ECUDA.
 */
size_t knn_shard_partial_reduce_workspace(int64_t n_local, int64_t row0, int64_t N_global,
                                          int32_t D, int32_t dtype, int32_t metric, int64_t M,
                                          int64_t L);
knn_status knn_shard_partial_reduce(const void* db_lp, const float* db_scale,
                                    const float* db_hnorm, int64_t n_local, int64_t row0,
                                    int64_t N_global, int32_t D, int32_t dtype, int32_t metric,
                                    const float* q, int64_t M, int64_t L, int64_t* keys,
                                    void* workspace, size_t ws_bytes, void* stream);
/* Kp = min(max(1, rerank_mult) * K, L, 4096), at least K; -1 if K < 1, L < 1,
 * K > L or K > 4096. */
int32_t knn_rescore_count(int32_t K, int32_t rerank_mult, int64_t L);
size_t knn_shard_rescore_workspace(int64_t M, int64_t L, int32_t D, int32_t metric, int32_t K,
                                   int32_t rerank_mult);
knn_status knn_shard_rescore(const int64_t* keys, int64_t M, int64_t L, int32_t K,
                             int32_t rerank_mult, const float* q, int32_t D, int32_t metric,
                             const float* x_f32, int64_t n_local, int64_t row0,
                             int64_t* cand_keys, void* workspace, size_t ws_bytes,
                             void* stream);
size_t knn_shard_finish_workspace(int64_t M, int32_t Kp, int32_t K);
knn_status knn_shard_finish(const int64_t* cand_keys, int64_t M, int32_t Kp, int32_t K,
                            int32_t metric, float* out_val, int32_t* out_idx, void* workspace,
                            size_t ws_bytes, void* stream);

/*
 * A database held by the library (the problem statement's fixed set of N
 * reference vectors, Sec. 2, prepared once for the contraction as
 * knn_prepare does). knn_db_create allocates device memory with cudaMalloc on
 * the current device -- the rows in `dtype` (N x knn_row_pitch(D)), the FP32
 * half norms (L2), the per-row scales (E4M3), and the FP32 rows the re-rank
 * reads (always for COS, where they are the unit-length rows; for IP / L2 a
 * copy of x when keep_f32 != 0, else the re-rank dequantises the stored rows)
 * -- prepares them from x (N x D FP32, device) on `stream` and returns once
 * the preparation has finished; x may be freed afterwards. The handle owns
 * these buffers until knn_db_destroy frees them (cudaFree, which waits for
 * the device). Errors: KNN_EINVAL (sizes, NULL, alignment), KNN_ENOMEM
 * (cudaMalloc failed), KNN_EUNSUPPORTED (D > 4096), KNN_ECUDA; on any error
 * nothing stays allocated and *out is NULL.
 *
 * knn_db_search is knn_search on the handle's buffers (same arguments from q
 * on, same rules); knn_db_search_workspace gives its workspace size (0 for
 * invalid arguments). knn_db_info reports N, D, metric and dtype (any output
 * pointer may be NULL). A handle may serve several streams and threads at
 * once (searches only read it); destroying it while a search that uses it is
 * in flight is the caller's error.
 */
typedef struct knn_db knn_db;

knn_status knn_db_create(const float* x, int64_t N, int32_t D, int32_t metric, int32_t dtype,
                         int32_t keep_f32, void* stream, knn_db** out);
knn_status knn_db_destroy(knn_db* db);
knn_status knn_db_info(const knn_db* db, int64_t* N, int32_t* D, int32_t* metric,
                       int32_t* dtype);
knn_status knn_db_search(const knn_db* db, const float* q, int64_t M, int32_t K, int64_t L,
                         int32_t bin_map, double recall_target, int32_t rerank_mult,
                         float* out_val, int32_t* out_idx, void* workspace, size_t ws_bytes,
                         void* stream);
size_t knn_db_search_workspace(const knn_db* db, int64_t M, int32_t K, int64_t L, int32_t bin_map,
                               double recall_target, int32_t rerank_mult);

/*
 * PartialReduce alone (Alg. 1; the paper's aggregate_to_topk = False,
 * App. A.1): for every query i and bin l the best internal score and its
 * index, out_v[i*L + l], out_a[i*L + l]. Scores are in the internal
 * orientation (see the conventions above; L2 is the relaxed score).
 * With KNN_BF16 (either bin map) the values are the FP32 accumulator of the
 * contraction, the L2 half norm entering it as a three-part BF16 split
 * (error below 2^-24 of the norm). With KNN_E4M3 the kernel keeps only the
 * top 32 - c bits of each FP32 score, c <= 13, while it reduces (the low bits
 * hold the row's position in its bin), and the per-query scale is left out of
 * the value (it does not change the order within a query). With KNN_E4M3_T
 * and IP or COS the values are the FP32 accumulator of the codes' products
 * times the database scale (per-query scale left out, as for KNN_E4M3); with
 * L2 it runs as KNN_E4M3. With KNN_F32 the values are the FP32 scores.
 */
knn_status knn_partial_reduce(const void* db_lp, const float* db_scale, const float* db_hnorm,
                              int64_t N, int32_t D, int32_t dtype, int32_t metric, const float* q,
                              int64_t M, int64_t L, int32_t bin_map, float* out_v, int32_t* out_a,
                              void* workspace, size_t ws_bytes, void* stream);

size_t knn_partial_reduce_workspace(int64_t N, int32_t D, int32_t dtype, int32_t metric,
                                    int64_t M, int64_t L, int32_t bin_map);

/*
 * The approx_max_k / approx_min_k operator on a score matrix the caller
 * already has (App. A.1: PartialReduce of Alg. 1 and ExactRescoring without
 * the fused contraction).
 *   scores      : M x N row-major, score_dtype KNN_F32 or KNN_BF16 (device).
 *   K           : results per row with aggregate_to_topk; also the K of the
 *                 recall law when L <= 0.
 *   L           : bins (1 <= L <= N); if L <= 0, the smallest L whose Eq. 13
 *                 recall for K is at least recall_target, computed for
 *                 planning_size rows (the paper's reduction_input_size_override:
 *                 the full input size when the caller holds one shard; <= 0
 *                 means N), clamped to N.
 *   bin_map     : knn_bin_map over the columns.
 *   is_min      : 0 = largest scores (approx_max_k), 1 = smallest (approx_min_k).
 *   aggregate_to_topk : 0 -> out_val / out_idx are M x L, the winner of every
 *                 bin in bin order (-1 / NaN for an empty bin); 1 -> M x K,
 *                 the best K bin winners, best first.
 *   workspace   : knn_approx_max_k_workspace(...) bytes, 256-byte aligned.
 * Values are the scores as given (same sign); ties keep the smaller column.
 * Reads every score once: HBM-bound. Errors: KNN_EINVAL (sizes, K > L with
 * aggregation, NULL, alignment, N >= 2^31), KNN_ENOMEM (workspace).
 */
knn_status knn_approx_max_k(const void* scores, int32_t score_dtype, int64_t M, int64_t N,
                            int32_t K, int64_t L, int64_t planning_size, double recall_target,
                            int32_t bin_map, int32_t is_min, int32_t aggregate_to_topk,
                            float* out_val, int32_t* out_idx, void* workspace, size_t ws_bytes,
                            void* stream);

size_t knn_approx_max_k_workspace(int64_t M, int64_t N, int32_t K, int64_t L,
                                  int64_t planning_size, double recall_target,
                                  int32_t aggregate_to_topk);

/*
 * Exact K-NN (Eq. 1-2): the top K over all N rows, scored in `dtype` with
 * FP32 accumulation (the L = N case of PartialReduce), then values recomputed
 * in FP32 from db_f32 (or db_lp if NULL). Same arguments and rules as
 * knn_search without L, recall_target and rerank_mult.
 */
knn_status knn_search_exact(const void* db_lp, const float* db_scale, const float* db_hnorm,
                            const float* db_f32, int64_t N, int32_t D, int32_t dtype,
                            int32_t metric, const float* q, int64_t M, int32_t K,
                            float* out_val, int32_t* out_idx, void* workspace, size_t ws_bytes,
                            void* stream);

size_t knn_search_exact_workspace(int64_t N, int32_t D, int32_t dtype, int32_t metric, int64_t M,
                                  int32_t K);

/*
 * Backward of the selected values (the differentiation pattern): with the
 * indices idx (M x K, int32, -1 = skip) held constant, the gradient of
 *   sum_{i,k} grad_val[i,k] * value(q_i, x_idx[i,k])
 * where value is the reported form (IP <q,x>; L2 ||q-x||^2; COS the cosine
 * of the rows as given). Rows are read as FP32 from x_f32 (N x D) if not
 * NULL, else from the prepared db_lp/db_scale (dequantised); queries q are
 * FP32 (M x D).
 *   dq : M x D FP32, overwritten (NULL = not needed).
 *   dx : N x D FP32 (NULL = not needed). If zero_dx != 0 every row of dx
 *        is overwritten (zeros where no entry selected it), else the
 *        entries are added into dx.
 *   workspace: NULL, or knn_backward_workspace bytes (256-byte aligned; a
 *        smaller one is KNN_ENOMEM). Row path: each row of dx is written
 *        once by one warp, its entries summed in (i, k) order, bit-
 *        reproducible; taken with a workspace when zero_dx != 0 (the faster
 *        way: no separate zero fill) or deterministic != 0. Otherwise: zero
 *        fill (if zero_dx), then FP32 atomic adds (order-dependent rounding;
 *        the faster way to add into an existing dx).
 *   deterministic: 1 = the row path always; the workspace is required
 *        (KNN_EINVAL if NULL); 0 = the workspace is optional. Not read when
 *        dx is NULL or M = 0.
 */
knn_status knn_backward(const void* db_lp, const float* db_scale, const float* x_f32, int64_t N,
                        int32_t D, int32_t dtype, int32_t metric, const float* q, int64_t M,
                        int32_t K, const int32_t* idx, const float* grad_val, float* dq,
                        float* dx, int32_t zero_dx, int32_t deterministic, void* workspace,
                        size_t ws_bytes, void* stream);

/* Bytes of the workspace of knn_backward: about 4 N + 4 M K + 4 min(N, M K)
 * (each part rounded up to 256 bytes) + 256: a list head per row, a link per
 * entry, the list of touched rows and its count. The same for both values of
 * `deterministic`. */
size_t knn_backward_workspace(int64_t N, int32_t D, int64_t M, int32_t K, int32_t deterministic);

/*
 * Measurement aid (no counterpart in the paper): while enabled, every search
 * call records a pair of CUDA events on its stream around each of its kernel
 * classes: 0 = query preparation, 1 = PartialReduce (K1), 2 = ExactRescoring
 * (K2), 3 = re-rank (K3). knn_profile_enable(1) (re)starts the record and
 * creates the events; knn_profile_enable(0) stops recording. knn_profile_read
 * synchronises on the recorded events and returns the summed elapsed time in
 * milliseconds and the number of launches of one class (at most 16384 are
 * kept per class). Not thread-safe with concurrent searches.
 */
knn_status knn_profile_enable(int32_t on);
knn_status knn_profile_read(int32_t kernel_class, double* total_ms, int64_t* launches);

/*
 * Measurement aid (no counterpart in the paper's algorithm; it measures the
 * inputs of its roofline, Sec. 4 Eq. 6 and Eq. 8-9, on this GPU): runs a
 * kernel that issues only one kind of FP32 instruction, in 16 independent
 * chains per thread, over 2048 threads per SM for `iters` iterations, and
 * returns the operations per second (thread-level: one instruction of one
 * thread = one operation) and the kernel time in ms, timed with CUDA events
 * on `stream` after one untimed launch. Synchronous.
 *   KNN_RATE_MINMAX : min/max, the compare-and-select operation (COP) of
 *                     PartialReduce: the gamma of Eq. 6.
 *   KNN_RATE_FFMA   : fused multiply-add (2 FLOP each): the roof of the
 *                     FP32 CUDA-core contraction.
 * Errors: KNN_EINVAL (unknown kind, iters < 1, NULL output), KNN_ECUDA.
 */
typedef enum { KNN_RATE_MINMAX = 0, KNN_RATE_FFMA = 1 } knn_rate_kind;
knn_status knn_measure_rate(int32_t kind, int64_t iters, double* ops_per_s, double* ms,
                            void* stream);

/*
 * Test aid for the failure handling (no counterpart in the paper): sets the
 * limit, in nanoseconds, of the tensor-core kernels' pipeline waits on the
 * current device (0 restores the default, 2 s). A wait that runs out makes its
 * CTA stop issuing work, let the copies and MMAs it already issued finish
 * (those waits keep the fixed 2 s limit), free its tensor memory and return;
 * the search's results are then undefined and knn_sync_status reports
 * KNN_ETIMEOUT once. A limit under 1000 ns (below the device timer's
 * resolution) makes every wait give up at its first check, i.e. the first
 * wait that does not complete at once runs out: that is how a test exercises
 * this path without a fault. Synchronous (it writes device memory through the legacy
 * stream); do not call it while searches are in flight. Errors: KNN_ECUDA.
 */
knn_status knn_set_wait_limit_ns(uint64_t ns);

/* Synchronise the current device and report a device-side wait timeout
 * (KNN_ETIMEOUT, flag then cleared) or a CUDA error (KNN_ECUDA). */
knn_status knn_sync_status(void);

#ifdef __cplusplus
}
#endif

#endif /* TPUKNN_H_ */
