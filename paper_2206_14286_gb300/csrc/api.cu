// api.cu -- the extern "C" boundary: argument checks, the bin planner
// (Eq. 13-14), work decomposition, workspace layout and kernel launches.
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.h"

using namespace tpuknn;

namespace tpuknn {

thread_local int g_last_cuda = 0;

int device_sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 152;
  }
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
      cudaGetLastError();
      n = 152;
    }
    cache[dev] = n;
  }
  return cache[dev];
}

}  // namespace tpuknn

namespace {

// ---------------------------------------------------------------------------
// Event pairs around kernel classes (knn_profile_*).
// ---------------------------------------------------------------------------
constexpr int kProfClasses = 4, kProfCap = 16384;
struct Profiler {
  bool on = false;
  cudaEvent_t* ev[kProfClasses] = {nullptr, nullptr, nullptr, nullptr};  // 2 * kProfCap each
  int64_t n[kProfClasses] = {0, 0, 0, 0};
} g_prof;

struct ProfScope {
  int cls;
  cudaStream_t st;
  int64_t slot;
  ProfScope(int c, cudaStream_t s) : cls(c), st(s), slot(-1) {
    if (g_prof.on && g_prof.ev[c] && g_prof.n[c] < kProfCap) {
      slot = g_prof.n[c]++;
      cudaEventRecord(g_prof.ev[c][2 * slot], st);
    }
  }
  ~ProfScope() {
    if (slot >= 0) cudaEventRecord(g_prof.ev[cls][2 * slot + 1], st);
  }
};

constexpr size_t kAlign = 256;
inline size_t al(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }
inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
inline bool valid_metric(int m) { return m == KNN_IP || m == KNN_L2 || m == KNN_COS; }
inline bool valid_dtype(int d) {
  return d == KNN_F32 || d == KNN_BF16 || d == KNN_E4M3 || d == KNN_E4M3_T;
}

knn_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return KNN_OK;
  g_last_cuda = (int)e;
  return KNN_ECUDA;
}

// Eq. 13 at L: ((L-1)/L)^(K-1).
double paper_recall(int64_t L, int K) {
  if (K <= 1) return 1.0;
  return std::pow((double)(L - 1) / (double)L, (double)(K - 1));
}

int64_t plan_bins(int64_t N, int K, double r, int round_to) {
  if (N < 1 || K < 1 || K > N || !(r > 0.0 && r < 1.0)) return -1;
  int64_t L = 1;
  if (K > 1) {
    // Eq. 14: L >= 1 / (1 - r^(1/(K-1))); then the smallest L meeting Eq. 13.
    double est = 1.0 / (1.0 - std::pow(r, 1.0 / (double)(K - 1)));
    if (!(est < 9.0e18)) return -1;
    L = (int64_t)std::ceil(est);
    if (L < 1) L = 1;
    while (L > 1 && paper_recall(L - 1, K) >= r) --L;
    while (paper_recall(L, K) < r) ++L;
  }
  if (round_to > 1) L = round_up(L, round_to);
  if (L > N) L = N;
  return L;
}

// Tile shape of each K1 variant (BQ = 0: the row length is not supported).
void k1_tile(int dtype, int D, int64_t M, int* BW, int* BQ) {
  dtype = stored_dtype(dtype);
  if (dtype == KNN_F32) {
    *BW = 64;
    *BQ = 128;
  } else {
    *BW = 128;
    const int maxq = k1_tc_query_tile(dtype, D);
    *BQ = (maxq == 256 && M <= 128) ? 128 : maxq;
  }
}

int bits_for(int64_t n) {  // bits to hold values 0..n-1
  int b = 0;
  while (((int64_t)1 << b) < n) ++b;
  return b;
}

constexpr int kMaxCodeBits = 13;

K1Plan make_plan(int64_t N, int64_t M, int64_t L, int D, int metric, int dtype,
                 int64_t force_splits) {
  K1Plan p{};
  p.N = N;
  p.M = M;
  p.L = L;
  p.D = D;
  p.pitch = (int)round_up(D, 16);
  p.metric = metric;
  p.dtype = stored_dtype(dtype);  // KNN_E4M3_T runs here as KNN_E4M3 (all scales equal)
  k1_tile(dtype, D, M, &p.BW, &p.BQ);
  if (p.BQ == 0) return p;
  p.g = L < p.BW ? (int)(p.BW / L) : 1;
  p.Lk = (int64_t)p.g * L;
  p.nstrips = cdiv(p.Lk, p.BW);
  p.nqtiles = cdiv(M, p.BQ);
  p.ntiles = cdiv(N, p.Lk);
  const int64_t units = p.nstrips * (p.nqtiles > 0 ? p.nqtiles : 1);
  int64_t splits;
  if (force_splits > 0) {
    splits = force_splits;
  } else {
    const int64_t sms = device_sm_count();
    splits = cdiv(sms, units);
    if (dtype == KNN_F32 && sms > 0) {
      // SIMT CTAs run two per SM: the split count with the least
      // (waves of 2 * sms CTAs) x (tiles per CTA), the smallest on ties,
      // which also keeps the per-split partials no larger than needed
      const int64_t wave = 2 * sms;
      int64_t best = -1;
      for (int64_t s = 1; s <= std::min<int64_t>(p.ntiles, 4 * wave); ++s) {
        const int64_t cost = cdiv(units * s, wave) * cdiv(p.ntiles, s);
        if (best < 0 || cost < best) {
          best = cost;
          splits = s;
        }
      }
    }
    if (dtype != KNN_F32 && sms > 0) {
      // tensor-core CTAs run one per SM: among a few split counts, take the
      // one whose last wave is fullest (units * splits CTAs over `sms`)
      double best = 0.0;
      int64_t pick = splits;
      for (int64_t s = splits; s < splits + 8 && s <= cdiv(N, p.Lk); ++s) {
        const int64_t blocks = units * s;
        const double fill = (double)blocks / (double)(cdiv(blocks, sms) * sms);
        if (fill > best + 1e-9) {
          best = fill;
          pick = s;
        }
      }
      splits = pick;
    }
  }
  if (splits < 1) splits = 1;
  if (splits > p.ntiles) splits = p.ntiles;
  if (dtype != KNN_F32) {
    const int64_t min_splits = cdiv(p.ntiles, (int64_t)1 << kMaxCodeBits);
    if (splits < min_splits) splits = min_splits;
  }
  p.tiles_per_split = cdiv(p.ntiles, splits);
  p.nsplits = cdiv(p.ntiles, p.tiles_per_split);
  // Tensor-core partials merge in K1 (one [M][Lk] array, code = global tile
  // ordinal) when the global ordinal fits the code; otherwise per split.
  p.atomic_merge = dtype != KNN_F32 && force_splits <= 0 && bits_for(p.ntiles) <= kMaxCodeBits;
  p.code_bits = dtype == KNN_F32 ? 0 : bits_for(p.atomic_merge ? p.ntiles : p.tiles_per_split);
  return p;
}

// Per-call query preparation buffers.
struct QueryBufs {
  size_t lp, scale, f32;
};
QueryBufs query_bytes(int64_t M, int D, int dtype, int metric) {
  QueryBufs b{};
  const int pitch = (int)round_up(D, 16);
  const int esz = dtype == KNN_F32 ? 4 : (dtype == KNN_BF16 ? 2 : 1);
  b.lp = al((size_t)M * pitch * esz);
  b.scale = stored_dtype(dtype) == KNN_E4M3 ? al((size_t)M * 4) : 0;
  b.f32 = (metric == KNN_COS && dtype != KNN_F32) ? al((size_t)M * D * 4) : 0;
  return b;
}

struct SearchArgs {
  const void* db_lp;
  const float* db_scale;
  const float* db_hnorm;
  const float* db_f32;
  int64_t N;
  int D, dtype, metric;
  const float* q;
  int64_t M;
  int K;
  int64_t L;
  double recall;
  int rerank;
  int bin_map;
};

// Checks that do not need the data pointers.
knn_status check_sizes(int64_t N, int D, int dtype, int metric, int64_t M, int K) {
  if (N < 1 || D < 1 || M < 0 || K < 1 || K > N) return KNN_EINVAL;
  if (!valid_dtype(dtype) || !valid_metric(metric)) return KNN_EINVAL;
  if (N >= ((int64_t)1 << 31) - 1) return KNN_EINVAL;
  if (D > kMaxD || K > kMaxK) return KNN_EUNSUPPORTED;
  return KNN_OK;
}

knn_status resolve_L(const SearchArgs& a, int64_t* L) {
  int64_t l = a.L;
  if (l <= 0) l = plan_bins(a.N, a.K, a.recall, 1);
  if (l < 1 || l > a.N || a.K > l) return KNN_EINVAL;
  *L = l;
  return KNN_OK;
}

int kprime(int K, int rerank, int64_t L) {
  int64_t kp = (int64_t)(rerank < 1 ? 1 : rerank) * K;
  if (kp > L) kp = L;
  if (kp > kMaxK) kp = kMaxK;
  if (kp < K) kp = K;
  return (int)kp;
}

struct SearchLayout {
  K1Plan plan;
  int Kp;
  QueryBufs qb;
  bool keys64;      // K1 merges 64-bit (score, ~index) keys into one [M][L] array
  bool contiguous;  // bins are runs of consecutive rows
  size_t off_qlp, off_qscale, off_qf32, off_part_v, off_part_a, off_cand, total;
};

knn_status layout_search(const SearchArgs& a, SearchLayout* s) {
  knn_status st = check_sizes(a.N, a.D, a.dtype, a.metric, a.M, a.K);
  if (st != KNN_OK) return st;
  if (a.bin_map != KNN_BINS_MOD && a.bin_map != KNN_BINS_CONTIGUOUS) return KNN_EINVAL;
  int64_t L;
  if ((st = resolve_L(a, &L)) != KNN_OK) return st;
  s->contiguous = a.bin_map == KNN_BINS_CONTIGUOUS;
  s->keys64 = k1_tcs_supported(a.dtype, a.D, a.metric, a.N, L);
  if (s->contiguous && !s->keys64) return KNN_EUNSUPPORTED;
  if (s->keys64) {
    // K2 reads the merged [M][L] keys directly: a plan with one bin per L
    K1Plan p{};
    p.N = a.N;
    p.M = a.M;
    p.L = L;
    p.Lk = L;
    p.g = 1;
    p.D = a.D;
    p.pitch = (int)round_up(a.D, 16);
    p.metric = a.metric;
    p.dtype = stored_dtype(a.dtype);
    p.nsplits = 1;
    s->plan = p;
    s->Kp = kprime(a.K, a.rerank, L);
    s->qb = query_bytes(a.M, a.D, a.dtype, a.metric);
    size_t o = 0;
    s->off_qlp = o;
    o += s->qb.lp;
    s->off_qscale = o;
    o += s->qb.scale;
    s->off_qf32 = o;
    o += s->qb.f32;
    s->off_part_v = o;
    o += al((size_t)a.M * L * 8);
    s->off_part_a = o;
    s->off_cand = o;
    o += al((size_t)a.M * s->Kp * 8);
    s->total = o > kAlign ? o : kAlign;
    return KNN_OK;
  }
  s->plan = make_plan(a.N, a.M, L, a.D, a.metric, a.dtype, 0);
  if (s->plan.BQ == 0) return KNN_EUNSUPPORTED;
  s->Kp = kprime(a.K, a.rerank, L);
  s->qb = query_bytes(a.M, a.D, a.dtype, a.metric);
  size_t o = 0;
  s->off_qlp = o;
  o += s->qb.lp;
  s->off_qscale = o;
  o += s->qb.scale;
  s->off_qf32 = o;
  o += s->qb.f32;
  const size_t n = (size_t)((s->plan.atomic_merge ? 1 : s->plan.nsplits) * s->plan.M * s->plan.Lk);
  s->off_part_v = o;
  o += al(n * 4);
  s->off_part_a = o;
  if (a.dtype == KNN_F32) o += al(n * 4);
  s->off_cand = o;
  o += al((size_t)a.M * s->Kp * 8);
  s->total = o > kAlign ? o : kAlign;
  return KNN_OK;
}

knn_status check_pointers(const SearchArgs& a, const float* out_val, const int32_t* out_idx) {
  if (!a.db_lp || !a.q || !out_val || !out_idx) return KNN_EINVAL;
  if (a.metric == KNN_L2 && !a.db_hnorm) return KNN_EINVAL;
  if (stored_dtype(a.dtype) == KNN_E4M3 && !a.db_scale) return KNN_EINVAL;
  if (!aligned(a.db_lp, 16) || !aligned(a.q, 4) || !aligned(out_val, 4) || !aligned(out_idx, 4))
    return KNN_EINVAL;
  if (a.db_f32 && !aligned(a.db_f32, 4)) return KNN_EINVAL;
  return KNN_OK;
}

// Prepare queries into the workspace; returns the FP32 query rows the
// re-rank reads and their stride.
cudaError_t prep_queries(const SearchArgs& a, const SearchLayout& s, char* ws, const float** qf32,
                         int64_t* q_stride, cudaStream_t st) {
  void* qlp = ws + s.off_qlp;
  float* qscale = s.qb.scale ? reinterpret_cast<float*>(ws + s.off_qscale) : nullptr;
  float* qf = s.qb.f32 ? reinterpret_cast<float*>(ws + s.off_qf32) : nullptr;
  // merged partials start at zero: the same launch clears them
  const bool keys64 = s.keys64;
  uint32_t* zbuf = (s.plan.atomic_merge || keys64) ? reinterpret_cast<uint32_t*>(ws + s.off_part_v)
                                                   : nullptr;
  const int64_t zn = keys64 ? 2 * s.plan.M * s.plan.L
                            : (s.plan.atomic_merge ? s.plan.M * s.plan.Lk : 0);
  // queries keep per-row scales with either E4M3 database
  cudaError_t e = launch_prep(a.q, a.M, a.D, s.plan.pitch, a.metric, stored_dtype(a.dtype), qlp,
                              qscale, nullptr, qf, st, zbuf, zn);
  if (a.dtype == KNN_F32) {
    *qf32 = reinterpret_cast<const float*>(qlp);
    *q_stride = s.plan.pitch;
  } else if (a.metric == KNN_COS) {
    *qf32 = qf;
    *q_stride = a.D;
  } else {
    *qf32 = a.q;
    *q_stride = a.D;
  }
  return e;
}

cudaError_t run_k1(const K1Plan& p, const SearchArgs& a, const void* xlp, const float* xscale,
                   const float* hnorm, const void* qlp, const float* qscale, Partials parts,
                   cudaStream_t st) {
  if (parts.keys64)
    return launch_k1_tcs(p.N, p.M, p.L, p.D, p.metric, a.dtype, a.bin_map, xlp, xscale, hnorm,
                         qlp, reinterpret_cast<unsigned long long*>(parts.v), st);
  if (a.dtype == KNN_F32)
    return launch_k1_simt(p, reinterpret_cast<const float*>(xlp), hnorm,
                          reinterpret_cast<const float*>(qlp), parts, st);
  return launch_k1_tc(p, xlp, xscale, hnorm, qlp, qscale, parts, st);
}

knn_status search_impl(const SearchArgs& a, float* out_val, int32_t* out_idx, void* workspace,
                       size_t ws_bytes, cudaStream_t st) {
  SearchLayout s;
  knn_status rc = layout_search(a, &s);
  if (rc != KNN_OK) return rc;
  if (a.M == 0) return KNN_OK;
  if ((rc = check_pointers(a, out_val, out_idx)) != KNN_OK) return rc;
  if (!workspace || !aligned(workspace, kAlign)) return KNN_EINVAL;
  if (ws_bytes < s.total) return KNN_ENOMEM;
  char* ws = reinterpret_cast<char*>(workspace);
  const float* qf32;
  int64_t q_stride;
  cudaError_t e;
  {
    ProfScope ps(0, st);
    e = prep_queries(a, s, ws, &qf32, &q_stride, st);
  }
  if (e != cudaSuccess) return cuda_status(e);
  const bool k64 = s.keys64;
  Partials parts{reinterpret_cast<float*>(ws + s.off_part_v),
                 (a.dtype == KNN_F32 && !k64) ? reinterpret_cast<int32_t*>(ws + s.off_part_a)
                                              : nullptr,
                 0, s.plan.atomic_merge, k64};
  const float* qscale = s.qb.scale ? reinterpret_cast<const float*>(ws + s.off_qscale) : nullptr;
  {
    ProfScope ps(1, st);
    e = run_k1(s.plan, a, a.db_lp, a.db_scale, a.db_hnorm, ws + s.off_qlp, qscale, parts, st);
  }
  if (e == cudaErrorNotSupported) return KNN_EUNSUPPORTED;
  if (e != cudaSuccess) return cuda_status(e);
  if (k64 && k23_supported(a.M, s.plan.L, s.Kp, a.K, a.D, qf32, q_stride, a.db_f32)) {
    // ExactRescoring and the FP32 re-rank in one launch (profiled as K2)
    ProfScope ps(2, st);
    e = launch_k23(reinterpret_cast<const uint64_t*>(parts.v), a.M, s.plan.L, s.Kp, a.K, a.D,
                   a.metric, qf32, q_stride, a.db_f32, a.N, out_val, out_idx, st);
    return cuda_status(e);
  }
  uint64_t* cand = reinterpret_cast<uint64_t*>(ws + s.off_cand);
  {
    ProfScope ps(2, st);
    e = launch_k2(s.plan, parts, s.Kp, nullptr, cand, st, /*sorted=*/false);
  }
  if (e != cudaSuccess) return cuda_status(e);
  {
    ProfScope ps(3, st);
    e = launch_k3(a.M, a.D, a.metric, cand, s.Kp, a.K, qf32, q_stride, a.db_f32, a.db_lp,
                  stored_dtype(a.dtype), s.plan.pitch, a.db_scale, a.N, out_val, out_idx, st);
  }
  return cuda_status(e);
}

// ---------------------------------------------------------------------------
// Exact search: chunks of Nc rows, each a PartialReduce with one bin per row
// (L = Nc: every bin holds exactly one row, so the bin winners are all
// scores), merged into a running top-K per query.
// ---------------------------------------------------------------------------
struct ExactLayout {
  int64_t Nc;
  K1Plan plan;  // for a full chunk
  QueryBufs qb;
  size_t off_qlp, off_qscale, off_qf32, off_part_v, off_part_a, off_run, total;
};

constexpr int64_t kExactPartialBudget = (int64_t)1 << 26;  // entries per chunk

knn_status layout_exact(const SearchArgs& a, ExactLayout* s) {
  knn_status st = check_sizes(a.N, a.D, a.dtype, a.metric, a.M, a.K);
  if (st != KNN_OK) return st;
  int BW, BQ;
  k1_tile(a.dtype, a.D, a.M, &BW, &BQ);
  if (BQ == 0) return KNN_EUNSUPPORTED;
  int64_t mq = a.M > 0 ? a.M : 1;
  int64_t nc = (kExactPartialBudget / mq) / BW * BW;
  if (nc < BW) nc = BW;
  if (nc > a.N) nc = a.N;
  s->Nc = nc;
  s->plan = make_plan(nc, a.M, nc, a.D, a.metric, a.dtype, 1);
  s->qb = query_bytes(a.M, a.D, a.dtype, a.metric);
  size_t o = 0;
  s->off_qlp = o;
  o += s->qb.lp;
  s->off_qscale = o;
  o += s->qb.scale;
  s->off_qf32 = o;
  o += s->qb.f32;
  const size_t n = (size_t)(s->plan.M * s->plan.Lk);
  s->off_part_v = o;
  o += al(n * 4);
  s->off_part_a = o;
  if (a.dtype == KNN_F32) o += al(n * 4);
  s->off_run = o;
  o += al((size_t)a.M * a.K * 8);
  s->total = o > kAlign ? o : kAlign;
  return KNN_OK;
}

knn_status exact_impl(const SearchArgs& a, float* out_val, int32_t* out_idx, void* workspace,
                      size_t ws_bytes, cudaStream_t st) {
  ExactLayout s;
  knn_status rc = layout_exact(a, &s);
  if (rc != KNN_OK) return rc;
  if (a.M == 0) return KNN_OK;
  if ((rc = check_pointers(a, out_val, out_idx)) != KNN_OK) return rc;
  if (!workspace || !aligned(workspace, kAlign)) return KNN_EINVAL;
  if (ws_bytes < s.total) return KNN_ENOMEM;
  char* ws = reinterpret_cast<char*>(workspace);
  SearchLayout sl{};
  sl.plan = s.plan;
  sl.qb = s.qb;
  sl.off_qlp = s.off_qlp;
  sl.off_qscale = s.off_qscale;
  sl.off_qf32 = s.off_qf32;
  const float* qf32;
  int64_t q_stride;
  cudaError_t e = prep_queries(a, sl, ws, &qf32, &q_stride, st);
  if (e != cudaSuccess) return cuda_status(e);
  const float* qscale = s.qb.scale ? reinterpret_cast<const float*>(ws + s.off_qscale) : nullptr;
  uint64_t* run = reinterpret_cast<uint64_t*>(ws + s.off_run);
  const int esz = knn_dtype_bytes(a.dtype);
  for (int64_t n0 = 0; n0 < a.N; n0 += s.Nc) {
    const int64_t nc = (a.N - n0) < s.Nc ? (a.N - n0) : s.Nc;
    K1Plan p = make_plan(nc, a.M, nc, a.D, a.metric, a.dtype, 1);
    Partials parts{reinterpret_cast<float*>(ws + s.off_part_v),
                   a.dtype == KNN_F32 ? reinterpret_cast<int32_t*>(ws + s.off_part_a) : nullptr,
                   n0, false, false};
    const char* xlp = reinterpret_cast<const char*>(a.db_lp) + (size_t)n0 * p.pitch * esz;
    const float* xs = a.db_scale ? a.db_scale + n0 : nullptr;
    const float* hn = a.db_hnorm ? a.db_hnorm + n0 : nullptr;
    e = run_k1(p, a, xlp, xs, hn, ws + s.off_qlp, qscale, parts, st);
    if (e == cudaErrorNotSupported) return KNN_EUNSUPPORTED;
    if (e != cudaSuccess) return cuda_status(e);
    e = launch_k2(p, parts, a.K, n0 == 0 ? nullptr : run, run, st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  e = launch_k3(a.M, a.D, a.metric, run, a.K, a.K, qf32, q_stride, a.db_f32, a.db_lp,
                stored_dtype(a.dtype), s.plan.pitch, a.db_scale, a.N, out_val, out_idx, st);
  return cuda_status(e);
}

// ---------------------------------------------------------------------------
// The library's own search scratch (knn_search_static). A file-scope device
// array is reserved when the module is loaded, so a search through it needs
// no allocation at call time. Its device address belongs to the CUDA context
// the module is loaded in: it is looked up with the device current and kept
// per device together with that context's unique id (cuCtxGetId). A call that
// finds another context current -- after cudaDeviceReset the device's
// primary context is a new one -- looks the address up again.
// ---------------------------------------------------------------------------
constexpr int kMaxDevices = 64;
static __device__ __align__(256) unsigned char g_static_ws[KNN_STATIC_WORKSPACE_BYTES];
struct StaticWsSlot {
  unsigned long long ctx_id = 0;  // 0: nothing cached
  void* addr = nullptr;
};
StaticWsSlot g_static_ws_slot[kMaxDevices];
std::mutex g_static_ws_mu;

// Unique id of the context current on this thread (0 if none is current).
knn_status current_context_id(unsigned long long* id) {
  static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
  static PFN_cuCtxGetId_v12000 get_id = nullptr;
  if (!get_cur || !get_id) {
    void* p1 = nullptr;
    void* p2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p1, 4000, cudaEnableDefault, &q1) !=
            cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &p2, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return KNN_ECUDA;
    }
    get_cur = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p1);
    get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p2);
  }
  CUcontext ctx = nullptr;
  if (get_cur(&ctx) != CUDA_SUCCESS) return KNN_ECUDA;
  *id = 0;
  if (ctx && get_id(ctx, id) != CUDA_SUCCESS) return KNN_ECUDA;
  return KNN_OK;
}

knn_status static_workspace(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e);
  if (dev < 0 || dev >= kMaxDevices) return KNN_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_static_ws_mu);
  unsigned long long id = 0;
  knn_status rc = current_context_id(&id);
  if (rc != KNN_OK) return rc;
  StaticWsSlot& slot = g_static_ws_slot[dev];
  if (id != 0 && slot.ctx_id == id) {
    *out = slot.addr;
    return KNN_OK;
  }
  // first call in this context (the lookup makes the device's primary
  // context current if no context was)
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_static_ws);
  if (e != cudaSuccess) return cuda_status(e);
  if (!p || !aligned(p, kAlign)) return KNN_ECUDA;
  if ((rc = current_context_id(&id)) != KNN_OK) return rc;
  slot.ctx_id = id;
  slot.addr = p;
  *out = p;
  return KNN_OK;
}

static knn_status search_host_impl(const void* db_lp, const float* db_scale,
                                   const float* db_hnorm, const float* db_f32, int64_t N,
                                   int32_t D, int32_t dtype, int32_t metric, const float* q_host,
                                   int64_t M, int32_t K, int64_t L, int32_t bin_map,
                                   double recall_target, int32_t rerank_mult, float* out_val_host,
                                   int32_t* out_idx_host, void* workspace, size_t ws_bytes,
                                   void* stream, bool sync) {
  size_t base = knn_search_workspace(N, D, dtype, metric, M, K, L, bin_map, recall_target,
                                     rerank_mult);
  if (base == 0) return KNN_EINVAL;
  if (M == 0) return KNN_OK;
  if (!q_host || !out_val_host || !out_idx_host) return KNN_EINVAL;
  if (!workspace || !aligned(workspace, kAlign)) return KNN_EINVAL;
  size_t need = knn_search_host_workspace(N, D, dtype, metric, M, K, L, bin_map, recall_target,
                                          rerank_mult);
  if (ws_bytes < need) return KNN_ENOMEM;
  char* ws = reinterpret_cast<char*>(workspace);
  float* qd = reinterpret_cast<float*>(ws + al(base));
  float* vd = reinterpret_cast<float*>(ws + al(base) + al((size_t)M * D * 4));
  int32_t* id = reinterpret_cast<int32_t*>(ws + al(base) + al((size_t)M * D * 4) +
                                           al((size_t)M * K * 4));
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(qd, q_host, (size_t)M * D * 4, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e);
  knn_status rc = knn_search(db_lp, db_scale, db_hnorm, db_f32, N, D, dtype, metric, qd, M, K, L,
                             bin_map, recall_target, rerank_mult, vd, id, ws, base, stream);
  if (rc != KNN_OK) return rc;
  e = cudaMemcpyAsync(out_val_host, vd, (size_t)M * K * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out_idx_host, id, (size_t)M * K * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && sync) e = cudaStreamSynchronize(st);
  return cuda_status(e);
}

}  // namespace

// ===========================================================================
// extern "C"
// ===========================================================================
extern "C" {

const char* knn_status_string(int s) {
  switch (s) {
    case KNN_OK: return "ok";
    case KNN_EINVAL: return "invalid argument";
    case KNN_ENOMEM: return "workspace too small";
    case KNN_ECUDA: return "CUDA error";
    case KNN_ETIMEOUT: return "device-side wait timed out";
    case KNN_EUNSUPPORTED: return "unsupported";
    default: return "unknown status";
  }
}

int knn_last_cuda_error(void) { return g_last_cuda; }

int32_t knn_dtype_bytes(int32_t dtype) {
  switch (dtype) {
    case KNN_F32: return 4;
    case KNN_BF16: return 2;
    case KNN_E4M3:
    case KNN_E4M3_T: return 1;
    default: return 0;
  }
}

int32_t knn_row_pitch(int32_t D) { return D < 1 ? -1 : (int32_t)round_up(D, 16); }

int64_t knn_plan_bins(int64_t N, int32_t K, double recall_target, int32_t round_to) {
  return plan_bins(N, K, recall_target, round_to);
}

knn_status knn_prepare(const float* x, int64_t rows, int32_t D, int32_t metric, int32_t dtype,
                       void* out_lp, float* out_scale, float* out_hnorm, float* out_f32,
                       void* stream) {
  if (rows < 0 || D < 1 || !valid_metric(metric) || !valid_dtype(dtype)) return KNN_EINVAL;
  if (D > kMaxD) return KNN_EUNSUPPORTED;
  if (rows == 0) return KNN_OK;
  if (!x || !out_lp || !aligned(out_lp, 16) || !aligned(x, 4)) return KNN_EINVAL;
  if (stored_dtype(dtype) == KNN_E4M3 && !out_scale) return KNN_EINVAL;
  if (metric == KNN_L2 && !out_hnorm) return KNN_EINVAL;
  if (metric == KNN_COS && !out_f32) return KNN_EINVAL;
  return cuda_status(launch_prep(x, rows, D, knn_row_pitch(D), metric, dtype, out_lp, out_scale,
                                 out_hnorm, out_f32, (cudaStream_t)stream));
}

size_t knn_search_workspace(int64_t N, int32_t D, int32_t dtype, int32_t metric, int64_t M,
                            int32_t K, int64_t L, int32_t bin_map, double recall_target,
                            int32_t rerank_mult) {
  SearchArgs a{nullptr, nullptr, nullptr, nullptr, N, D, dtype, metric, nullptr, M, K, L,
               recall_target, rerank_mult, bin_map};
  SearchLayout s;
  if (layout_search(a, &s) != KNN_OK) return 0;
  return s.total;
}

knn_status knn_search(const void* db_lp, const float* db_scale, const float* db_hnorm,
                      const float* db_f32, int64_t N, int32_t D, int32_t dtype, int32_t metric,
                      const float* q, int64_t M, int32_t K, int64_t L, int32_t bin_map,
                      double recall_target, int32_t rerank_mult, float* out_val,
                      int32_t* out_idx, void* workspace, size_t ws_bytes, void* stream) {
  SearchArgs a{db_lp, db_scale, db_hnorm, db_f32, N, D, dtype, metric, q, M, K, L,
               recall_target, rerank_mult, bin_map};
  return search_impl(a, out_val, out_idx, workspace, ws_bytes, (cudaStream_t)stream);
}

size_t knn_search_host_workspace(int64_t N, int32_t D, int32_t dtype, int32_t metric, int64_t M,
                                 int32_t K, int64_t L, int32_t bin_map, double recall_target,
                                 int32_t rerank_mult) {
  size_t base = knn_search_workspace(N, D, dtype, metric, M, K, L, bin_map, recall_target,
                                     rerank_mult);
  if (base == 0) return 0;
  return al(base) + al((size_t)M * D * 4) + al((size_t)M * K * 4) * 2;
}

knn_status knn_search_host(const void* db_lp, const float* db_scale, const float* db_hnorm,
                           const float* db_f32, int64_t N, int32_t D, int32_t dtype,
                           int32_t metric, const float* q_host, int64_t M, int32_t K, int64_t L,
                           int32_t bin_map, double recall_target, int32_t rerank_mult,
                           float* out_val_host, int32_t* out_idx_host, void* workspace,
                           size_t ws_bytes, void* stream) {
  return search_host_impl(db_lp, db_scale, db_hnorm, db_f32, N, D, dtype, metric, q_host, M, K, L,
                          bin_map, recall_target, rerank_mult, out_val_host, out_idx_host,
                          workspace, ws_bytes, stream, true);
}

knn_status knn_search_host_async(const void* db_lp, const float* db_scale,
                                 const float* db_hnorm, const float* db_f32, int64_t N,
                                 int32_t D, int32_t dtype, int32_t metric, const float* q_host,
                                 int64_t M, int32_t K, int64_t L, int32_t bin_map,
                                 double recall_target, int32_t rerank_mult, float* out_val_host,
                                 int32_t* out_idx_host, void* workspace, size_t ws_bytes,
                                 void* stream) {
  return search_host_impl(db_lp, db_scale, db_hnorm, db_f32, N, D, dtype, metric, q_host, M, K, L,
                          bin_map, recall_target, rerank_mult, out_val_host, out_idx_host,
                          workspace, ws_bytes, stream, false);
}

knn_status knn_search_static(const void* db_lp, const float* db_scale, const float* db_hnorm,
                             const float* db_f32, int64_t N, int32_t D, int32_t dtype,
                             int32_t metric, const float* q, int64_t M, int32_t K, int64_t L,
                             int32_t bin_map, double recall_target, int32_t rerank_mult,
                             float* out_val, int32_t* out_idx, void* stream) {
  SearchArgs a{db_lp, db_scale, db_hnorm, db_f32, N, D, dtype, metric, q, M, K, L,
               recall_target, rerank_mult, bin_map};
  // every size check comes before the device is touched
  SearchLayout s;
  knn_status rc = layout_search(a, &s);
  if (rc != KNN_OK) return rc;
  if (s.total > (size_t)KNN_STATIC_WORKSPACE_BYTES) return KNN_ENOMEM;
  if (a.M == 0) return KNN_OK;
  if ((rc = check_pointers(a, out_val, out_idx)) != KNN_OK) return rc;
  void* ws = nullptr;
  if ((rc = static_workspace(&ws)) != KNN_OK) return rc;
  return search_impl(a, out_val, out_idx, ws, (size_t)KNN_STATIC_WORKSPACE_BYTES,
                     (cudaStream_t)stream);
}

size_t knn_partial_reduce_workspace(int64_t N, int32_t D, int32_t dtype, int32_t metric,
                                    int64_t M, int64_t L, int32_t bin_map) {
  if (L < 1 || L > N) return 0;
  SearchArgs a{nullptr, nullptr, nullptr, nullptr, N, D, dtype, metric, nullptr, M, 1, L, 0.5, 1,
               bin_map};
  SearchLayout s;
  if (layout_search(a, &s) != KNN_OK) return 0;
  return s.total;
}

knn_status knn_partial_reduce(const void* db_lp, const float* db_scale, const float* db_hnorm,
                              int64_t N, int32_t D, int32_t dtype, int32_t metric, const float* q,
                              int64_t M, int64_t L, int32_t bin_map, float* out_v, int32_t* out_a,
                              void* workspace, size_t ws_bytes, void* stream) {
  if (L < 1 || L > N) return KNN_EINVAL;
  SearchArgs a{db_lp, db_scale, db_hnorm, nullptr, N, D, dtype, metric, q, M, 1, L, 0.5, 1,
               bin_map};
  SearchLayout s;
  knn_status rc = layout_search(a, &s);
  if (rc != KNN_OK) return rc;
  if (M == 0) return KNN_OK;
  if ((rc = check_pointers(a, out_v, out_a)) != KNN_OK) return rc;
  if (!workspace || !aligned(workspace, kAlign)) return KNN_EINVAL;
  if (ws_bytes < s.total) return KNN_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = reinterpret_cast<char*>(workspace);
  const float* qf32;
  int64_t q_stride;
  cudaError_t e = prep_queries(a, s, ws, &qf32, &q_stride, st);
  if (e != cudaSuccess) return cuda_status(e);
  const bool k64 = s.keys64;
  Partials parts{reinterpret_cast<float*>(ws + s.off_part_v),
                 (dtype == KNN_F32 && !k64) ? reinterpret_cast<int32_t*>(ws + s.off_part_a)
                                            : nullptr,
                 0, s.plan.atomic_merge, k64};
  const float* qscale = s.qb.scale ? reinterpret_cast<const float*>(ws + s.off_qscale) : nullptr;
  e = run_k1(s.plan, a, db_lp, db_scale, db_hnorm, ws + s.off_qlp, qscale, parts, st);
  if (e == cudaErrorNotSupported) return KNN_EUNSUPPORTED;
  if (e != cudaSuccess) return cuda_status(e);
  return cuda_status(launch_merge_bins(s.plan, parts, out_v, out_a, st));
}

// ---------------------------------------------------------------------------
// approx_max_k on a given score matrix (App. A.1)
// ---------------------------------------------------------------------------
static knn_status amk_resolve(int64_t M, int64_t N, int32_t K, int64_t L, int64_t planning_size,
                              double recall_target, int32_t aggregate, int64_t* Lout) {
  if (M < 0 || N < 1 || N >= ((int64_t)1 << 31)) return KNN_EINVAL;
  if (L <= 0) {
    if (K < 1) return KNN_EINVAL;
    L = plan_bins(planning_size > 0 ? planning_size : N, K, recall_target, 1);
    if (L < 1) return KNN_EINVAL;
    if (L > N) L = N;
  }
  if (L > N) return KNN_EINVAL;
  if (aggregate && (K < 1 || K > L || K > kMaxK)) return KNN_EINVAL;
  *Lout = L;
  return KNN_OK;
}

size_t knn_approx_max_k_workspace(int64_t M, int64_t N, int32_t K, int64_t L,
                                  int64_t planning_size, double recall_target,
                                  int32_t aggregate_to_topk) {
  int64_t Lr;
  if (amk_resolve(M, N, K, L, planning_size, recall_target, aggregate_to_topk, &Lr) != KNN_OK)
    return 0;
  size_t t = al((size_t)M * Lr * 8) + (aggregate_to_topk ? al((size_t)M * K * 8) : 0);
  return t > kAlign ? t : kAlign;
}

knn_status knn_approx_max_k(const void* scores, int32_t score_dtype, int64_t M, int64_t N,
                            int32_t K, int64_t L, int64_t planning_size, double recall_target,
                            int32_t bin_map, int32_t is_min, int32_t aggregate_to_topk,
                            float* out_val, int32_t* out_idx, void* workspace, size_t ws_bytes,
                            void* stream) {
  int64_t Lr;
  knn_status rc = amk_resolve(M, N, K, L, planning_size, recall_target, aggregate_to_topk, &Lr);
  if (rc != KNN_OK) return rc;
  if (score_dtype != KNN_F32 && score_dtype != KNN_BF16) return KNN_EINVAL;
  if (bin_map != KNN_BINS_MOD && bin_map != KNN_BINS_CONTIGUOUS) return KNN_EINVAL;
  if (M == 0) return KNN_OK;
  if (!scores || !out_val || !out_idx || !aligned(out_val, 4) || !aligned(out_idx, 4) ||
      !aligned(scores, score_dtype == KNN_BF16 ? 2 : 4))
    return KNN_EINVAL;
  if (!workspace || !aligned(workspace, kAlign)) return KNN_EINVAL;
  const size_t need = knn_approx_max_k_workspace(M, N, K, Lr, 0, recall_target, aggregate_to_topk);
  if (ws_bytes < need) return KNN_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = reinterpret_cast<char*>(workspace);
  unsigned long long* G = reinterpret_cast<unsigned long long*>(ws);
  cudaError_t e = cudaMemsetAsync(G, 0, (size_t)M * Lr * 8, st);
  if (e == cudaSuccess)
    e = launch_bin_max(scores, score_dtype, M, N, Lr, bin_map, is_min ? 1 : 0, G, st);
  if (e != cudaSuccess) return cuda_status(e);
  if (!aggregate_to_topk)
    return cuda_status(launch_keys_to_pairs(reinterpret_cast<const uint64_t*>(G), M * Lr,
                                            is_min ? 1 : 0, out_val, out_idx, st));
  K1Plan p{};
  p.M = M;
  p.N = N;
  p.L = Lr;
  p.Lk = Lr;
  p.g = 1;
  p.nsplits = 1;
  Partials parts{reinterpret_cast<float*>(G), nullptr, 0, false, true};
  uint64_t* keys = reinterpret_cast<uint64_t*>(ws + al((size_t)M * Lr * 8));
  e = launch_k2(p, parts, K, nullptr, keys, st);
  if (e == cudaSuccess)
    e = launch_keys_to_pairs(keys, M * K, is_min ? 1 : 0, out_val, out_idx, st);
  return cuda_status(e);
}

size_t knn_search_exact_workspace(int64_t N, int32_t D, int32_t dtype, int32_t metric, int64_t M,
                                  int32_t K) {
  SearchArgs a{nullptr, nullptr, nullptr, nullptr, N, D, dtype, metric, nullptr, M, K, N, 0.5, 1,
               KNN_BINS_MOD};
  ExactLayout s;
  if (layout_exact(a, &s) != KNN_OK) return 0;
  return s.total;
}

knn_status knn_search_exact(const void* db_lp, const float* db_scale, const float* db_hnorm,
                            const float* db_f32, int64_t N, int32_t D, int32_t dtype,
                            int32_t metric, const float* q, int64_t M, int32_t K,
                            float* out_val, int32_t* out_idx, void* workspace, size_t ws_bytes,
                            void* stream) {
  SearchArgs a{db_lp, db_scale, db_hnorm, db_f32, N, D, dtype, metric, q, M, K, N, 0.5, 1,
               KNN_BINS_MOD};
  return exact_impl(a, out_val, out_idx, workspace, ws_bytes, (cudaStream_t)stream);
}

size_t knn_backward_workspace(int64_t N, int32_t D, int64_t M, int32_t K, int32_t deterministic) {
  (void)D;
  (void)deterministic;  // one size serves both modes
  return backward_ws_bytes(N, M, K);
}

knn_status knn_backward(const void* db_lp, const float* db_scale, const float* x_f32, int64_t N,
                        int32_t D, int32_t dtype, int32_t metric, const float* q, int64_t M,
                        int32_t K, const int32_t* idx, const float* grad_val, float* dq,
                        float* dx, int32_t zero_dx, int32_t deterministic, void* workspace,
                        size_t ws_bytes, void* stream) {
  if (N < 1 || D < 1 || M < 0 || K < 1 || !valid_metric(metric) || !valid_dtype(dtype))
    return KNN_EINVAL;
  if (D > kMaxD) return KNN_EUNSUPPORTED;
  if (!x_f32 && !db_lp) return KNN_EINVAL;
  if (!x_f32 && stored_dtype(dtype) == KNN_E4M3 && !db_scale) return KNN_EINVAL;
  if (M > 0 && (!q || !idx || !grad_val)) return KNN_EINVAL;
  if (M * (int64_t)K >= ((int64_t)1 << 31)) return KNN_EUNSUPPORTED;
  const size_t need = backward_ws_bytes(N, M, K);
  if (dx && M > 0 && (deterministic || workspace)) {
    if (!workspace || !aligned(workspace, kAlign)) return KNN_EINVAL;
    if (ws_bytes < need) return KNN_ENOMEM;
  }
  if (!dq && !dx) return KNN_OK;
  return cuda_status(launch_backward(M, D, K, metric, q, x_f32, db_lp, stored_dtype(dtype),
                                     knn_row_pitch(D),
                                     db_scale, N, idx, grad_val, dq, dx, zero_dx, deterministic,
                                     dx && M > 0 ? workspace : nullptr, (cudaStream_t)stream));
}

// ---------------------------------------------------------------------------
// N-sharded search (knn_shard_*): the shard's rows are global rows
// [row0, row0 + n_local) of an N_global-row database; bins are j mod L of the
// global index, which the local grid view keeps when row0 is a multiple of L.
// ---------------------------------------------------------------------------
static knn_status shard_layout(int64_t n_local, int64_t row0, int64_t N_global, int32_t D,
                               int32_t dtype, int32_t metric, int64_t M, int64_t L,
                               SearchLayout* s, size_t* total) {
  if (N_global < 1 || N_global >= ((int64_t)1 << 31) - 1 || M < 0) return KNN_EINVAL;
  if (n_local < 1 || row0 < 0 || row0 + n_local > N_global) return KNN_EINVAL;
  if (L < 1 || L > n_local || row0 % L != 0) return KNN_EINVAL;
  SearchArgs a{nullptr, nullptr, nullptr, nullptr, n_local, D, dtype, metric, nullptr, M, 1, L,
               0.5, 1, KNN_BINS_MOD};
  knn_status st = layout_search(a, s);
  if (st != KNN_OK) return st;
  *total = al(s->total) + 2 * al((size_t)M * L * 4);
  return KNN_OK;
}

size_t knn_shard_partial_reduce_workspace(int64_t n_local, int64_t row0, int64_t N_global,
                                          int32_t D, int32_t dtype, int32_t metric, int64_t M,
                                          int64_t L) {
  SearchLayout s;
  size_t t = 0;
  if (shard_layout(n_local, row0, N_global, D, dtype, metric, M, L, &s, &t) != KNN_OK) return 0;
  return t;
}

knn_status knn_shard_partial_reduce(const void* db_lp, const float* db_scale,
                                    const float* db_hnorm, int64_t n_local, int64_t row0,
                                    int64_t N_global, int32_t D, int32_t dtype, int32_t metric,
                                    const float* q, int64_t M, int64_t L, int64_t* keys,
                                    void* workspace, size_t ws_bytes, void* stream) {
  SearchLayout s;
  size_t total = 0;
  knn_status rc = shard_layout(n_local, row0, N_global, D, dtype, metric, M, L, &s, &total);
  if (rc != KNN_OK) return rc;
  if (M == 0) return KNN_OK;
  SearchArgs a{db_lp, db_scale, db_hnorm, nullptr, n_local, D, dtype, metric, q, M, 1, L, 0.5, 1,
               KNN_BINS_MOD};
  if (!keys || !aligned(keys, 8)) return KNN_EINVAL;
  if ((rc = check_pointers(a, reinterpret_cast<float*>(keys), reinterpret_cast<int32_t*>(keys))) !=
      KNN_OK)
    return rc;
  if (!workspace || !aligned(workspace, kAlign)) return KNN_EINVAL;
  if (ws_bytes < total) return KNN_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = reinterpret_cast<char*>(workspace);
  const float* qf32;
  int64_t q_stride;
  cudaError_t e = prep_queries(a, s, ws, &qf32, &q_stride, st);
  if (e != cudaSuccess) return cuda_status(e);
  const bool k64 = s.keys64;
  // pair and packed partials decode their rows with the shard's offset; the
  // 64-bit keys hold local rows, offset when they become signed keys
  Partials parts{reinterpret_cast<float*>(ws + s.off_part_v),
                 (dtype == KNN_F32 && !k64) ? reinterpret_cast<int32_t*>(ws + s.off_part_a)
                                            : nullptr,
                 k64 ? 0 : row0, s.plan.atomic_merge, k64};
  const float* qscale = s.qb.scale ? reinterpret_cast<const float*>(ws + s.off_qscale) : nullptr;
  e = run_k1(s.plan, a, db_lp, db_scale, db_hnorm, ws + s.off_qlp, qscale, parts, st);
  if (e == cudaErrorNotSupported) return KNN_EUNSUPPORTED;
  if (e != cudaSuccess) return cuda_status(e);
  float* V = reinterpret_cast<float*>(ws + al(s.total));
  int32_t* A = reinterpret_cast<int32_t*>(ws + al(s.total) + al((size_t)M * L * 4));
  e = launch_merge_bins(s.plan, parts, V, A, st);
  if (e == cudaSuccess) e = launch_pairs_to_signed_keys(V, A, M * L, k64 ? row0 : 0, keys, st);
  return cuda_status(e);
}

int32_t knn_rescore_count(int32_t K, int32_t rerank_mult, int64_t L) {
  if (K < 1 || L < 1 || K > L || K > kMaxK) return -1;
  return kprime(K, rerank_mult, L);
}

size_t knn_shard_rescore_workspace(int64_t M, int64_t L, int32_t D, int32_t metric, int32_t K,
                                   int32_t rerank_mult) {
  if (M < 0 || D < 1 || D > kMaxD || !valid_metric(metric)) return 0;
  const int32_t Kp = knn_rescore_count(K, rerank_mult, L);
  if (Kp < 1) return 0;
  size_t t = al((size_t)M * L * 8) + al((size_t)M * Kp * 8);
  if (metric == KNN_COS) t += al((size_t)M * knn_row_pitch(D) * 4);
  return t > kAlign ? t : kAlign;
}

knn_status knn_shard_rescore(const int64_t* keys, int64_t M, int64_t L, int32_t K,
                             int32_t rerank_mult, const float* q, int32_t D, int32_t metric,
                             const float* x_f32, int64_t n_local, int64_t row0,
                             int64_t* cand_keys, void* workspace, size_t ws_bytes,
                             void* stream) {
  const size_t need = knn_shard_rescore_workspace(M, L, D, metric, K, rerank_mult);
  if (need == 0 || n_local < 1 || row0 < 0 || row0 + n_local >= ((int64_t)1 << 31))
    return KNN_EINVAL;
  if (M == 0) return KNN_OK;
  if (!keys || !q || !x_f32 || !cand_keys || !aligned(keys, 8) || !aligned(cand_keys, 8) ||
      !aligned(q, 4) || !aligned(x_f32, 4))
    return KNN_EINVAL;
  if (!workspace || !aligned(workspace, kAlign)) return KNN_EINVAL;
  if (ws_bytes < need) return KNN_ENOMEM;
  const int32_t Kp = knn_rescore_count(K, rerank_mult, L);
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = reinterpret_cast<char*>(workspace);
  uint64_t* G = reinterpret_cast<uint64_t*>(ws);
  uint64_t* cand = reinterpret_cast<uint64_t*>(ws + al((size_t)M * L * 8));
  cudaError_t e = launch_signed_to_keys(keys, M * L, G, st);
  K1Plan p{};
  p.M = M;
  p.L = L;
  p.Lk = L;
  p.g = 1;
  p.nsplits = 1;
  Partials parts{reinterpret_cast<float*>(G), nullptr, 0, false, true};
  if (e == cudaSuccess) e = launch_k2(p, parts, Kp, nullptr, cand, st, /*sorted=*/false);
  const float* qf = q;
  int64_t q_stride = D;
  if (e == cudaSuccess && metric == KNN_COS) {
    // cosine: the candidates' unit rows against the unit queries
    float* qn = reinterpret_cast<float*>(ws + al((size_t)M * L * 8) + al((size_t)M * Kp * 8));
    const int pitch = knn_row_pitch(D);
    e = launch_prep(q, M, D, pitch, KNN_COS, KNN_F32, qn, nullptr, nullptr, nullptr, st);
    qf = qn;
    q_stride = pitch;
  }
  if (e == cudaSuccess)
    e = launch_score_owned(cand, M, Kp, qf, q_stride, x_f32, n_local, row0, D, metric, cand_keys,
                           st);
  return cuda_status(e);
}

size_t knn_shard_finish_workspace(int64_t M, int32_t Kp, int32_t K) {
  if (M < 0 || K < 1 || Kp < K || Kp > kMaxK) return 0;
  const size_t t = al((size_t)M * Kp * 8) + al((size_t)M * K * 8);
  return t > kAlign ? t : kAlign;
}

knn_status knn_shard_finish(const int64_t* cand_keys, int64_t M, int32_t Kp, int32_t K,
                            int32_t metric, float* out_val, int32_t* out_idx, void* workspace,
                            size_t ws_bytes, void* stream) {
  const size_t need = knn_shard_finish_workspace(M, Kp, K);
  if (need == 0 || !valid_metric(metric)) return KNN_EINVAL;
  if (M == 0) return KNN_OK;
  if (!cand_keys || !out_val || !out_idx || !aligned(cand_keys, 8) || !aligned(out_val, 4) ||
      !aligned(out_idx, 4))
    return KNN_EINVAL;
  if (!workspace || !aligned(workspace, kAlign)) return KNN_EINVAL;
  if (ws_bytes < need) return KNN_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = reinterpret_cast<char*>(workspace);
  uint64_t* C = reinterpret_cast<uint64_t*>(ws);
  uint64_t* top = reinterpret_cast<uint64_t*>(ws + al((size_t)M * Kp * 8));
  cudaError_t e = launch_signed_to_keys(cand_keys, M * Kp, C, st);
  K1Plan p{};
  p.M = M;
  p.L = Kp;
  p.Lk = Kp;
  p.g = 1;
  p.nsplits = 1;
  Partials parts{reinterpret_cast<float*>(C), nullptr, 0, false, true};
  if (e == cudaSuccess) e = launch_k2(p, parts, K, nullptr, top, st);
  // internal scores are larger-is-better: L2 reports the squared distance
  if (e == cudaSuccess)
    e = launch_keys_to_pairs(top, M * K, metric == KNN_L2 ? 1 : 0, out_val, out_idx, st);
  return cuda_status(e);
}

// ---------------------------------------------------------------------------
// Library-owned database (knn_db_*): the prepared rows and their side arrays
// in device memory the handle allocates and frees.
// ---------------------------------------------------------------------------
struct knn_db {
  int64_t N;
  int32_t D, metric, dtype;
  int device;
  void* lp;
  float* scale;
  float* hnorm;
  float* f32;
};

static void db_free(knn_db* h) {
  if (!h) return;
  int cur = -1;
  const bool switched = cudaGetDevice(&cur) == cudaSuccess && cur != h->device &&
                        cudaSetDevice(h->device) == cudaSuccess;
  if (h->lp) cudaFree(h->lp);
  if (h->scale) cudaFree(h->scale);
  if (h->hnorm) cudaFree(h->hnorm);
  if (h->f32) cudaFree(h->f32);
  if (switched) cudaSetDevice(cur);
  delete h;
}

knn_status knn_db_create(const float* x, int64_t N, int32_t D, int32_t metric, int32_t dtype,
                         int32_t keep_f32, void* stream, knn_db** out) {
  if (!out) return KNN_EINVAL;
  *out = nullptr;
  if (N < 1 || N >= ((int64_t)1 << 31) - 1 || D < 1 || !valid_metric(metric) ||
      !valid_dtype(dtype) || !x || !aligned(x, 4))
    return KNN_EINVAL;
  if (D > kMaxD) return KNN_EUNSUPPORTED;
  knn_db* h = new (std::nothrow) knn_db{N, D, metric, dtype, 0, nullptr, nullptr, nullptr, nullptr};
  if (!h) return KNN_ENOMEM;
  cudaError_t e = cudaGetDevice(&h->device);
  const size_t lp_bytes = (size_t)N * knn_row_pitch(D) * knn_dtype_bytes(dtype);
  const bool want_f32 = metric == KNN_COS || keep_f32;
  if (e == cudaSuccess) e = cudaMalloc(&h->lp, lp_bytes);
  if (e == cudaSuccess && stored_dtype(dtype) == KNN_E4M3)
    e = cudaMalloc(reinterpret_cast<void**>(&h->scale), (size_t)N * 4);
  if (e == cudaSuccess && metric == KNN_L2)
    e = cudaMalloc(reinterpret_cast<void**>(&h->hnorm), (size_t)N * 4);
  if (e == cudaSuccess && want_f32)
    e = cudaMalloc(reinterpret_cast<void**>(&h->f32), (size_t)N * D * 4);
  cudaStream_t st = (cudaStream_t)stream;
  // the re-rank source: the unit rows for COS (written by the preparation),
  // else a copy of the rows as given
  if (e == cudaSuccess && want_f32 && metric != KNN_COS)
    e = cudaMemcpyAsync(h->f32, x, (size_t)N * D * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess)
    e = launch_prep(x, N, D, knn_row_pitch(D), metric, dtype, h->lp, h->scale, h->hnorm,
                    metric == KNN_COS ? h->f32 : nullptr, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    const knn_status rc = e == cudaErrorMemoryAllocation ? KNN_ENOMEM : cuda_status(e);
    cudaGetLastError();
    db_free(h);
    return rc;
  }
  *out = h;
  return KNN_OK;
}

knn_status knn_db_destroy(knn_db* db) {
  if (!db) return KNN_EINVAL;
  db_free(db);
  return KNN_OK;
}

knn_status knn_db_info(const knn_db* db, int64_t* N, int32_t* D, int32_t* metric,
                       int32_t* dtype) {
  if (!db) return KNN_EINVAL;
  if (N) *N = db->N;
  if (D) *D = db->D;
  if (metric) *metric = db->metric;
  if (dtype) *dtype = db->dtype;
  return KNN_OK;
}

size_t knn_db_search_workspace(const knn_db* db, int64_t M, int32_t K, int64_t L, int32_t bin_map,
                               double recall_target, int32_t rerank_mult) {
  if (!db) return 0;
  return knn_search_workspace(db->N, db->D, db->dtype, db->metric, M, K, L, bin_map,
                              recall_target, rerank_mult);
}

knn_status knn_db_search(const knn_db* db, const float* q, int64_t M, int32_t K, int64_t L,
                         int32_t bin_map, double recall_target, int32_t rerank_mult,
                         float* out_val, int32_t* out_idx, void* workspace, size_t ws_bytes,
                         void* stream) {
  if (!db) return KNN_EINVAL;
  return knn_search(db->lp, db->scale, db->hnorm, db->f32, db->N, db->D, db->dtype, db->metric, q,
                    M, K, L, bin_map, recall_target, rerank_mult, out_val, out_idx, workspace,
                    ws_bytes, stream);
}

knn_status knn_profile_enable(int32_t on) {
  g_prof.on = false;
  if (!on) return KNN_OK;
  for (int c = 0; c < kProfClasses; ++c) {
    if (!g_prof.ev[c]) {
      cudaEvent_t* ev = new (std::nothrow) cudaEvent_t[2 * kProfCap];
      if (!ev) return KNN_ENOMEM;
      for (int i = 0; i < 2 * kProfCap; ++i) {
        cudaError_t e = cudaEventCreate(&ev[i]);
        if (e != cudaSuccess) return cuda_status(e);
      }
      g_prof.ev[c] = ev;
    }
    g_prof.n[c] = 0;
  }
  g_prof.on = true;
  return KNN_OK;
}

knn_status knn_profile_read(int32_t kernel_class, double* total_ms, int64_t* launches) {
  if (kernel_class < 0 || kernel_class >= kProfClasses || !total_ms || !launches)
    return KNN_EINVAL;
  double t = 0.0;
  const int64_t n = g_prof.n[kernel_class];
  for (int64_t i = 0; i < n; ++i) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(g_prof.ev[kernel_class][2 * i + 1]);
    if (e == cudaSuccess)
      e = cudaEventElapsedTime(&ms, g_prof.ev[kernel_class][2 * i],
                               g_prof.ev[kernel_class][2 * i + 1]);
    if (e != cudaSuccess) return cuda_status(e);
    t += ms;
  }
  *total_ms = t;
  *launches = n;
  return KNN_OK;
}

knn_status knn_measure_rate(int32_t kind, int64_t iters, double* ops_per_s, double* ms,
                            void* stream) {
  if ((kind != KNN_RATE_MINMAX && kind != KNN_RATE_FFMA) || iters < 1 || !ops_per_s || !ms)
    return KNN_EINVAL;
  return cuda_status(measure_rate(kind, iters, ops_per_s, ms, (cudaStream_t)stream));
}

knn_status knn_set_wait_limit_ns(uint64_t ns) {
  const bool a = k1_tc_set_wait_limit((unsigned long long)ns);
  const bool b = k1_tcs_set_wait_limit((unsigned long long)ns);
  return (a && b) ? KNN_OK : KNN_ECUDA;
}

knn_status knn_sync_status(void) {
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e);
  const bool t1 = k1_tc_take_timeout();
  const bool t2 = k1_tcs_take_timeout();
  if (t1 || t2) return KNN_ETIMEOUT;
  return KNN_OK;
}

}  // extern "C"
