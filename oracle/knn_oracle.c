/*
 * knn_oracle.c -- plain FP64 CPU oracle for the TPU-KNN search path
 * (arXiv 2206.14286).
 *
 * TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load this library. The product path (the
 * CUDA library and its Python binding) never calls it, and this file shares
 * no code, header, table or constant with it.
 *
 * Everything here is written for a reader checking it against the paper by
 * eye: straight loops, FP64 arithmetic, no blocking or fusion. OpenMP splits
 * the outer loop over queries only; each query's work is sequential and its
 * result does not depend on the thread count.
 *
 * Conventions
 *   - Matrices are row-major. Q is M x D (queries), X is N x D (database).
 *   - metric 0 = inner product (MIPS, Eq. 2), 1 = Euclidean (Eq. 1 with the
 *     l2 distance), 2 = cosine (Sec. 2: distance 1 - <x,y>/(|x||y|)).
 *   - Internally every metric is a score where larger is better:
 *       IP : s = <q,x>
 *       L2 : s = -||q - x||^2   (same argmin as ||q-x||_2, App. A.2 Eq. 15-16)
 *       COS: s = <q,x> / (||q|| ||x||)  (argmin of the cosine distance)
 *     Reported values: IP -> <q,x>, L2 -> ||q-x||^2, COS -> cosine similarity.
 *   - Ties between equal scores go to the smaller database index (the paper
 *     is silent; this is the reading the library also takes).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (contraction off so
 * that the FP32/FP64 preparation routines round every operation separately,
 * identically on x86-64 and aarch64).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_IP 0
#define ORC_L2 1
#define ORC_COS 2

/* ---------------------------------------------------------------------- */
/* Scores (Sec. 2, Eq. 1-2)                                                */
/* ---------------------------------------------------------------------- */

static double dot(const double *a, const double *b, int D) {
  double s = 0.0;
  for (int d = 0; d < D; ++d) s += a[d] * b[d];
  return s;
}

/* Larger-is-better score of database row x for query q. */
static double score(const double *q, const double *x, int D, int metric) {
  if (metric == ORC_IP) return dot(q, x, D);
  if (metric == ORC_L2) {
    double s = 0.0;
    for (int d = 0; d < D; ++d) {
      double t = q[d] - x[d];
      s += t * t;
    }
    return -s;
  }
  /* cosine similarity; a zero row has no direction and scores 0 */
  double nq = sqrt(dot(q, q, D)), nx = sqrt(dot(x, x, D));
  if (nq == 0.0 || nx == 0.0) return 0.0;
  return dot(q, x, D) / (nq * nx);
}

/* The value the search reports for an internal score. */
static double reported(double s, int metric) { return metric == ORC_L2 ? -s : s; }

double orc_score(const double *q, const double *x, int D, int metric) {
  return score(q, x, D, metric);
}

/* a ranks before b: larger score first, then smaller index */
static int ranks_before(double sa, int64_t ja, double sb, int64_t jb) {
  return sa > sb || (sa == sb && ja < jb);
}

/* Insert (s, j) into a list kept sorted by ranks_before, capacity K. */
static void insert_sorted(double *vs, int64_t *js, int *cnt, int K, double s, int64_t j) {
  int n = *cnt;
  if (n == K && !ranks_before(s, j, vs[n - 1], js[n - 1])) return;
  int pos = (n < K) ? n : K - 1;
  while (pos > 0 && ranks_before(s, j, vs[pos - 1], js[pos - 1])) {
    vs[pos] = vs[pos - 1];
    js[pos] = js[pos - 1];
    --pos;
  }
  vs[pos] = s;
  js[pos] = j;
  if (n < K) *cnt = n + 1;
}

/* ---------------------------------------------------------------------- */
/* Exact K-NN (Eq. 1 / Eq. 2): K-argmax of the score over all N rows.      */
/* out_val[M*K] holds reported values, out_idx[M*K] indices, best first.   */
/* Slots beyond N (K > N) get index -1 and value NaN.                      */
/* ---------------------------------------------------------------------- */
void orc_exact_topk(const double *Q, int64_t M, const double *X, int64_t N, int D,
                    int metric, int K, double *out_val, int64_t *out_idx) {
#pragma omp parallel
  {
    double *vs = (double *)malloc(sizeof(double) * (size_t)K);
    int64_t *js = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
#pragma omp for schedule(dynamic, 1)
    for (int64_t i = 0; i < M; ++i) {
      int cnt = 0;
      const double *q = Q + i * D;
      for (int64_t j = 0; j < N; ++j)
        insert_sorted(vs, js, &cnt, K, score(q, X + j * D, D, metric), j);
      for (int k = 0; k < K; ++k) {
        out_val[i * K + k] = k < cnt ? reported(vs[k], metric) : NAN;
        out_idx[i * K + k] = k < cnt ? js[k] : -1;
      }
    }
    free(vs);
    free(js);
  }
}

/* ---------------------------------------------------------------------- */
/* PartialReduce (Alg. 1): for every query i and row j, compute the score  */
/* y_ij, take its bin l = j mod L, and keep the bin's best score and index */
/* (strict '>' while j ascends, so ties keep the smaller j).               */
/* V[M*L] holds internal (larger-is-better) scores, A[M*L] indices; a bin  */
/* with no rows (only when L > N) keeps V = -inf and A = -1.               */
/* ---------------------------------------------------------------------- */
void orc_partial_reduce(const double *Q, int64_t M, const double *X, int64_t N, int D,
                        int metric, int64_t L, double *V, int64_t *A) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < M; ++i) {
    double *v = V + i * L;
    int64_t *a = A + i * L;
    for (int64_t l = 0; l < L; ++l) {
      v[l] = -INFINITY;
      a[l] = -1;
    }
    const double *q = Q + i * D;
    for (int64_t j = 0; j < N; ++j) {
      double y = score(q, X + j * D, D, metric);
      int64_t l = j % L;
      if (y > v[l]) {
        v[l] = y;
        a[l] = j;
      }
    }
  }
}

/* ---------------------------------------------------------------------- */
/* PartialReduce with contiguous bins (Alg. 1 uses l = ShiftRight(j, W): a  */
/* bin is a run of consecutive rows). For an L that does not divide N the  */
/* runs are balanced: with q = N / L and r = N mod L, bin l holds rows     */
/* [l*q + min(l, r), (l+1)*q + min(l+1, r)), so the first r bins have one   */
/* row more. Same outputs and tie rule as orc_partial_reduce.              */
/* ---------------------------------------------------------------------- */
static int64_t contiguous_bin(int64_t j, int64_t N, int64_t L) {
  const int64_t q = N / L, r = N % L;
  const int64_t big = r * (q + 1); /* rows held by the first r bins */
  return j < big ? j / (q + 1) : r + (j - big) / q;
}

void orc_partial_reduce_contiguous(const double *Q, int64_t M, const double *X, int64_t N, int D,
                                   int metric, int64_t L, double *V, int64_t *A) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < M; ++i) {
    double *v = V + i * L;
    int64_t *a = A + i * L;
    for (int64_t l = 0; l < L; ++l) {
      v[l] = -INFINITY;
      a[l] = -1;
    }
    const double *q = Q + i * D;
    for (int64_t j = 0; j < N; ++j) {
      double y = score(q, X + j * D, D, metric);
      int64_t l = contiguous_bin(j, N, L);
      if (y > v[l]) {
        v[l] = y;
        a[l] = j;
      }
    }
  }
}

/* ---------------------------------------------------------------------- */
/* approx_max_k on a score matrix the caller already has (App. A.1: the   */
/* operator behind Alg. 1, applied to given scores). For every row i of S */
/* (M x N, row-major) and bin l, the largest S[i][j] over the columns j of */
/* bin l and that j: bins j mod L, or (contiguous != 0) the balanced runs  */
/* of consecutive columns above. Strict '>' while j ascends, so ties keep  */
/* the smaller j; an empty bin keeps V = -inf, A = -1.                    */
/* ---------------------------------------------------------------------- */
void orc_bin_max(const double *S, int64_t M, int64_t N, int64_t L, int contiguous, double *V,
                 int64_t *A) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < M; ++i) {
    double *v = V + i * L;
    int64_t *a = A + i * L;
    for (int64_t l = 0; l < L; ++l) {
      v[l] = -INFINITY;
      a[l] = -1;
    }
    for (int64_t j = 0; j < N; ++j) {
      const double y = S[i * N + j];
      const int64_t l = contiguous ? contiguous_bin(j, N, L) : j % L;
      if (y > v[l]) {
        v[l] = y;
        a[l] = j;
      }
    }
  }
}

/* ---------------------------------------------------------------------- */
/* ExactRescoring (Sec. 5): the top-K of the L (score, index) pairs of     */
/* each query, best first. Empty bins (A = -1) are skipped. Values stay in */
/* the internal orientation; indices -1 pad when fewer than K are valid.   */
/* ---------------------------------------------------------------------- */
void orc_topk_pairs(const double *V, const int64_t *A, int64_t M, int64_t L, int K,
                    double *out_val, int64_t *out_idx) {
#pragma omp parallel
  {
    double *vs = (double *)malloc(sizeof(double) * (size_t)K);
    int64_t *js = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
      int cnt = 0;
      for (int64_t l = 0; l < L; ++l)
        if (A[i * L + l] >= 0) insert_sorted(vs, js, &cnt, K, V[i * L + l], A[i * L + l]);
      for (int k = 0; k < K; ++k) {
        out_val[i * K + k] = k < cnt ? vs[k] : NAN;
        out_idx[i * K + k] = k < cnt ? js[k] : -1;
      }
    }
    free(vs);
    free(js);
  }
}

/* ---------------------------------------------------------------------- */
/* Re-rank: score the Kp candidate rows of each query (cand[M*Kp], -1 =    */
/* none) with the rows given here and keep the best K, best first, as      */
/* reported values.                                                        */
/* ---------------------------------------------------------------------- */
void orc_rerank(const double *Q, int64_t M, const double *X, int64_t N, int D, int metric,
                const int64_t *cand, int Kp, int K, double *out_val, int64_t *out_idx) {
#pragma omp parallel
  {
    double *vs = (double *)malloc(sizeof(double) * (size_t)K);
    int64_t *js = (int64_t *)malloc(sizeof(int64_t) * (size_t)K);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < M; ++i) {
      int cnt = 0;
      for (int c = 0; c < Kp; ++c) {
        int64_t j = cand[i * Kp + c];
        if (j < 0 || j >= N) continue;
        insert_sorted(vs, js, &cnt, K, score(Q + i * D, X + j * D, D, metric), j);
      }
      for (int k = 0; k < K; ++k) {
        out_val[i * K + k] = k < cnt ? reported(vs[k], metric) : NAN;
        out_idx[i * K + k] = k < cnt ? js[k] : -1;
      }
    }
    free(vs);
    free(js);
  }
}

/* ---------------------------------------------------------------------- */
/* Gradient of  sum_{i,k} g[i,k] * f(q_i, x_{idx[i,k]})  where f is the    */
/* reported value of the metric; indices are constants.                    */
/*   IP : f = <q,x>            df/dq = x,                df/dx = q         */
/*   L2 : f = ||q-x||^2        df/dq = 2(q-x),           df/dx = 2(x-q)    */
/*   COS: f = <q,x>/(|q||x|)   df/dq = x/(|q||x|) - f q/|q|^2, and the     */
/*        mirror image for x.                                              */
/* dQ (M*D) is overwritten, dX (N*D) is accumulated into; either may be    */
/* NULL. Accumulation into dX runs in (i, k) order.                        */
/* ---------------------------------------------------------------------- */
void orc_grad(const double *Q, int64_t M, const double *X, int64_t N, int D, int metric,
              const int64_t *idx, int K, const double *g, double *dQ, double *dX) {
  double *tq = (double *)malloc(sizeof(double) * (size_t)D);
  double *tx = (double *)malloc(sizeof(double) * (size_t)D);
  if (dQ) memset(dQ, 0, sizeof(double) * (size_t)(M * D));
  for (int64_t i = 0; i < M; ++i) {
    const double *q = Q + i * D;
    for (int k = 0; k < K; ++k) {
      int64_t j = idx[i * K + k];
      if (j < 0 || j >= N) continue;
      const double *x = X + j * D;
      double w = g[i * K + k];
      if (metric == ORC_IP) {
        for (int d = 0; d < D; ++d) {
          tq[d] = x[d];
          tx[d] = q[d];
        }
      } else if (metric == ORC_L2) {
        for (int d = 0; d < D; ++d) {
          tq[d] = 2.0 * (q[d] - x[d]);
          tx[d] = 2.0 * (x[d] - q[d]);
        }
      } else {
        double nq = sqrt(dot(q, q, D)), nx = sqrt(dot(x, x, D));
        if (nq == 0.0 || nx == 0.0) {
          for (int d = 0; d < D; ++d) tq[d] = tx[d] = 0.0;
        } else {
          double f = dot(q, x, D) / (nq * nx);
          for (int d = 0; d < D; ++d) {
            tq[d] = x[d] / (nq * nx) - f * q[d] / (nq * nq);
            tx[d] = q[d] / (nq * nx) - f * x[d] / (nx * nx);
          }
        }
      }
      for (int d = 0; d < D; ++d) {
        if (dQ) dQ[i * D + d] += w * tq[d];
        if (dX) dX[j * D + d] += w * tx[d];
      }
    }
  }
  free(tq);
  free(tx);
}

/* ---------------------------------------------------------------------- */
/* Input preparation the method needs before the contraction. These take  */
/* their decisions (a rounded code) in the precision stated, so that any  */
/* other implementation following the same definition agrees bit for bit. */
/* ---------------------------------------------------------------------- */

/* IEEE binary32 -> bfloat16, round to nearest, ties to even; returns the
 * rounded value. (bfloat16 = the top 16 bits of a binary32.) */
double orc_bf16_round(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (double)f; /* inf / nan pass */
  uint32_t keep = u >> 16, rest = u & 0xffffu;
  if (rest > 0x8000u || (rest == 0x8000u && (keep & 1u))) keep += 1u;
  uint32_t r = keep << 16;
  float out;
  memcpy(&out, &r, 4);
  return (double)out;
}

void orc_bf16_round_array(const float *x, int64_t n, double *out) {
  for (int64_t t = 0; t < n; ++t) out[t] = orc_bf16_round(x[t]);
}

/* OCP FP8 E4M3 ("e4m3fn"): 1 sign, 4 exponent bits (bias 7), 3 mantissa
 * bits, no infinities, largest finite 448, smallest normal 2^-6, subnormal
 * step 2^-9. Round to nearest even, saturating to +-448. */
double orc_e4m3_round(double v) {
  double a = fabs(v);
  if (a == 0.0) return v;
  double r;
  if (a >= 448.0) {
    r = 448.0;
  } else if (a < ldexp(1.0, -6)) {
    r = nearbyint(a / ldexp(1.0, -9)) * ldexp(1.0, -9); /* subnormal grid */
  } else {
    int e;
    frexp(a, &e); /* a = m * 2^e, m in [0.5, 1) -> leading bit at 2^(e-1) */
    double step = ldexp(1.0, (e - 1) - 3);
    r = nearbyint(a / step) * step;
    if (r > 448.0) r = 448.0;
  }
  return v < 0.0 ? -r : r;
}

/* Per-row E4M3 quantisation: scale s = max_d |x_d| / 448 (binary32
 * division), code = E4M3(x_d / s) with the division in binary32, dequantised
 * value = code * s (exact in binary64). A zero row uses s = 1. */
void orc_e4m3_rows(const float *x, int64_t rows, int D, double *out, float *scale) {
  for (int64_t r = 0; r < rows; ++r) {
    const float *xr = x + r * D;
    float mx = 0.0f;
    for (int d = 0; d < D; ++d) {
      float a = fabsf(xr[d]);
      if (a > mx) mx = a;
    }
    float s = mx > 0.0f ? mx / 448.0f : 1.0f;
    scale[r] = s;
    for (int d = 0; d < D; ++d) {
      float t = xr[d] / s;
      out[r * D + d] = orc_e4m3_round((double)t) * (double)s;
    }
  }
}

/* E4M3 quantisation with one given scale s for every value (the database-
 * wide scale: s = max |x| / 448 over the whole database, binary32 division,
 * computed by the caller): code = E4M3(x / s) with the division in binary32,
 * dequantised value = code * s (exact in binary64). */
void orc_e4m3_scaled(const float *x, int64_t n, float s, double *out) {
  for (int64_t t = 0; t < n; ++t) {
    float q = x[t] / s;
    out[t] = orc_e4m3_round((double)q) * (double)s;
  }
}

/* Cosine preparation (Sec. 2: cosine search = MIPS on l2-normalised rows):
 * n2 = sum_d x_d^2 accumulated in binary64 in index order, inv = 1/sqrt(n2),
 * y_d = binary32(x_d * inv). A zero row stays zero. */
void orc_normalize_rows(const float *x, int64_t rows, int D, float *y) {
  for (int64_t r = 0; r < rows; ++r) {
    const float *xr = x + r * D;
    double n2 = 0.0;
    for (int d = 0; d < D; ++d) {
      double t = (double)xr[d];
      double sq = t * t;
      n2 = n2 + sq;
    }
    if (n2 == 0.0) {
      for (int d = 0; d < D; ++d) y[r * D + d] = 0.0f;
      continue;
    }
    double inv = 1.0 / sqrt(n2);
    for (int d = 0; d < D; ++d) y[r * D + d] = (float)((double)xr[d] * inv);
  }
}

/* ---------------------------------------------------------------------- */
/* Thread count of the OpenMP loops over queries (timing runs only: results */
/* do not depend on it). Returns the previous maximum; n < 1 only reads it. */
/* ---------------------------------------------------------------------- */
int orc_set_threads(int n) {
  int prev = omp_get_max_threads();
  if (n > 0) omp_set_num_threads(n);
  return prev;
}
