"""ctypes front end of the FP64 oracle in ``knn_oracle.c``.

Test infrastructure only (see the package docstring). Arrays are converted
to C-contiguous float64 / int64 / float32 as each routine requires; results
come back as numpy arrays.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

IP, L2, COS = 0, 1, 2
METRICS = {"ip": IP, "l2": L2, "cos": COS}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "knn_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liborc.so")
_lock = threading.Lock()
_lib = None


def lib_path():
    return _LIB


def build(force=False):
    """Compile knn_oracle.c with gcc (OpenMP, FP contraction off)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int
            lib.orc_exact_topk.argtypes = [P, i64, P, i64, i32, i32, i32, P, P]
            lib.orc_partial_reduce.argtypes = [P, i64, P, i64, i32, i32, i64, P, P]
            lib.orc_partial_reduce_contiguous.argtypes = [P, i64, P, i64, i32, i32, i64, P, P]
            lib.orc_topk_pairs.argtypes = [P, P, i64, i64, i32, P, P]
            lib.orc_bin_max.argtypes = [P, i64, i64, i64, i32, P, P]
            lib.orc_rerank.argtypes = [P, i64, P, i64, i32, i32, P, i32, i32, P, P]
            lib.orc_grad.argtypes = [P, i64, P, i64, i32, i32, P, i32, P, P, P]
            lib.orc_score.argtypes = [P, P, i32, i32]
            lib.orc_score.restype = ctypes.c_double
            lib.orc_bf16_round_array.argtypes = [P, i64, P]
            lib.orc_e4m3_rows.argtypes = [P, i64, i32, P, P]
            lib.orc_e4m3_scaled.argtypes = [P, i64, ctypes.c_float, P]
            lib.orc_normalize_rows.argtypes = [P, i64, i32, P]
            lib.orc_e4m3_round.argtypes = [ctypes.c_double]
            lib.orc_e4m3_round.restype = ctypes.c_double
            lib.orc_set_threads.argtypes = [i32]
            lib.orc_set_threads.restype = i32
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _metric(m):
    return METRICS[m] if isinstance(m, str) else int(m)


def score(q, x, metric):
    """Larger-is-better score of one row pair (IP, -||q-x||^2, or cosine)."""
    q, x = _f64(q), _f64(x)
    return _load().orc_score(_p(q), _p(x), q.shape[0], _metric(metric))


def exact_topk(Q, X, K, metric):
    """Exact K-NN (Eq. 1-2): (values, indices), each M x K, best first.

    Values are reported forms: IP -> <q,x>, L2 -> ||q-x||^2, COS -> cosine.
    """
    Q, X = _f64(Q), _f64(X)
    M, D = Q.shape
    N = X.shape[0]
    val = np.empty((M, K), np.float64)
    idx = np.empty((M, K), np.int64)
    _load().orc_exact_topk(_p(Q), M, _p(X), N, D, _metric(metric), K, _p(val), _p(idx))
    return val, idx


def partial_reduce(Q, X, L, metric, bins="mod"):
    """PartialReduce (Alg. 1): (V, A), each M x L.

    bins="mod": bin l = j mod L. bins="contiguous": bin l is the l-th of L
    balanced runs of consecutive rows (Alg. 1's ShiftRight for any L).
    V holds larger-is-better scores (L2: -||q-x||^2); empty bins have
    V = -inf, A = -1.
    """
    Q, X = _f64(Q), _f64(X)
    M, D = Q.shape
    N = X.shape[0]
    V = np.empty((M, L), np.float64)
    A = np.empty((M, L), np.int64)
    fn = _load().orc_partial_reduce if bins == "mod" else _load().orc_partial_reduce_contiguous
    fn(_p(Q), M, _p(X), N, D, _metric(metric), L, _p(V), _p(A))
    return V, A


def topk_pairs(V, A, K):
    """ExactRescoring (Sec. 5): the best K (value, index) pairs per row."""
    V, A = _f64(V), _i64(A)
    M, L = V.shape
    val = np.empty((M, K), np.float64)
    idx = np.empty((M, K), np.int64)
    _load().orc_topk_pairs(_p(V), _p(A), M, L, K, _p(val), _p(idx))
    return val, idx


def bin_max(S, L, bins="mod"):
    """Per row of the score matrix S (M x N) and bin: the largest score and its
    column (App. A.1 applied to given scores). (V, A), each M x L; an empty
    bin has V = -inf, A = -1."""
    S = _f64(S)
    M, N = S.shape
    V = np.empty((M, L), np.float64)
    A = np.empty((M, L), np.int64)
    _load().orc_bin_max(_p(S), M, N, L, 0 if bins == "mod" else 1, _p(V), _p(A))
    return V, A


def approx_max_k(S, K, L, bins="mod", is_min=False, aggregate_to_topk=True):
    """The paper's approx_max_k / approx_min_k operator on a score matrix.

    is_min: the K smallest (approx_min_k), done as the K largest of -S.
    aggregate_to_topk=False returns the L bin winners (V, A), M x L, in bin
    order; True returns the best K of them, best first. Values keep the sign
    of S."""
    Sx = -_f64(S) if is_min else _f64(S)
    V, A = bin_max(Sx, L, bins)
    if aggregate_to_topk:
        V, A = topk_pairs(V, A, K)
    return (-V if is_min else V), A


def _report(v, metric):
    return -v if _metric(metric) == L2 else v


def binwise_topk(Q, X, K, L, metric, bins="mod"):
    """The approximate method end to end: PartialReduce then ExactRescoring.

    Returns reported values and indices, M x K, best first.
    """
    V, A = partial_reduce(Q, X, L, metric, bins)
    val, idx = topk_pairs(V, A, K)
    return _report(val, metric), idx


def rerank(Q, X, cand, K, metric):
    """Score the candidate rows ``cand`` (M x Kp, -1 = none) and keep K."""
    Q, X, cand = _f64(Q), _f64(X), _i64(cand)
    M, D = Q.shape
    N = X.shape[0]
    Kp = cand.shape[1]
    val = np.empty((M, K), np.float64)
    idx = np.empty((M, K), np.int64)
    _load().orc_rerank(_p(Q), M, _p(X), N, D, _metric(metric), _p(cand), Kp, K,
                       _p(val), _p(idx))
    return val, idx


def grad(Q, X, idx, g, metric, want_dq=True, want_dx=True):
    """Gradient of sum g[i,k] * value(q_i, x_idx[i,k]) w.r.t. Q and X."""
    Q, X, idx, g = _f64(Q), _f64(X), _i64(idx), _f64(g)
    M, D = Q.shape
    N = X.shape[0]
    K = idx.shape[1]
    dQ = np.zeros((M, D), np.float64) if want_dq else None
    dX = np.zeros((N, D), np.float64) if want_dx else None
    _load().orc_grad(_p(Q), M, _p(X), N, D, _metric(metric), _p(idx), K, _p(g),
                     _p(dQ) if dQ is not None else None,
                     _p(dX) if dX is not None else None)
    return dQ, dX


def bf16_round(x):
    """Round binary32 values to bfloat16 (nearest, ties to even), as float64."""
    x = _f32(x)
    out = np.empty(x.shape, np.float64)
    _load().orc_bf16_round_array(_p(x), x.size, _p(out))
    return out


def e4m3_rows(x):
    """Per-row E4M3 quantisation: (dequantised values float64, scales float32)."""
    x = _f32(x)
    rows, D = x.shape
    out = np.empty((rows, D), np.float64)
    sc = np.empty((rows,), np.float32)
    _load().orc_e4m3_rows(_p(x), rows, D, _p(out), _p(sc))
    return out, sc


def e4m3_tensor_scale(x):
    """The database-wide E4M3 scale: max |x| over all values / 448 in binary32
    (1 for an all-zero database)."""
    mx = np.float32(np.abs(_f32(x)).max()) if np.size(x) else np.float32(0.0)
    return np.float32(mx / np.float32(448.0)) if mx > 0 else np.float32(1.0)


def e4m3_scaled(x, s):
    """E4M3 quantisation of every value with the one scale s: dequantised
    values (float64), code = E4M3(x / s) with the division in binary32."""
    x = _f32(x)
    out = np.empty(x.shape, np.float64)
    _load().orc_e4m3_scaled(_p(x), x.size, ctypes.c_float(float(s)), _p(out))
    return out


def e4m3_tensor(x):
    """E4M3 with one database-wide scale: (dequantised values, the scale)."""
    s = e4m3_tensor_scale(x)
    return e4m3_scaled(x, s), s


def e4m3_round(v):
    """E4M3 rounding of one value (nearest even, saturating at 448)."""
    return _load().orc_e4m3_round(float(v))


def normalize_rows(x):
    """Cosine preparation: rows scaled to unit l2 norm, returned as float32."""
    x = _f32(x)
    rows, D = x.shape
    y = np.empty((rows, D), np.float32)
    _load().orc_normalize_rows(_p(x), rows, D, _p(y))
    return y


def set_threads(n):
    """Threads of the oracle's OpenMP loops over queries (for timing runs;
    results do not depend on it). Returns the previous count; n < 1 only
    reads it."""
    return _load().orc_set_threads(int(n))
