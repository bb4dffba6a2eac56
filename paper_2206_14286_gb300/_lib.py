"""ctypes declarations of the C ABI in include/tpuknn.h.

The library is loaded from ``_build/libtpuknn.so`` (built by ``build.py``).
There is no fallback: a missing or unloadable library raises.
"""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtpuknn.so")

KNN_OK, KNN_EINVAL, KNN_ENOMEM, KNN_ECUDA, KNN_ETIMEOUT, KNN_EUNSUPPORTED = range(6)
METRIC = {"ip": 0, "l2": 1, "cos": 2}
DTYPE = {"f32": 0, "bf16": 1, "e4m3": 2, "e4m3t": 3}
BINS = {"mod": 0, "contiguous": 1}
RATE = {"minmax": 0, "ffma": 1}
STATIC_WORKSPACE_BYTES = 16 << 20  # KNN_STATIC_WORKSPACE_BYTES

# every function the header declares, with (restype, argtypes)
P, I32, I64, SZ, DBL = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_double
SIGNATURES = {
    "knn_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "knn_last_cuda_error": (ctypes.c_int, []),
    "knn_dtype_bytes": (I32, [I32]),
    "knn_row_pitch": (I32, [I32]),
    "knn_plan_bins": (I64, [I64, I32, DBL, I32]),
    "knn_prepare": (ctypes.c_int, [P, I64, I32, I32, I32, P, P, P, P, P]),
    "knn_search": (ctypes.c_int, [P, P, P, P, I64, I32, I32, I32, P, I64, I32, I64, I32, DBL,
                                  I32, P, P, P, SZ, P]),
    "knn_search_workspace": (SZ, [I64, I32, I32, I32, I64, I32, I64, I32, DBL, I32]),
    "knn_search_host": (ctypes.c_int, [P, P, P, P, I64, I32, I32, I32, P, I64, I32, I64, I32,
                                       DBL, I32, P, P, P, SZ, P]),
    "knn_search_host_async": (ctypes.c_int, [P, P, P, P, I64, I32, I32, I32, P, I64, I32, I64,
                                             I32, DBL, I32, P, P, P, SZ, P]),
    "knn_search_host_workspace": (SZ, [I64, I32, I32, I32, I64, I32, I64, I32, DBL, I32]),
    "knn_search_static": (ctypes.c_int, [P, P, P, P, I64, I32, I32, I32, P, I64, I32, I64, I32,
                                         DBL, I32, P, P, P]),
    "knn_partial_reduce": (ctypes.c_int, [P, P, P, I64, I32, I32, I32, P, I64, I64, I32, P, P, P,
                                          SZ, P]),
    "knn_partial_reduce_workspace": (SZ, [I64, I32, I32, I32, I64, I64, I32]),
    "knn_search_exact": (ctypes.c_int, [P, P, P, P, I64, I32, I32, I32, P, I64, I32, P, P, P, SZ,
                                        P]),
    "knn_search_exact_workspace": (SZ, [I64, I32, I32, I32, I64, I32]),
    "knn_approx_max_k": (ctypes.c_int, [P, I32, I64, I64, I32, I64, I64, DBL, I32, I32, I32, P, P,
                                        P, SZ, P]),
    "knn_approx_max_k_workspace": (SZ, [I64, I64, I32, I64, I64, DBL, I32]),
    "knn_backward": (ctypes.c_int, [P, P, P, I64, I32, I32, I32, P, I64, I32, P, P, P, P, I32,
                                    I32, P, SZ, P]),
    "knn_backward_workspace": (SZ, [I64, I32, I64, I32, I32]),
    "knn_shard_partial_reduce_workspace": (SZ, [I64, I64, I64, I32, I32, I32, I64, I64]),
    "knn_shard_partial_reduce": (ctypes.c_int, [P, P, P, I64, I64, I64, I32, I32, I32, P, I64, I64,
                                                P, P, SZ, P]),
    "knn_rescore_count": (I32, [I32, I32, I64]),
    "knn_shard_rescore_workspace": (SZ, [I64, I64, I32, I32, I32, I32]),
    "knn_shard_rescore": (ctypes.c_int, [P, I64, I64, I32, I32, P, I32, I32, P, I64, I64, P, P, SZ,
                                         P]),
    "knn_shard_finish_workspace": (SZ, [I64, I32, I32]),
    "knn_shard_finish": (ctypes.c_int, [P, I64, I32, I32, I32, P, P, P, SZ, P]),
    "knn_db_create": (ctypes.c_int, [P, I64, I32, I32, I32, I32, P, P]),
    "knn_db_destroy": (ctypes.c_int, [P]),
    "knn_db_info": (ctypes.c_int, [P, P, P, P, P]),
    "knn_db_search": (ctypes.c_int, [P, P, I64, I32, I64, I32, DBL, I32, P, P, P, SZ, P]),
    "knn_db_search_workspace": (SZ, [P, I64, I32, I64, I32, DBL, I32]),
    "knn_measure_rate": (ctypes.c_int, [I32, I64, P, P, P]),
    "knn_set_wait_limit_ns": (ctypes.c_int, [ctypes.c_uint64]),
    "knn_sync_status": (ctypes.c_int, []),
    "knn_profile_enable": (ctypes.c_int, [I32]),
    "knn_profile_read": (ctypes.c_int, [I32, P, P]),
}

_lib = None


class KnnError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = get().knn_status_string(status).decode() if _lib else str(status)
        if status == KNN_ECUDA:
            msg += " (cudaError %d)" % get().knn_last_cuda_error()
        super().__init__("%s: %s" % (what, msg) if what else msg)


def get():
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtpuknn.so is not built (%s); run "
                               "paper_2206_14286_gb300.build.build()" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status, what=""):
    if status != KNN_OK:
        raise KnnError(status, what)
