"""The C ABI library builds, loads and exports what include/tpuknn.h declares;
host-only entry points (planner, pitch, argument checks) behave as stated.
No GPU is needed: no call here launches a kernel."""
import ctypes
import os
import re

import pytest

from paper_2206_14286_gb300 import build as B
from paper_2206_14286_gb300 import _lib
from oracle import recall as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return _lib.get()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tpuknn.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(knn_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, "binding lacks " + n


def test_binding_declares_only_header_functions():
    assert set(_lib.SIGNATURES) <= set(declared_functions())


@pytest.mark.parametrize("N,K,r", [(16384, 10, 0.95), (10 ** 6, 10, 0.95), (10 ** 7, 100, 0.95),
                                   (10 ** 6, 32, 0.95), (1000, 2, 0.5), (10 ** 6, 10, 0.99)])
def test_plan_bins_matches_oracle_eq14(lib, N, K, r):
    assert lib.knn_plan_bins(N, K, r, 1) == min(R.min_bins(K, r), N)


def test_plan_bins_rounding_and_edges(lib):
    assert lib.knn_plan_bins(10 ** 6, 10, 0.95, 128) == 256
    assert lib.knn_plan_bins(10 ** 7, 100, 0.95, 128) == 2048
    assert lib.knn_plan_bins(100, 10, 0.95, 1) == 100        # clamped to N
    assert lib.knn_plan_bins(1000, 1, 0.99, 1) == 1          # K = 1
    assert lib.knn_plan_bins(1000, 1, 0.99, 128) == 128
    for bad in [(0, 1, 0.9, 1), (10, 0, 0.9, 1), (10, 11, 0.9, 1), (10, 2, 1.0, 1),
                (10, 2, 0.0, 1)]:
        assert lib.knn_plan_bins(*bad) == -1


def test_pitch_and_dtype_bytes(lib):
    assert [lib.knn_row_pitch(d) for d in (1, 16, 17, 96, 100, 128)] == [16, 16, 32, 96, 112, 128]
    assert lib.knn_row_pitch(0) == -1
    assert [lib.knn_dtype_bytes(t) for t in (0, 1, 2, 7)] == [4, 2, 1, 0]


def test_status_strings(lib):
    for s in range(6):
        assert lib.knn_status_string(s)


def test_invalid_arguments_rejected_before_any_launch(lib):
    f = lib.knn_search
    # N = 0, K > N, bad metric, bad dtype, K > L: all EINVAL without touching a device
    base = dict(db=None, sc=None, hn=None, f32=None, N=100, D=8, dt=0, me=0, q=None, M=4, K=3,
                L=10, bm=0, r=0.9, rr=1, ov=None, oi=None, ws=None, wsb=0, st=None)

    def call(**kw):
        a = dict(base, **kw)
        return f(a["db"], a["sc"], a["hn"], a["f32"], a["N"], a["D"], a["dt"], a["me"], a["q"],
                 a["M"], a["K"], a["L"], a["bm"], a["r"], a["rr"], a["ov"], a["oi"], a["ws"],
                 a["wsb"], a["st"])

    assert call(N=0) == _lib.KNN_EINVAL
    assert call(K=101) == _lib.KNN_EINVAL
    assert call(me=5) == _lib.KNN_EINVAL
    assert call(dt=9) == _lib.KNN_EINVAL
    assert call(K=20, L=10) == _lib.KNN_EINVAL
    assert call(L=101) == _lib.KNN_EINVAL
    assert call(D=5000) == _lib.KNN_EUNSUPPORTED
    assert call() == _lib.KNN_EINVAL           # null pointers
    assert call(M=0) == _lib.KNN_OK            # empty query set is a no-op
    assert call(bm=7) == _lib.KNN_EINVAL       # unknown bin map
    assert call(bm=1) == _lib.KNN_EUNSUPPORTED  # contiguous bins: BF16 only
    # workspace queries return 0 for invalid requests
    assert lib.knn_search_workspace(0, 8, 0, 0, 4, 3, 10, 0, 0.9, 1) == 0
    assert lib.knn_search_exact_workspace(100, 8, 0, 0, 4, 101) == 0
    assert lib.knn_partial_reduce_workspace(100, 8, 0, 0, 4, 101, 0) == 0


def test_workspace_grows_with_queries(lib):
    for bm in (0, 1):
        a = lib.knn_search_workspace(10 ** 6, 128, 1, 1, 1024, 10, 256, bm, 0.95, 2)
        b = lib.knn_search_workspace(10 ** 6, 128, 1, 1, 2048, 10, 256, bm, 0.95, 2)
        assert 0 < a < b
        assert lib.knn_search_host_workspace(10 ** 6, 128, 1, 1, 1024, 10, 256, bm, 0.95, 2) > a


def test_approx_max_k_argument_checks_need_no_device(lib):
    f = lib.knn_approx_max_k
    # (scores, dtype, M, N, K, L, planning, r, bins, is_min, agg, val, idx, ws, wsb, stream)
    base = [None, 0, 4, 100, 5, 10, 0, 0.9, 0, 0, 1, None, None, None, 0, None]

    def call(**kw):
        a = list(base)
        pos = {"dt": 1, "M": 2, "N": 3, "K": 4, "L": 5, "bins": 8, "agg": 10}
        for k, v in kw.items():
            a[pos[k]] = v
        return f(*a)

    assert call(M=0) == _lib.KNN_OK
    assert call(N=0) == _lib.KNN_EINVAL
    assert call(L=101) == _lib.KNN_EINVAL
    assert call(K=11) == _lib.KNN_EINVAL                 # K > L with aggregation
    assert call(K=11, agg=0) == _lib.KNN_EINVAL          # still NULL pointers
    assert call(dt=2) == _lib.KNN_EINVAL                 # E4M3 scores are not accepted
    assert call(bins=5) == _lib.KNN_EINVAL
    assert call() == _lib.KNN_EINVAL                     # NULL pointers
    assert lib.knn_approx_max_k_workspace(4, 100, 5, 10, 0, 0.9, 1) >= 4 * 10 * 8 + 4 * 5 * 8
    assert lib.knn_approx_max_k_workspace(4, 100, 5, 0, 0, 0.9, 0) > 0   # L planned
    assert lib.knn_approx_max_k_workspace(4, 100, 0, 0, 0, 0.9, 0) == 0  # no K to plan L


def test_db_handle_rejects_bad_arguments_without_a_device(lib):
    import ctypes
    h = ctypes.c_void_p(123)
    f = lib.knn_db_create
    # (x, N, D, metric, dtype, keep_f32, stream, out)
    assert f(None, 100, 8, 0, 1, 1, None, ctypes.byref(h)) == _lib.KNN_EINVAL
    assert h.value is None                               # *out cleared on error
    assert f(None, 100, 8, 0, 1, 1, None, None) == _lib.KNN_EINVAL
    assert f(8, 0, 8, 0, 1, 1, None, ctypes.byref(h)) == _lib.KNN_EINVAL      # N = 0
    assert f(8, 100, 8, 7, 1, 1, None, ctypes.byref(h)) == _lib.KNN_EINVAL    # metric
    assert f(8, 100, 8, 0, 9, 1, None, ctypes.byref(h)) == _lib.KNN_EINVAL    # dtype
    assert f(6, 100, 8, 0, 1, 1, None, ctypes.byref(h)) == _lib.KNN_EINVAL    # misaligned x
    assert f(8, 100, 5000, 0, 1, 1, None, ctypes.byref(h)) == _lib.KNN_EUNSUPPORTED
    assert lib.knn_db_destroy(None) == _lib.KNN_EINVAL
    assert lib.knn_db_info(None, None, None, None, None) == _lib.KNN_EINVAL
    assert lib.knn_db_search_workspace(None, 10, 5, 64, 0, 0.95, 2) == 0
    assert lib.knn_db_search(None, None, 10, 5, 64, 0, 0.95, 2, None, None, None, 0,
                             None) == _lib.KNN_EINVAL


def test_shard_calls_reject_bad_layouts(lib):
    """Host-side checks of the sharded calls' layout rules (no launch)."""
    f = lib.knn_shard_partial_reduce_workspace
    # (n_local, row0, N_global, D, dtype, metric, M, L)
    assert f(1000, 0, 3000, 64, 1, 1, 10, 128) > 0
    assert f(1000, 100, 3000, 64, 1, 1, 10, 128) == 0       # row0 not a multiple of L
    assert f(100, 0, 3000, 64, 1, 1, 10, 128) == 0          # L > n_local
    assert f(1000, 2560, 3000, 64, 1, 1, 10, 128) == 0      # past N_global
    assert lib.knn_rescore_count(10, 2, 128) == 20
    assert lib.knn_rescore_count(10, 2, 15) == 15
    assert lib.knn_rescore_count(11, 1, 10) == -1


def test_host_entries_reject_bad_arguments_without_a_device(lib):
    """knn_search_host and knn_search_host_async check their arguments before
    any copy: invalid sizes, null host buffers, a missing or small workspace."""
    for f in (lib.knn_search_host, lib.knn_search_host_async):
        base = [None, None, None, None, 100, 8, 0, 0, None, 4, 3, 10, 0, 0.9, 1, None, None,
                None, 0, None]

        def call(**kw):
            a = list(base)
            pos = {"N": 4, "K": 10, "L": 11, "q": 8, "ov": 15, "oi": 16, "ws": 17, "wsb": 18,
                   "M": 9}
            for k, v in kw.items():
                a[pos[k]] = v
            return f(*a)

        assert call(N=0) == _lib.KNN_EINVAL
        assert call(K=20) == _lib.KNN_EINVAL          # K > L
        assert call(M=0) == _lib.KNN_OK               # empty query set
        assert call() == _lib.KNN_EINVAL              # null host buffers
        buf = ctypes.create_string_buffer(64)
        p = ctypes.addressof(buf)
        assert call(q=p, ov=p, oi=p) == _lib.KNN_EINVAL          # no workspace
        assert call(q=p, ov=p, oi=p, ws=4096, wsb=16) == _lib.KNN_ENOMEM   # too small


@pytest.mark.parametrize("N,M,K", [(1, 1, 1), (1000, 7, 3), (1_000_000, 4096, 32), (50, 100, 10)])
def test_backward_workspace_size(lib, N, M, K):
    """A list head per row, a link per entry, the touched-row list (at most
    min(N, M K) rows) and its count, each rounded up to 256 bytes; the same
    for both modes."""
    def r(b):
        return (b + 255) // 256 * 256
    E = M * K
    want = r(4 * N) + r(4 * E) + r(4 * min(N, E)) + 256
    for det in (0, 1):
        assert lib.knn_backward_workspace(N, 16, M, K, det) == want


def test_e4m3_database_scale_dtype(lib):
    """KNN_E4M3_T stores one byte per element like KNN_E4M3."""
    assert lib.knn_dtype_bytes(_lib.DTYPE["e4m3t"]) == 1 == lib.knn_dtype_bytes(_lib.DTYPE["e4m3"])
