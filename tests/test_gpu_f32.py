"""Parity of the FP32 CUDA path (SIMT PartialReduce, ExactRescoring, re-rank,
exact search, backward) and of the row preparation against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2206_14286_gb300 import synth
from paper_2206_14286_gb300 import search as S
from tests import parity as PT
from tests.gpu_util import db, dev, host, ensure_built

pytestmark = pytest.mark.gpu
METRICS = ["ip", "l2", "cos"]


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def inputs(N, M, D, seed=0, scale=1.0):
    g = rng(seed)
    X = (g.standard_normal((N, D)) * scale).astype(np.float32)
    Q = (g.standard_normal((M, D)) * scale).astype(np.float32)
    return X, Q


def prepared_f32(A, metric):
    """The FP32 rows the kernel sees (cosine: unit rows by the oracle's rule)."""
    return oracle.normalize_rows(A) if metric == "cos" else A.astype(np.float32)


# ----------------------------------------------------------------------------
# Row preparation (bit-exact where a rounded code is decided)
# ----------------------------------------------------------------------------
def test_prepare_f32_cos_bits():
    X, _ = inputs(777, 0, 45, seed=1, scale=3.0)
    X[5] = 0.0
    d = db(X, "cos", "f32")
    ref = oracle.normalize_rows(X)
    lp = d.lp.view(torch.float32).reshape(777, d.pitch).cpu().numpy()
    np.testing.assert_array_equal(lp[:, :45], ref)
    assert (lp[:, 45:] == 0).all()
    np.testing.assert_array_equal(d.f32.cpu().numpy(), ref)


@pytest.mark.parametrize("metric", ["ip", "l2", "cos"])
def test_prepare_bf16_bits(metric):
    X, _ = inputs(1000, 0, 100, seed=2, scale=2.0)
    d = db(X, metric, "bf16")
    src = oracle.normalize_rows(X) if metric == "cos" else X
    ref = oracle.bf16_round(src)
    lp = d.lp.view(torch.bfloat16).reshape(1000, d.pitch).float().cpu().numpy()
    np.testing.assert_array_equal(lp[:, :100].astype(np.float64), ref)
    assert (lp[:, 100:] == 0).all()
    if metric == "l2":
        np.testing.assert_allclose(d.hnorm.cpu().numpy(), 0.5 * (ref * ref).sum(1), rtol=1e-6)


@pytest.mark.parametrize("metric", ["ip", "l2", "cos"])
def test_prepare_e4m3_bits(metric):
    X, _ = inputs(1000, 0, 96, seed=3, scale=2.0)
    X[7] = 0.0
    d = db(X, metric, "e4m3")
    src = oracle.normalize_rows(X) if metric == "cos" else X
    ref, sc = oracle.e4m3_rows(src)
    np.testing.assert_array_equal(d.scale.cpu().numpy(), sc)
    codes = d.lp.view(torch.float8_e4m3fn).reshape(1000, d.pitch).float().cpu().numpy()
    deq = codes[:, :96].astype(np.float64) * sc[:, None].astype(np.float64)
    np.testing.assert_array_equal(deq, ref)
    if metric == "l2":
        np.testing.assert_allclose(d.hnorm.cpu().numpy(), 0.5 * (ref * ref).sum(1), rtol=1e-6)


@pytest.mark.parametrize("metric", ["ip", "l2", "cos"])
@pytest.mark.parametrize("rows,D", [(1000, 96), (70001, 40), (1, 16)])
def test_prepare_e4m3_tensor_bits(metric, rows, D):
    """One database-wide scale: every row's scale is max |y| / 448 over all
    rows (y the unit row for COS), codes E4M3(y / s), bit for bit."""
    X, _ = inputs(rows, 0, D, seed=rows + D, scale=2.0)
    X[:: max(1, rows // 3)] *= 1e-3      # rows far below the largest
    if rows > 7:
        X[7] = 0.0
    d = db(X, metric, "e4m3t")
    src = oracle.normalize_rows(X) if metric == "cos" else X
    ref, s = oracle.e4m3_tensor(src)
    assert (d.scale.cpu().numpy() == s).all()
    codes = d.lp.view(torch.float8_e4m3fn).reshape(rows, d.pitch).float().cpu().numpy()
    assert (codes[:, D:] == 0).all()
    np.testing.assert_array_equal(codes[:, :D].astype(np.float64) * np.float64(s), ref)
    if metric == "l2":
        np.testing.assert_allclose(d.hnorm.cpu().numpy(), 0.5 * (ref * ref).sum(1), rtol=1e-6)


# ----------------------------------------------------------------------------
# PartialReduce (Alg. 1) alone
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("L", [1, 5, 64, 100, 777, 3001])
def test_partial_reduce_f32(metric, L):
    N, M, D = 3001, 70, 72
    X, Q = inputs(N, M, D, seed=4)
    d = db(X, metric, "f32")
    V, A = d.partial_reduce(dev(Q), L)
    V, A = host(V).astype(np.float64), host(A)
    Xp, Qp = prepared_f32(X, metric), prepared_f32(Q, metric)
    Vo, Ao = oracle.partial_reduce(Qp, Xp, L, "ip" if metric == "cos" else metric)
    tol = PT.REL_F32 * PT.query_scale(Qp, Xp, metric)
    if metric == "l2":  # kernel reports <q,x> - |x|^2/2 = (|q|^2 - |q-x|^2) / 2
        Vo = (Vo + (Qp.astype(np.float64) ** 2).sum(1)[:, None]) / 2.0
    Sm = PT.score_matrix(Qp, Xp, "ip" if metric == "cos" else metric)
    best, second = PT.bin_best_second(Sm, L)
    decided = (best - second) > 2 * tol[:, None]
    assert (A >= 0).all()
    np.testing.assert_array_equal(A[decided], Ao[decided])
    assert np.all(np.abs(V - Vo) <= tol[:, None])
    # undecided bins still return a member of the bin within tolerance of its best
    assert np.all(A % L == np.arange(L)[None, :])
    assert decided.mean() > 0.95


# ----------------------------------------------------------------------------
# Search (PartialReduce + ExactRescoring + re-rank)
# ----------------------------------------------------------------------------
def run_and_check(X, Q, metric, K, L, rerank, dtype="f32"):
    d = db(X, metric, dtype)
    val, idx = d.search(dev(Q), K, L=L, rerank=rerank)
    gv, gi = host(val), host(idx)
    Xp, Qp = prepared_f32(X, metric), prepared_f32(Q, metric)
    om = "ip" if metric == "cos" else metric
    Kp = min(max(1, rerank) * K, L)
    V, A = oracle.partial_reduce(Qp, Xp, L, om)
    _, cand = oracle.topk_pairs(V, A, Kp)
    ov, oi = oracle.rerank(Qp, Xp, cand, K, om)
    Sm = PT.score_matrix(Qp, Xp, om)
    tol = PT.REL_F32 * PT.query_scale(Qp, Xp, metric)
    dec = PT.decided_mask(Sm, L, Kp, Sm, cand, K, tol)
    frac = PT.check_search(gv, gi, ov, oi, Sm, Sm, L, om, tol, dec)
    return frac, gi


@pytest.mark.parametrize("metric", METRICS)
def test_search_f32_small_ragged(metric):
    X, Q = inputs(5003, 77, 40, seed=5)
    for K, L, rr in [(10, 100, 1), (10, 100, 2), (7, 64, 3), (1, 1, 1), (16, 5003, 1), (3, 3, 1)]:
        frac, _ = run_and_check(X, Q, metric, K, L, rr)
        assert frac > 0.9, (K, L, rr, frac)


def test_search_f32_iid_16k_ip_k10_l1024():
    """The plain FP32 workload: N=16384 x D=128 i.i.d. N(0,1), M=64, IP, K=10, L=1024."""
    w = synth.workload("iid_ip_16k")
    frac, gi = run_and_check(w["X"], w["Q"], "ip", 10, 1024, 1)
    assert frac > 0.9
    # recall against the exact top-10 (FP64 oracle) meets the law of Sec. 5.1
    _, ei = oracle.exact_topk(w["Q"], w["X"], 10, "ip")
    rec = np.mean([len(set(gi[i]) & set(ei[i])) / 10 for i in range(64)])
    assert rec >= 0.95


@pytest.mark.parametrize("metric", METRICS)
def test_exact_search_f32(metric):
    X, Q = inputs(20000, 33, 24, seed=6)
    d = db(X, metric, "f32")
    val, idx = d.search_exact(dev(Q), 12)
    gv, gi = host(val), host(idx)
    Xp, Qp = prepared_f32(X, metric), prepared_f32(Q, metric)
    om = "ip" if metric == "cos" else metric
    ov, oi = oracle.exact_topk(Qp, Xp, 12, om)
    Sm = PT.score_matrix(Qp, Xp, om)
    tol = PT.REL_F32 * PT.query_scale(Qp, Xp, metric)
    N = X.shape[0]
    dec = PT.decided_mask(Sm, N, 12, Sm, oi, 12, tol)
    # the exact search is the L = N case of the bin-wise search
    assert PT.check_search(gv, gi, ov, oi, Sm, Sm, N, om, tol, dec) > 0.9
    v2, i2 = d.search(dev(Q), 12, L=N, rerank=1)
    np.testing.assert_array_equal(host(i2)[dec], gi[dec])


def test_exact_search_spans_several_chunks():
    X, Q = inputs(70001, 1100, 16, seed=7)  # chunk = 2^26 / 1100 rows -> two chunks
    d = db(X, "ip", "f32")
    _, gi = d.search_exact(dev(Q), 5)
    ov, oi = oracle.exact_topk(Q[:50], X, 5, "ip")
    Sm = PT.score_matrix(Q[:50], X, "ip")
    tol = PT.REL_F32 * PT.query_scale(Q[:50], X, "ip")
    dec = PT.decided_mask(Sm, 70001, 5, Sm, oi, 5, tol)
    np.testing.assert_array_equal(host(gi)[:50][dec], oi[dec])


def test_search_degenerate_cases():
    X, Q = inputs(130, 9, 3, seed=8)
    d = db(X, "ip", "f32")
    # empty query set
    v, i = d.search(dev(Q[:0]), 4, L=10)
    assert v.shape == (0, 4)
    # K = 1, L = 1: global argmax
    _, i = d.search(dev(Q), 1, L=1)
    np.testing.assert_array_equal(host(i)[:, 0], np.argmax(Q.astype(np.float64) @ X.T.astype(np.float64), 1))
    # N smaller than a tile, K = L = N
    d2 = db(X[:7], "l2", "f32")
    _, i = d2.search(dev(Q), 7, L=7)
    assert all(sorted(r) == list(range(7)) for r in host(i))
    # D = 1
    d3 = db(X[:, :1], "ip", "f32")
    _, i = d3.search(dev(Q[:, :1]), 2, L=130)
    S1 = Q[:, :1].astype(np.float64) @ X[:, :1].T.astype(np.float64)
    assert (host(i)[:, 0] == np.argmax(S1, 1)).mean() > 0.8
    S.sync_status()


def test_search_host_entry_matches_device_entry():
    X, Q = inputs(4000, 50, 32, seed=9)
    d = db(X, "l2", "f32")
    v1, i1 = d.search(dev(Q), 8, L=64)
    v2, i2 = d.search_host(torch.from_numpy(Q).pin_memory(), 8, L=64)
    np.testing.assert_array_equal(host(i1), i2.numpy())
    np.testing.assert_array_equal(host(v1), v2.numpy())


@pytest.mark.parametrize("dtype,metric", [("bf16", "l2"), ("f32", "ip")])
def test_async_host_search_on_two_streams_matches_the_synchronous_call(dtype, metric):
    """knn_search_host_async: three query batches, two streams in flight (a
    workspace slot and host outputs each, slot 0 used twice on stream 0),
    give bit for bit what the synchronous knn_search_host gives."""
    X, Q = inputs(30000, 300, 64, seed=97)
    d = db(X, metric, dtype)
    qs = [torch.from_numpy(np.ascontiguousarray(Q[k::3])).pin_memory() for k in range(3)]
    ref = [d.search_host(q, 10, L=256) for q in qs]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [(torch.full((100, 10), float("nan"), dtype=torch.float32).pin_memory(),
             torch.full((100, 10), -7, dtype=torch.int32).pin_memory()) for _ in range(3)]
    for k in range(3):
        d.search_host(qs[k], 10, L=256, stream=streams[k % 2], wait=False, slot=k % 2,
                      out=outs[k])
    for st in streams:
        st.synchronize()
    S.sync_status()
    for (v, i), (rv, ri) in zip(outs, ref):
        assert torch.equal(i, ri)
        assert torch.equal(v.view(torch.int32), rv.view(torch.int32))


@pytest.mark.parametrize("dtype,metric", [("bf16", "l2"), ("e4m3", "cos")])
def test_searches_in_flight_on_two_streams_match_sequential_ones(dtype, metric):
    """Device-buffer searches with two in flight on two streams (a workspace
    slot each, as the bench's timed loop runs them) give bit for bit the
    results of the same searches one after another."""
    X, Q = inputs(40000, 600, 96, seed=98)
    d = db(X, metric, dtype)
    qs = [dev(np.ascontiguousarray(Q[k::4])) for k in range(4)]
    ref = [d.search(q, 16, L=512) for q in qs]
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    cur = torch.cuda.current_stream()
    for st in streams:
        st.wait_stream(cur)
    outs = []
    for k, q in enumerate(qs):
        st = streams[k % 2]
        with torch.cuda.stream(st):
            v = torch.full((150, 16), float("nan"), device="cuda")
            i = torch.full((150, 16), -7, dtype=torch.int32, device="cuda")
        outs.append(d.search(q, 16, L=512, out=(v, i), stream=st, slot=k % 2))
    for st in streams:
        cur.wait_stream(st)
    torch.cuda.synchronize()
    S.sync_status()
    for (v, i), (rv, ri) in zip(outs, ref):
        assert torch.equal(i, ri)
        assert torch.equal(v.view(torch.int32), rv.view(torch.int32))


def test_recall_plan_and_invalid_calls():
    ensure_built()
    assert S.plan_bins(10 ** 6, 10, 0.95) == 176
    X, Q = inputs(100, 4, 8, seed=10)
    d = db(X, "ip", "f32")
    with pytest.raises(Exception):
        d.search(dev(Q), 20, L=10)      # K > L
    with pytest.raises(Exception):
        d.search(dev(Q), 5, L=101)      # L > N


# ----------------------------------------------------------------------------
# Backward
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("metric", METRICS)
def test_backward_f32_matches_oracle(metric):
    g = rng(11)
    N, M, D, K = 500, 40, 24, 6
    X, Q = inputs(N, M, D, seed=11)
    idx = np.stack([g.permutation(N)[:K] for _ in range(M)]).astype(np.int32)
    idx[3, :] = idx[2, :]            # rows selected by several queries
    idx[5, 2] = -1                   # a skipped slot
    w = g.standard_normal((M, K)).astype(np.float32)
    d = db(X, metric, "f32")
    xf = dev(X)
    # atomic adds, the row kernel, the row kernel as the required deterministic mode
    for det, atomic in ((False, True), (False, False), (True, False)):
        dq, dx = d.backward(dev(Q), torch.from_numpy(idx).cuda(), dev(w), deterministic=det,
                            x_f32=xf, atomic=atomic)
        oi = idx.astype(np.int64)
        odq, odx = oracle.grad(Q, X, oi, w.astype(np.float64), metric)
        sq = np.abs(odq).max() + 1.0
        sx = np.abs(odx).max() + 1.0
        np.testing.assert_allclose(host(dq), odq, atol=1e-5 * sq * K, rtol=1e-5)
        np.testing.assert_allclose(host(dx), odx, atol=1e-5 * sx * M, rtol=1e-5)


def test_backward_deterministic_is_bitwise_repeatable():
    g = rng(12)
    N, M, D, K = 300, 600, 16, 8
    X, Q = inputs(N, M, D, seed=12)
    idx = g.integers(0, 20, size=(M, K)).astype(np.int32)  # heavy row sharing
    w = g.standard_normal((M, K)).astype(np.float32)
    d = db(X, "ip", "f32")
    outs = [host(d.backward(dev(Q), torch.from_numpy(idx).cuda(), dev(w), want_dq=False,
                            deterministic=True, x_f32=dev(X))[1]) for _ in range(3)]
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
    _, odx = oracle.grad(Q, X, idx.astype(np.int64), w.astype(np.float64), "ip", want_dq=False)
    np.testing.assert_allclose(outs[0], odx, rtol=1e-5, atol=1e-4)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("K,L", [(100, 2048), (150, 3000), (10, 1025), (64, 4097), (40, 8192)])
def test_search_many_queries_large_L_cta_rescoring(dtype, K, L):
    """L > 1024 or K' > 64 take a CTA ExactRescoring kernel: up to L = 2048
    and K' = 256 the one that sorts 256-key lists per warp and merges them,
    beyond that (up to L = 8192, 8 / 16 / 32 keys per thread) the radix
    select, whose set the re-rank orders. 1500 queries against the oracle
    catch a lost candidate."""
    X, Q = inputs(20000, 1500, 32, seed=91)
    if dtype == "f32":
        # few queries are decided at all 100 ranks; the per-query rules (values
        # by rank, own values, bin maxima) still apply to every query, and the
        # returned sets must match the oracle's
        _, gi = run_and_check(X, Q, "ip", K, L, 2)
        V, A = oracle.partial_reduce(Q, X, L, "ip")
        _, cand = oracle.topk_pairs(V, A, 2 * K)
        _, oi = oracle.rerank(Q, X, cand, K, "ip")
        agree = np.mean([len(set(gi[r]) & set(oi[r])) / K for r in range(len(Q))])
        assert agree > 0.999, agree
    else:
        from tests.test_gpu_lowp import run_lowp
        run_lowp(X, Q, "ip", "bf16", K, L, 2)


@pytest.mark.parametrize("dtype,metric", [("f32", "ip"), ("bf16", "l2"), ("bf16", "cos"),
                                          ("e4m3", "cos")])
def test_search_is_repeatable_whatever_the_workspace_holds(dtype, metric):
    """The same call twice, the workspace filled with different bytes before
    each: results must be bit-identical (nothing reads scratch it did not
    write, and no step depends on thread timing)."""
    X, Q = inputs(30000, 700, 64, seed=93)
    d = db(X, metric, dtype)
    outs = []
    for fill in (0x00, 0xA5, 0x5A):
        for t in d._ws.values():
            t.fill_(fill)
        v, i = d.search(dev(Q), 100, L=2048, rerank=2)
        outs.append((host(v), host(i)))
        for t in d._ws.values():
            t.fill_(fill ^ 0xFF)
    for v, i in outs[1:]:
        assert np.array_equal(i, outs[0][1])
        assert np.array_equal(v.view(np.uint32), outs[0][0].view(np.uint32))


@pytest.mark.parametrize("metric,dtype,keep", [("l2", "bf16", True), ("cos", "e4m3", False),
                                               ("ip", "f32", True), ("ip", "bf16", False)])
def test_owned_database_handle_matches_prepared_buffers(metric, dtype, keep):
    """knn_db_create / knn_db_search / knn_db_destroy: the library-owned
    database gives the same results, bit for bit, as knn_search on buffers
    the caller prepared with knn_prepare (the same kernels on the same
    bytes); without kept FP32 rows both re-rank from the stored rows."""
    import ctypes
    from paper_2206_14286_gb300 import search as S, _lib
    ensure_built()
    g = np.random.Generator(np.random.PCG64(91))
    X = g.standard_normal((20011, 96)).astype(np.float32)
    Q = g.standard_normal((130, 96)).astype(np.float32)
    Xd = dev(X)
    ref = S.Database(Xd, metric=metric, dtype=dtype, keep_f32=keep)
    own = S.OwnedDatabase(Xd, metric=metric, dtype=dtype, keep_f32=keep)
    del Xd                                  # the handle keeps its own copy
    torch.cuda.empty_cache()
    n, d, me, dt = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _lib.check(_lib.get().knn_db_info(own.handle, ctypes.byref(n), ctypes.byref(d),
                                      ctypes.byref(me), ctypes.byref(dt)))
    assert (n.value, d.value, me.value, dt.value) == (20011, 96, _lib.METRIC[metric],
                                                      _lib.DTYPE[dtype])
    for K, L, rr in [(10, 256, 2), (7, 100, 1)]:
        a = ref.search(dev(Q), K, L=L, rerank=rr)
        b = own.search(dev(Q), K, L=L, rerank=rr)
        torch.cuda.synchronize()
        assert torch.equal(a[1], b[1]) and torch.equal(a[0], b[0]), (K, L, rr)
    own.close()
    S.sync_status()


@pytest.mark.parametrize("metric", ["ip", "l2"])
def test_search_at_the_largest_K_and_D(metric):
    """The largest K a search accepts (4096, so K' = 4096 candidates through
    the streaming ExactRescoring kernel and the re-rank) and the largest row
    length (4096 elements)."""
    X, Q = inputs(20000, 12, 16, seed=95)
    frac, gi = run_and_check(X, Q, metric, 4096, 8192, 1)
    V, A = oracle.partial_reduce(Q, X, 8192, metric)
    _, cand = oracle.topk_pairs(V, A, 4096)
    _, oi = oracle.rerank(Q, X, cand, 4096, metric)
    agree = np.mean([len(set(gi[r]) & set(oi[r])) / 4096 for r in range(len(Q))])
    assert agree > 0.999, agree
    X, Q = inputs(3000, 20, 4096, seed=96)
    frac, _ = run_and_check(X, Q, metric, 10, 300, 2)
    # decided fraction for ip measured at 0.65 of the 20 queries (l2 above 0.8)
    assert frac > 0.5, frac
    S.sync_status()
