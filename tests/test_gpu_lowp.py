"""Parity of the tensor-core paths (BF16 and FP8-E4M3 with per-row scales)
against the FP64 oracle run on the same dequantised values the GPU saw.

The bin step runs on the stored (rounded) rows and queries; the final values
are FP32 scores of the FP32 rows (re-rank). The oracle mirrors both steps.
Tolerance: the stated rel 1e-2 of the natural score scale for the bin step
(BF16/FP8) and rel 1e-5 for re-ranked FP32 values; then the tighter bound of
each kernel's arithmetic: the BF16 kernel keeps the FP32 accumulator in its
keys (3e-5 of the scale, plus 2^-20 of the largest |x|^2 for the L2 half-norm
split), the E4M3 kernel's packed key keeps 2^-10 of a score's magnitude."""
import numpy as np
import pytest
import torch

import oracle
from paper_2206_14286_gb300 import synth
from tests import parity as PT
from tests.gpu_util import db, dev, host

pytestmark = pytest.mark.gpu
METRICS = ["ip", "l2", "cos"]


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def inputs(N, M, D, seed=0):
    g = rng(seed)
    return g.standard_normal((N, D)).astype(np.float32), g.standard_normal((M, D)).astype(np.float32)


def stored(A, metric, dtype, query=False):
    """(dequantised stored rows, FP32 rows used by the re-rank) per the oracle.
    'e4m3t' stores the database with one scale and the queries per row."""
    src = oracle.normalize_rows(A) if metric == "cos" else A.astype(np.float32)
    if dtype == "bf16":
        return oracle.bf16_round(src), src.astype(np.float64)
    if dtype == "e4m3t" and not query:
        deq, _ = oracle.e4m3_tensor(src)
        return deq, src.astype(np.float64)
    deq, _ = oracle.e4m3_rows(src)
    return deq, src.astype(np.float64)


def tcs_e4m3(dtype, metric):
    """E4M3 with one database scale runs the BF16 kernel's design (FP32
    accumulator in the keys) for IP and COS; with L2 it runs as 'e4m3'."""
    return dtype == "e4m3t" and metric != "l2"


def om(metric):
    return "ip" if metric == "cos" else metric


# ----------------------------------------------------------------------------
# PartialReduce alone
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", ["bf16", "e4m3", "e4m3t"])
@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("shape", [(3001, 70, 72), (5000, 300, 128), (2500, 40, 256), (700, 9, 16)])
def test_partial_reduce_lowp(dtype, metric, shape):
    N, M, D = shape
    X, Q = inputs(N, M, D, seed=N + M)
    Xs, _ = stored(X, metric, dtype)
    Qs, _ = stored(Q, metric, dtype, query=True)
    d = db(X, metric, dtype)
    Sm = PT.score_matrix(Qs, Xs, om(metric))
    for L in (1, 5, 100, 128, 300, N):
        V, A = d.partial_reduce(dev(Q), L)
        V, A = host(V).astype(np.float64), host(A)
        Vo, Ao = oracle.partial_reduce(Qs, Xs, L, om(metric))
        if metric == "l2":
            Vo = (Vo + (Qs ** 2).sum(1)[:, None]) / 2.0
        if dtype != "bf16" and metric != "l2":
            # the kernel leaves the per-query scale out of the value
            _, qsc = oracle.e4m3_rows(oracle.normalize_rows(Q) if metric == "cos" else Q)
            Vo = Vo / qsc[:, None].astype(np.float64)
        scale = PT.query_scale(Qs, Xs, metric)
        if tcs_e4m3(dtype, metric):
            # FP32 accumulator of the codes' exact products, times the
            # database scale (in the scale without the query's)
            tol_bin = PT.fp32_acc_tol(Qs, Xs, metric)
            tight = (tol_bin / qsc)[:, None] + 2.0 ** -20 * np.abs(Vo)
        elif dtype == "bf16":
            # the BF16 kernel keeps the FP32 accumulator in its 64-bit keys;
            # its values are in the relaxed scale (half of -|q-x|^2 for L2)
            tol_bin = PT.fp32_acc_tol(Qs, Xs, metric)
            tight = (tol_bin / 2 if metric == "l2" else tol_bin)[:, None] + \
                2.0 ** -20 * np.abs(Vo)
        else:
            # the E4M3 kernel's packed 32-bit key keeps the top bits of each
            # FP32 score (its low bits hold the row's position in its bin)
            tol_bin = PT.REL_LOWP * scale
            tight = 2.0 ** -9 * np.abs(Vo) + 1e-5 * scale[:, None]
            if metric != "l2":
                tight = 2.0 ** -9 * np.abs(Vo) + 1e-5 * scale[:, None] / qsc[:, None]
        best, second = PT.bin_best_second(Sm, L)
        decided = (best - second) > 2 * tol_bin[:, None]
        assert np.all(A % L == np.arange(L)[None, :])
        np.testing.assert_array_equal(A[decided], Ao[decided])
        err = np.abs(V - Vo)
        # undecided bins may hold a different near-best member: compare by its own score
        own = Sm[np.arange(M)[:, None], A]
        if metric == "l2":
            own = (own + (Qs ** 2).sum(1)[:, None]) / 2.0
        if dtype != "bf16" and metric != "l2":
            own = own / qsc[:, None]
        assert np.all(err[decided] <= tight[decided]), (L, err[decided].max())
        assert np.all(np.abs(V - own) <= tight), (L,)
        if dtype == "bf16" or tcs_e4m3(dtype, metric):
            assert decided.mean() > 0.9, (L, decided.mean())


@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("shape", [(1500, 33, 768), (900, 5, 1000), (600, 3, 4096), (2049, 17, 200)])
def test_partial_reduce_bf16_long_rows(metric, shape):
    """BF16 rows longer than 128 elements: the K loop walks one 128-byte K
    block per stage (query tile resident up to 256, streamed beyond)."""
    N, M, D = shape
    X, Q = inputs(N, M, D, seed=N + D)
    Xs, _ = stored(X, metric, "bf16")
    Qs, _ = stored(Q, metric, "bf16")
    d = db(X, metric, "bf16")
    Sm = PT.score_matrix(Qs, Xs, om(metric))
    scale = PT.query_scale(Qs, Xs, metric)
    for L in (1, 16, 100, N):
        V, A = d.partial_reduce(dev(Q), L)
        V, A = host(V).astype(np.float64), host(A)
        Vo, Ao = oracle.partial_reduce(Qs, Xs, L, om(metric))
        if metric == "l2":
            Vo = (Vo + (Qs ** 2).sum(1)[:, None]) / 2.0
        tol = PT.REL_LOWP * scale
        best, second = PT.bin_best_second(Sm, L)
        decided = (best - second) > 2 * tol[:, None]
        assert np.all(A % L == np.arange(L)[None, :])
        np.testing.assert_array_equal(A[decided], Ao[decided])
        # FP32 accumulation of D products (and the three-part split of h for L2)
        tight = 3e-5 * scale[:, None] + 2.0 ** -20 * np.abs(Vo)
        own = Sm[np.arange(M)[:, None], A]
        if metric == "l2":
            own = (own + (Qs ** 2).sum(1)[:, None]) / 2.0
        assert np.all(np.abs(V - Vo)[decided] <= tight[decided]), (L,)
        assert np.all(np.abs(V - own) <= tight), (L,)


@pytest.mark.parametrize("metric", METRICS)
def test_search_bf16_long_rows(metric):
    X, Q = inputs(3000, 40, 768, seed=77)
    # i.i.d. rows of length 768: the score gaps lie inside the stated tolerance,
    # so few queries are decided; the within-tolerance checks still apply
    for K, L, rr in [(10, 128, 2), (5, 3000, 1)]:
        run_lowp(X, Q, metric, "bf16", K, L, rr)
    # planted neighbours: each query is a row plus small noise, so that row is
    # the best by a wide margin (score ~ D against ~3.5 sqrt(D) for the rest)
    # and must come back first
    g = rng(78)
    rows = g.choice(3000, size=40, replace=False)
    Qp = (X[rows] + 0.01 * g.standard_normal((40, 768))).astype(np.float32)
    _, gi = run_lowp(X, Qp, metric, "bf16", 1, 128, 2)
    assert np.array_equal(gi[:, 0], rows)


# ----------------------------------------------------------------------------
# Search with FP32 re-rank
# ----------------------------------------------------------------------------
def lowp_oracle_side(X, Q, metric, dtype, K, L, rerank, bins="mod"):
    """The oracle's answer and the decided masks of run_lowp (no GPU)."""
    Xs, Xf = stored(X, metric, dtype)
    Qs, Qf = stored(Q, metric, dtype, query=True)
    Kp = min(max(1, rerank) * K, L)
    V, A = oracle.partial_reduce(Qs, Xs, L, om(metric), bins=bins)
    _, cand = oracle.topk_pairs(V, A, Kp)
    ov, oi = oracle.rerank(Qf, Xf, cand, K, om(metric))
    S_lp = PT.score_matrix(Qs, Xs, om(metric))
    S_f = PT.score_matrix(Qf, Xf, om(metric))
    scale_lp = PT.query_scale(Qs, Xs, metric)
    tol_lp = PT.REL_LOWP * scale_lp
    tol_f = PT.REL_F32 * PT.query_scale(Qf, Xf, metric)
    # the stated rule: rel 1e-2 (BF16/FP8) for the bin step
    dec = PT.decided_mask(S_lp, L, Kp, S_f, cand, K, tol_lp, bins=bins)
    # a stricter rule derived from the kernels' arithmetic: the BF16 kernel
    # keeps the FP32 accumulator in its keys; the E4M3 kernel's packed key
    # keeps scores to 2^-10 of their magnitude, plus FP32 accumulation
    if dtype == "bf16" or tcs_e4m3(dtype, metric):
        tol_d = PT.fp32_acc_tol(Qs, Xs, metric)
    else:
        tol_d = 2.0 ** -9 * (scale_lp if metric == "l2" else np.abs(S_lp).max(1)) + \
            3e-5 * scale_lp
    tol_df = np.maximum(tol_f, 3e-5 * PT.query_scale(Qf, Xf, metric))
    dec2 = PT.decided_mask(S_lp, L, Kp, S_f, cand, K, tol_d, tol_df, bins=bins) | dec
    return dict(ov=ov, oi=oi, S_lp=S_lp, S_f=S_f, tol_lp=tol_lp, tol_d=tol_d, tol_df=tol_df,
                dec=dec, dec2=dec2)


def run_lowp(X, Q, metric, dtype, K, L, rerank, bins="mod"):
    d = db(X, metric, dtype)
    val, idx = d.search(dev(Q), K, L=L, rerank=rerank, bins=bins)
    gv, gi = host(val), host(idx)
    o = lowp_oracle_side(X, Q, metric, dtype, K, L, rerank, bins)
    ov, oi, S_lp, S_f = o["ov"], o["oi"], o["S_lp"], o["S_f"]
    PT.check_search(gv, gi, ov, oi, S_lp, S_f, L, om(metric), o["tol_lp"], o["dec"], bins=bins)
    dec2 = o["dec2"]
    frac = PT.check_search(gv, gi, ov, oi, S_lp, S_f, L, om(metric),
                           np.maximum(o["tol_d"], o["tol_df"]), dec2, bins=bins)
    # values are FP32 re-ranked: FP32 tolerance where decided
    np.testing.assert_allclose(gv[dec2], ov[dec2], rtol=0, atol=float(np.max(o["tol_df"])) + 1e-6)
    return frac, gi


@pytest.mark.parametrize("dtype", ["bf16", "e4m3", "e4m3t"])
@pytest.mark.parametrize("metric", METRICS)
def test_search_lowp_small(dtype, metric):
    X, Q = inputs(6007, 131, 64, seed=21)
    for K, L, rr in [(10, 176, 2), (10, 256, 1), (4, 4, 1), (1, 1, 1), (8, 6007, 1)]:
        frac, _ = run_lowp(X, Q, metric, dtype, K, L, rr)
        # floors a little under the decided fractions, which depend on the
        # oracle side alone (BF16: 0.83-1.0; E4M3 IP/COS: 0.37-0.97; E4M3 L2,
        # whose packed-key truncation scales with the norm-dominated relaxed
        # score: 0.08-0.78)
        floor = 0.75 if dtype == "bf16" or tcs_e4m3(dtype, metric) else \
            (0.05 if metric == "l2" else 0.3)
        assert frac > floor, (K, L, rr, frac)


# ----------------------------------------------------------------------------
# Contiguous bins (Alg. 1's ShiftRight): BF16 kernel with queries on TMEM lanes
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("metric", METRICS)
@pytest.mark.parametrize("shape", [(3001, 70, 72), (5000, 300, 128), (700, 9, 16),
                                   (20011, 130, 128), (4000, 129, 256)])
def test_partial_reduce_contiguous_bf16(metric, shape):
    N, M, D = shape
    X, Q = inputs(N, M, D, seed=N + M + 7)
    Xs, _ = stored(X, metric, "bf16")
    Qs, _ = stored(Q, metric, "bf16")
    d = db(X, metric, "bf16")
    Sm = PT.score_matrix(Qs, Xs, om(metric))
    scale = PT.query_scale(Qs, Xs, metric)
    tight = 3e-5 * scale[:, None]     # FP32 accumulation; no packed-key truncation here
    for L in (1, 5, 100, 128, 300, N):
        V, A = d.partial_reduce(dev(Q), L, bins="contiguous")
        V, A = host(V).astype(np.float64), host(A)
        Vo, Ao = oracle.partial_reduce(Qs, Xs, L, om(metric), bins="contiguous")
        if metric == "l2":
            Vo = (Vo + (Qs ** 2).sum(1)[:, None]) / 2.0
        bins = np.array_split(np.arange(N), L)
        owner = np.concatenate([np.full(len(r), b) for b, r in enumerate(bins)])
        assert np.all(owner[A] == np.arange(L)[None, :]), L
        best, second = PT.bin_best_second(Sm, L, bins="contiguous")
        decided = (best - second) > 2 * tight
        np.testing.assert_array_equal(A[decided], Ao[decided])
        own = Sm[np.arange(M)[:, None], A]
        if metric == "l2":
            own = (own + (Qs ** 2).sum(1)[:, None]) / 2.0
            tl = tight / 2 + 2.0 ** -20 * (Xs ** 2).sum(1).max()
        else:
            tl = tight
        assert np.all(np.abs(V - Vo) <= tl), (L, np.abs(V - Vo).max())
        assert np.all(np.abs(V - own) <= tl), L
        assert decided.mean() > 0.9


@pytest.mark.parametrize("metric", METRICS)
def test_search_contiguous_bf16_small(metric):
    X, Q = inputs(6007, 131, 64, seed=31)
    for K, L, rr in [(10, 176, 2), (10, 256, 1), (4, 4, 1), (1, 1, 1), (8, 6007, 1)]:
        frac, _ = run_lowp(X, Q, metric, "bf16", K, L, rr, bins="contiguous")
        assert frac > 0.75, (K, L, rr, frac)      # decided: 0.82-1.0


@pytest.mark.parametrize("dtype", ["bf16", "e4m3", "e4m3t"])
@pytest.mark.parametrize("metric", ["ip", "l2"])
def test_exact_search_lowp(dtype, metric):
    X, Q = inputs(9000, 150, 96, seed=22)
    d = db(X, metric, dtype)
    val, idx = d.search_exact(dev(Q), 7)
    gv, gi = host(val), host(idx)
    Xs, Xf = stored(X, metric, dtype)
    Qs, Qf = stored(Q, metric, dtype, query=True)
    _, cand = oracle.exact_topk(Qs, Xs, 7, metric)
    ov, oi = oracle.rerank(Qf, Xf, cand, 7, metric)
    S_lp = PT.score_matrix(Qs, Xs, metric)
    S_f = PT.score_matrix(Qf, Xf, metric)
    tol = PT.REL_LOWP * PT.query_scale(Qs, Xs, metric)
    dec = PT.decided_mask(S_lp, 9000, 7, S_f, cand, 7, tol)
    PT.check_search(gv, gi, ov, oi, S_lp, S_f, 9000, metric, tol, dec)


@pytest.mark.parametrize("bins", ["mod", "contiguous"])
@pytest.mark.parametrize("metric", ["ip", "l2"])
def test_partial_reduce_many_query_tiles(bins, metric):
    """More 256-query tiles than SMs: a CTA takes several tiles in turn over
    the same database rows (query tile reloaded between them)."""
    N, M, D = 600, 39500, 32
    X, Q = inputs(N, M, D, seed=5)
    Xs, _ = stored(X, metric, "bf16")
    Qs, _ = stored(Q, metric, "bf16")
    d = db(X, metric, "bf16")
    Sm = PT.score_matrix(Qs, Xs, om(metric))
    scale = PT.query_scale(Qs, Xs, metric)
    tight = 3e-5 * scale[:, None] + 2.0 ** -20 * np.abs(Sm).max(1)[:, None]
    for L in (7, 100):
        V, A = d.partial_reduce(dev(Q), L, bins=bins)
        V, A = host(V).astype(np.float64), host(A)
        Vo, Ao = oracle.partial_reduce(Qs, Xs, L, om(metric), bins=bins)
        if metric == "l2":
            Vo = (Vo + (Qs ** 2).sum(1)[:, None]) / 2.0
        best, second = PT.bin_best_second(Sm, L, bins=bins)
        decided = (best - second) > 2 * tight
        np.testing.assert_array_equal(A[decided], Ao[decided])
        own = Sm[np.arange(M)[:, None], A]
        if metric == "l2":
            own = (own + (Qs ** 2).sum(1)[:, None]) / 2.0
        assert np.all(np.abs(V - own) <= tight), L
        assert decided.mean() > 0.9, L


@pytest.mark.parametrize("metric", METRICS)
def test_search_fused_rescoring_bounds(metric):
    """ExactRescoring and the FP32 re-rank run as one launch when L <= 1024,
    Kp <= 32 and K <= 32: its edges (one and 32 keys per lane, Kp = 32)."""
    X, Q = inputs(5000, 77, 64, seed=41)
    for K, L, rr in [(16, 1024, 2), (32, 1024, 1), (32, 33, 1), (3, 40, 8), (1, 32, 1)]:
        frac, gi = run_lowp(X, Q, metric, "bf16", K, L, rr)
        # with K up to 32 and bins of ~5 rows more queries hold a near-tie
        # within twice the tolerance (decided: 0.38-1.0); the checks in
        # run_lowp cover every query
        assert frac > 0.3, (K, L, rr, frac)
        # every row returned once per query
        for r in gi:
            assert len(set(r[r >= 0].tolist())) == int((r >= 0).sum())


@pytest.mark.parametrize("dtype", ["bf16", "e4m3t"])
@pytest.mark.parametrize("metric", METRICS)
def test_search_ragged_last_grid_row(dtype, metric):
    """With j mod L bins the N mod L rows of the ragged last grid row are
    scored by their own kernel and merge with the tensor-core bins: one such
    row, and a few hundred of them, with L up to the fused rescoring's 1024."""
    if dtype == "e4m3t" and metric == "l2":
        pytest.skip("E4M3 with L2 runs the per-row-scale kernel, which has no ragged path")
    for N, L in [(257, 64), (1456, 300), (2657, 600), (2303, 1024)]:
        X, Q = inputs(N, 77, 64, seed=N)
        frac, gi = run_lowp(X, Q, metric, dtype, 10, L, 2)
        assert frac > 0.75, (N, L, frac)          # decided: 0.80-0.95
        ragged = N - (N // L) * L
        assert ragged in (1, 256, 257, 255)


@pytest.mark.parametrize("metric", ["ip", "cos"])
def test_search_contiguous_e4m3t_small(metric):
    """Contiguous bins with E4M3 codes and one database scale (the BF16
    kernel's run walk with E4M3 MMAs)."""
    X, Q = inputs(6007, 131, 64, seed=32)
    for K, L, rr in [(10, 176, 2), (4, 4, 1), (8, 6007, 1)]:
        frac, _ = run_lowp(X, Q, metric, "e4m3t", K, L, rr, bins="contiguous")
        assert frac > 0.75, (K, L, rr, frac)


@pytest.mark.parametrize("metric", ["ip", "cos"])
@pytest.mark.parametrize("shape", [(1500, 33, 768), (600, 3, 4096), (2049, 17, 200)])
def test_partial_reduce_e4m3t_long_rows(metric, shape):
    """E4M3 rows longer than 128 bytes walk one 128-byte K block per stage
    (up to 4096 elements), as BF16 rows longer than 64 elements do."""
    N, M, D = shape
    X, Q = inputs(N, M, D, seed=N + D + 1)
    Xs, _ = stored(X, metric, "e4m3t")
    Qs, _ = stored(Q, metric, "e4m3t", query=True)
    _, qsc = oracle.e4m3_rows(oracle.normalize_rows(Q) if metric == "cos" else Q)
    d = db(X, metric, "e4m3t")
    Sm = PT.score_matrix(Qs, Xs, om(metric))
    tol = PT.fp32_acc_tol(Qs, Xs, metric)
    for L in (1, 16, 100, N):
        V, A = d.partial_reduce(dev(Q), L)
        V, A = host(V).astype(np.float64), host(A)
        Vo, Ao = oracle.partial_reduce(Qs, Xs, L, om(metric))
        Vo = Vo / qsc[:, None]
        best, second = PT.bin_best_second(Sm, L)
        decided = (best - second) > 2 * tol[:, None]
        assert np.all(A % L == np.arange(L)[None, :])
        np.testing.assert_array_equal(A[decided], Ao[decided])
        tight = (tol / qsc)[:, None] + 2.0 ** -20 * np.abs(Vo)
        own = Sm[np.arange(M)[:, None], A] / qsc[:, None]
        assert np.all(np.abs(V - Vo)[decided] <= tight[decided]), (L,)
        assert np.all(np.abs(V - own) <= tight), (L,)


@pytest.mark.parametrize("K,L,rr", [(100, 2049, 3), (64, 4097, 8), (1, 2500, 2500), (10, 8192, 300)])
def test_search_select_rescoring_edges(K, L, rr):
    """ExactRescoring as a radix select (L > 2048 or K' > 256, up to 8192):
    the key-per-thread boundaries (L = 2049, 4097, 8192) and K' = L (every
    bin winner re-ranked: the select keeps them all). i.i.d. rows of length
    32 leave few queries decided at every rank (0-0.13 here); run_lowp's
    per-query rules (values by rank, own values, bin maxima) cover them all."""
    X, Q = inputs(20000, 45, 32, seed=L + K)
    _, gi = run_lowp(X, Q, "ip", "bf16", K, L, rr)
    for r in gi:
        assert len(set(r.tolist())) == K
