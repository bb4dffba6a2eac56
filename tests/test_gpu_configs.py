"""Full-size workloads checked on sampled queries.

FP8-E4M3 with per-row scales, cosine, N = 10,000,000 x D = 96 rows from a
1024-centre mixture, M = 10,000 queries, K = 100, L from the recall law for
0.95, FP32 re-rank of 2K candidates. The GPU runs the whole batch; the FP64
oracle follows the same steps for a few sampled queries. The database does not
fit the oracle in FP64 at once, so PartialReduce runs on chunks of 2^20 rows,
a multiple of L: a row keeps its bin (j mod L) inside its chunk, and a bin's
maximum is the maximum of its chunk maxima, ties to the smaller row, which is
the earlier chunk. The re-rank scores the gathered candidate rows.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2206_14286_gb300 import synth
from tests.gpu_util import db, dev, host

pytestmark = pytest.mark.gpu
CHUNK = 1 << 20


def chunked_partial_reduce(Qs_fn, X, L, metric):
    """PartialReduce over all rows of X, oracle per chunk, maxima merged."""
    V = A = None
    for c0 in range(0, X.shape[0], CHUNK):
        assert c0 % L == 0
        Xc = Qs_fn(X[c0:c0 + CHUNK])
        v, a = oracle.partial_reduce(Qs_fn.q, Xc, L, metric)
        a = np.where(a >= 0, a + c0, -1)
        if V is None:
            V, A = v, a
        else:
            better = v > V          # equal keeps the earlier (smaller) row
            V = np.where(better, v, V)
            A = np.where(better, a, A)
    return V, A


def chunked_exact(Q, X, K, metric, prep):
    vals, idxs = [], []
    for c0 in range(0, X.shape[0], CHUNK):
        v, i = oracle.exact_topk(Q, prep(X[c0:c0 + CHUNK]), K, metric)
        vals.append(v)
        idxs.append(i + c0)
    v = np.concatenate(vals, 1)
    i = np.concatenate(idxs, 1)
    order = np.lexsort((i, -v), axis=1)
    return np.take_along_axis(v, order, 1)[:, :K], np.take_along_axis(i, order, 1)[:, :K]


def test_e4m3_cosine_10m_k100_sampled():
    from paper_2206_14286_gb300 import search as S
    w = synth.workload("mix_cos_10m")
    X, Q, K = w["X"], w["Q"], w["K"]
    N, D = X.shape
    M = Q.shape[0]
    L = S.plan_bins(N, K, 0.95, round_to=128)
    assert L == 2048 and CHUNK % L == 0
    d = db(X, "cos", "e4m3")
    val, idx = d.search(dev(Q), K, L=L, rerank=2)
    gv, gi = host(val), host(idx)
    assert gi.shape == (M, K) and np.all((gi >= 0) & (gi < N))
    # the GPU returns distinct rows, best first
    assert all(len(set(r)) == K for r in gi[:200])
    assert np.all(np.diff(gv, axis=1) <= 0)
    del d
    torch.cuda.empty_cache()

    samp = np.random.Generator(np.random.PCG64(9)).choice(M, size=6, replace=False)
    Qn = oracle.normalize_rows(Q[samp])
    Qs, _ = oracle.e4m3_rows(Qn)

    def stored_rows(Xc):            # what the GPU contracts: E4M3 codes x row scale
        return oracle.e4m3_rows(oracle.normalize_rows(Xc))[0]
    stored_rows.q = Qs
    V, A = chunked_partial_reduce(stored_rows, X, L, "ip")
    _, cand = oracle.topk_pairs(V, A, 2 * K)
    # FP32 re-rank on the unit rows of the candidates only
    uniq, inv = np.unique(cand[cand >= 0], return_inverse=True)
    Xsub = oracle.normalize_rows(X[uniq])
    csub = np.full(cand.shape, -1, np.int64)
    csub[cand >= 0] = inv
    ov, oi_sub = oracle.rerank(Qn, Xsub, csub, K, "ip")
    oi = np.where(oi_sub >= 0, uniq[np.maximum(oi_sub, 0)], -1)

    # the GPU's answer for each sampled query against the oracle's
    agree = np.mean([len(set(gi[s]) & set(oi[k])) / K for k, s in enumerate(samp)])
    assert agree > 0.97, agree
    # values: FP32 cosines of the same rows
    np.testing.assert_allclose(np.sort(gv[samp], 1), np.sort(ov, 1), rtol=0, atol=2e-3)
    # every returned value is the FP32 cosine of its own row
    for k, s in enumerate(samp):
        own = oracle.normalize_rows(X[gi[s]]).astype(np.float64) @ Qn[k].astype(np.float64)
        np.testing.assert_allclose(gv[s], own, rtol=0, atol=1e-5)
    # recall@100 against the exact FP32 cosine top-100. Reported, with a floor:
    # the bin step ranks by E4M3 scores (3 mantissa bits), and among the
    # near-tied neighbours of a 1024-centre mixture that choice often differs
    # from FP32's inside a bin, which no re-rank recovers (measured 0.755 on
    # these six queries; the oracle's own E4M3 search agrees with the GPU above).
    _, ei = chunked_exact(Qn, X, K, "ip", oracle.normalize_rows)
    rec = np.mean([len(set(gi[s]) & set(ei[k])) / K for k, s in enumerate(samp)])
    orec = np.mean([len(set(oi[k]) & set(ei[k])) / K for k in range(len(samp))])
    print("E4M3 cosine 10M x 96, K=100, L=%d: recall@100 vs FP32 exact %.3f (oracle %.3f)"
          % (L, rec, orec))
    assert abs(rec - orec) <= 0.03
    assert rec >= 0.6, rec
