"""The N-sharded search's kernels (knn_shard_*) on one GPU.

The shards of a database run one after another on the same GPU, and an
element-wise torch.maximum over their int64 key arrays stands in for the
all-reduce MAX that merges them across GPUs (the kernels never wait on each
other, so nothing here needs several devices). Checked:
  * the merged PartialReduce keys equal, bin by bin, PartialReduce of the
    whole database (knn_partial_reduce): bit for bit for BF16 and FP32, where
    every row's score is computed by the same kernel arithmetic whichever shard
    holds it; by the oracle's parity rule for E4M3, whose packed keys depend on
    the tile count;
  * the final answer against the FP64 oracle (PartialReduce -> top Kp -> FP32
    re-rank on the whole database) by the parity rule of tests/parity.py.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2206_14286_gb300 import search as S
from paper_2206_14286_gb300 import shard as SH
from tests import parity as PT
from tests.gpu_util import db, dev, ensure_built, host
from tests.test_gpu_lowp import lowp_oracle_side, om

pytestmark = pytest.mark.gpu
SIGN = np.uint64(1 << 63)


def unpack(keys):
    k = np.asarray(keys).view(np.uint64) ^ SIGN
    o = k >> np.uint64(32)
    u = np.where((o & np.uint64(0x80000000)) != 0, o & np.uint64(0x7FFFFFFF),
                 (~o) & np.uint64(0xFFFFFFFF))
    idx = ((~k) & np.uint64(0xFFFFFFFF)).astype(np.int64)
    return u.astype(np.uint32).view(np.float32), np.where(k == 0, -1, idx)


@pytest.mark.parametrize("dtype,metric", [("bf16", "l2"), ("bf16", "ip"), ("f32", "ip"),
                                          ("e4m3", "cos"), ("bf16", "cos")])
@pytest.mark.parametrize("shards", [1, 3])
def test_sharded_search_equals_the_whole_database(dtype, metric, shards):
    ensure_built()
    g = np.random.Generator(np.random.PCG64(99 + shards))
    N, D, M, K, rr = 20011, 64, 150, 10, 2
    X = g.standard_normal((N, D)).astype(np.float32)
    Q = g.standard_normal((M, D)).astype(np.float32)
    L = S.plan_bins(N, K, 0.95, round_to=128)
    bounds = SH.shard_bounds(N, shards, L)
    parts = [SH.DatabaseShard(dev(X[r0:r0 + n]), r0, N, metric, dtype) for r0, n in bounds]
    q = dev(Q)
    keys = [p.partial(q, L) for p in parts]
    merged = keys[0]
    for k in keys[1:]:
        merged = torch.maximum(merged, k)            # the all-reduce MAX
    cands = [p.rescore(merged, q, K, rr, L) for p in parts]
    mc = cands[0]
    for c in cands[1:]:
        mc = torch.maximum(mc, c)
    outs = [p.finish(mc, K) for p in parts]
    torch.cuda.synchronize()
    S.sync_status()
    for v, i in outs[1:]:                             # every shard gets the same answer
        assert torch.equal(v, outs[0][0]) and torch.equal(i, outs[0][1])
    gv, gi = host(outs[0][0]), host(outs[0][1])

    # exchange 1 against PartialReduce of the whole database
    whole = db(X, metric, dtype)
    V, A = whole.partial_reduce(q, L)
    V, A = host(V), host(A)
    ms, mi = unpack(host(merged))
    if dtype != "e4m3":
        np.testing.assert_array_equal(mi, A)
        np.testing.assert_array_equal(ms, V)
    else:
        assert np.all(mi % L == np.arange(L)[None, :])
        agree = (mi == A).mean()
        assert agree > 0.97, agree

    # the answer against the oracle
    if dtype == "f32":
        Xs = oracle.normalize_rows(X) if metric == "cos" else X.astype(np.float64)
        Qs = oracle.normalize_rows(Q) if metric == "cos" else Q.astype(np.float64)
        Vo, Ao = oracle.partial_reduce(Qs, Xs, L, om(metric))
        _, cand = oracle.topk_pairs(Vo, Ao, min(rr * K, L))
        ov, oi = oracle.rerank(Qs, Xs, cand, K, om(metric))
        S_ = PT.score_matrix(Qs, Xs, om(metric))
        tol = PT.REL_F32 * PT.query_scale(Qs, Xs, metric)
        dec = PT.decided_mask(S_, L, min(rr * K, L), S_, cand, K, tol)
        frac = PT.check_search(gv, gi, ov, oi, S_, S_, L, om(metric), tol, dec)
    else:
        o = lowp_oracle_side(X, Q, metric, dtype, K, L, rr)
        frac = PT.check_search(gv, gi, o["ov"], o["oi"], o["S_lp"], o["S_f"], L, om(metric),
                               np.maximum(o["tol_d"], o["tol_df"]), o["dec2"])
    # decided fractions from the oracle side alone: 0.78-0.91 (E4M3: 0.24-0.31)
    assert frac > (0.6 if dtype != "e4m3" else 0.15), frac
    # and against the unsharded search: the same rows
    wv, wi = whole.search(q, K, L=L, rerank=rr)
    wv, wi = host(wv), host(wi)
    same = np.mean([len(set(gi[k]) & set(wi[k])) / K for k in range(M)])
    assert same > (0.99 if dtype != "e4m3" else 0.97), same
