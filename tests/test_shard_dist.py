"""The N-sharded search's host logic on the CPU: world_size-2 gloo ranks.

Each rank holds one shard of the rows (paper_2206_14286_gb300.shard.shard_bounds:
starts at multiples of L) and runs the package's orchestration
(shard.sharded_search: PartialReduce keys -> all-reduce MAX -> rescoring keys
-> all-reduce MAX -> top K) with the exchanges over gloo. The three per-shard
calls are stood in for by the FP64 oracle producing the keys the library's
knn_shard_* calls exchange (ordered FP32 score, complement of the global row,
XOR 2^63, read as int64): so this checks the partition, the key order and the
merge by a signed MAX, and the two exchange steps. The merged bin winners
must equal the oracle's PartialReduce (Alg. 1) of the whole database, and the
answer its ExactRescoring + re-rank, bit for bit.
"""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SIGN = np.uint64(1 << 63)
MASK32 = np.uint64(0xFFFFFFFF)


def pack(score, idx):
    """(score, global row) -> signed-order int64 keys; idx < 0 -> INT64_MIN."""
    u = np.asarray(score, np.float32).view(np.uint32).astype(np.uint64)
    o = np.where((u & np.uint64(0x80000000)) != 0, (~u) & MASK32, u | np.uint64(0x80000000))
    k = (o << np.uint64(32)) | ((~np.asarray(idx).astype(np.uint64)) & MASK32)
    k = np.where(np.asarray(idx) < 0, np.uint64(0), k)
    return (k ^ SIGN).view(np.int64)


def unpack(keys):
    k = np.asarray(keys).view(np.uint64) ^ SIGN
    o = k >> np.uint64(32)
    u = np.where((o & np.uint64(0x80000000)) != 0, o & np.uint64(0x7FFFFFFF), (~o) & MASK32)
    score = u.astype(np.uint32).view(np.float32)
    idx = ((~k) & MASK32).astype(np.int64)
    return np.where(k == 0, np.nan, score), np.where(k == 0, -1, idx)


def oracle_scores(q, X, rows, metric):
    """FP64 larger-is-better scores of query q against rows X[rows]."""
    x = np.asarray(X[rows], np.float64)
    q = np.asarray(q, np.float64)
    if metric == "ip":
        return x @ q
    if metric == "l2":
        return -((x - q) ** 2).sum(1)
    return (x @ q) / (np.linalg.norm(x, axis=1) * np.linalg.norm(q))


class OracleShard:
    """The contract of knn_shard_partial_reduce / _rescore / _finish for the
    rows [row0, row0 + n), computed by the FP64 oracle (scores rounded to FP32
    as the keys hold them)."""

    def __init__(self, X_local, row0, metric):
        self.X, self.row0, self.metric = X_local, row0, metric
        self.merged = None

    def partial(self, q, L):
        import oracle
        V, A = oracle.partial_reduce(q.numpy(), self.X, L, self.metric)
        A = np.where(A >= 0, A + self.row0, -1)
        return torch.from_numpy(pack(V.astype(np.float32), A))

    def rescore(self, keys, q, K, rerank, L):
        self.merged = keys.clone()
        Kp = min(max(1, rerank) * K, L)
        top = -np.sort(-keys.numpy(), axis=1)[:, :Kp]
        _, idx = unpack(top)
        out = np.full(idx.shape, np.iinfo(np.int64).min, np.int64)
        for i in range(idx.shape[0]):
            own = (idx[i] >= self.row0) & (idx[i] < self.row0 + self.X.shape[0])
            s = oracle_scores(q.numpy()[i], self.X, idx[i][own] - self.row0, self.metric)
            out[i, own] = pack(s.astype(np.float32), idx[i][own])
        return torch.from_numpy(out)

    def finish(self, cand, K):
        top = -np.sort(-cand.numpy(), axis=1)[:, :K]
        s, idx = unpack(top)
        return (-s if self.metric == "l2" else s), idx


def data(metric):
    g = np.random.Generator(np.random.PCG64(404))
    X = g.standard_normal((3001, 24)).astype(np.float32)
    Q = g.standard_normal((25, 24)).astype(np.float32)
    return X, Q


K, L, RERANK = 5, 64, 3


def _rank(rank, world, port, metric, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    from paper_2206_14286_gb300 import shard as SH
    X, Q = data(metric)
    row0, n = SH.shard_bounds(X.shape[0], world, L)[rank]
    sh = OracleShard(X[row0:row0 + n], row0, metric)
    val, idx = SH.sharded_search(sh, torch.from_numpy(Q), K, L, RERANK, SH.dist_allreduce_max())
    out[rank] = (val, idx, sh.merged.numpy(), (row0, n))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_bounds_align_to_bins_and_cover_the_rows():
    from paper_2206_14286_gb300 import shard as SH
    for N, S, L_ in [(1_000_000, 8, 256), (3001, 2, 64), (10_000_000, 3, 8192), (640, 5, 128)]:
        b = SH.shard_bounds(N, S, L_)
        assert len(b) == S and b[0][0] == 0
        assert all(r0 % L_ == 0 and n >= L_ for r0, n in b)
        assert all(b[k][0] + b[k][1] == b[k + 1][0] for k in range(S - 1))
        assert b[-1][0] + b[-1][1] == N
    with pytest.raises(ValueError):
        SH.shard_bounds(300, 4, 128)        # a shard would hold fewer than L rows


@pytest.mark.parametrize("metric", ["ip", "l2", "cos"])
def test_two_gloo_ranks_merge_to_the_whole_database(metric):
    import oracle
    world = 2
    port = 29600 + (os.getpid() + ["ip", "l2", "cos"].index(metric)) % 1000
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, metric, out), nprocs=world, join=True)
    X, Q = data(metric)
    # both ranks hold the same answer
    for a, b in zip(out[0][:3], out[1][:3]):
        np.testing.assert_array_equal(a, b)
    val, idx, merged, _ = out[0]
    assert out[0][3] == (0, 1536) and out[1][3] == (1536, 1465)
    # exchange 1: the merged bin winners are PartialReduce of the whole database
    V, A = oracle.partial_reduce(Q, X, L, metric)
    ms, mi = unpack(merged)
    np.testing.assert_array_equal(mi, A)
    np.testing.assert_array_equal(ms, V.astype(np.float32))
    # exchange 2 and the finish: ExactRescoring's top Kp, FP32 re-rank, top K
    Kp = min(RERANK * K, L)
    _, cand = oracle.topk_pairs(V, A, Kp)
    ov, oi = oracle.rerank(Q, X, cand, K, metric)
    np.testing.assert_array_equal(idx, oi)
    np.testing.assert_allclose(val, ov, rtol=1e-6, atol=1e-6)
