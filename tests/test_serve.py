"""The continuous-batching server: host logic on the CPU (arena, batch
planning), and on the GPU the property the server promises -- each request's
result is the same alone and in the mix -- plus admission by memory, overlap
of batches, and failure handling with a fake failing call on the host."""
import collections

import numpy as np
import pytest
import torch

from paper_2206_14286_gb300 import serve as SV
from paper_2206_14286_gb300 import synth


# ----------------------------------------------------------------------------
# host logic (no GPU)
# ----------------------------------------------------------------------------
def test_arena_first_fit_and_coalescing():
    a = SV.Arena(10 * 256, "cpu")
    b1 = a.alloc(300)           # 512
    b2 = a.alloc(256)
    b3 = a.alloc(1)
    assert (b1, b2, b3) == ((0, 512), (512, 256), (768, 256))
    assert a.used == 1024 and a.alloc(10 * 256) is None
    a.release(b2)
    assert a.alloc(512) == (1024, 512)        # the 256 hole is too small
    assert a.alloc(200) == (512, 256)         # first fit fills the hole
    a.release(b1)
    a.release((512, 256))
    a.release(b3)
    a.release((1024, 512))
    assert a.free == [(0, 2560)] and a.used == 0
    assert a.peak == 1536


class _R:
    def __init__(self, db, m, K):
        self.db, self.K = db, K
        self.q = np.zeros((m, 1))


def test_plan_batch_class_order_and_limits():
    pend = collections.deque([_R("a", 5, 10), _R("b", 7, 10), _R("a", 6, 10), _R("a", 3, 100),
                              _R("a", 9, 10), _R("a", 2, 10)])
    need = lambda name, K, M: M * 100
    got = SV.plan_batch(pend, 16, need, lambda n: (0, n))
    take, M, blk = got
    assert [r.q.shape[0] for r in take] == [5, 6] and M == 11   # 9 more would pass 16
    assert all(r.db == "a" and r.K == 10 for r in take)
    # memory-limited: shrink from the tail until it fits
    got = SV.plan_batch(pend, 100, need, lambda n: (0, n) if n <= 1200 else None)
    assert [r.q.shape[0] for r in got[0]] == [5, 6]
    # even the head does not fit: nothing launches
    assert SV.plan_batch(pend, 100, need, lambda n: None) is None
    assert SV.plan_batch(collections.deque(), 100, need, lambda n: (0, n)) is None


def test_serving_trace_is_seeded_and_shaped():
    dbs = {"db1": (16, 4), "db2": (24, 4)}
    a = synth.serving_trace(300, 500.0, dbs, m_max=512)
    b = synth.serving_trace(300, 500.0, dbs, m_max=512)
    assert all(x[0] == y[0] and x[1] == y[1] and x[3] == y[3] and np.array_equal(x[2], y[2])
               for x, y in zip(a, b))
    ts = np.array([x[0] for x in a])
    assert np.all(np.diff(ts) > 0)
    ms = np.array([x[2].shape[0] for x in a])
    assert ms.min() >= 1 and ms.max() <= 512
    assert {x[3] for x in a} == {10, 100}
    assert all(x[2].shape[1] == dbs[x[1]][0] for x in a)
    # mean gap ~ 1/rate (Poisson), within 5 sigma
    gaps = np.diff(np.concatenate([[0.0], ts]))
    assert abs(gaps.mean() - 1 / 500.0) < 5 * (1 / 500.0) / np.sqrt(300)


# ----------------------------------------------------------------------------
# GPU
# ----------------------------------------------------------------------------
def _raw():
    X1 = synth.mixture(60000, 64, 64, 71)
    X2 = synth.mixture(90000, 96, 64, 72)
    return {"db1": (X1, "l2"), "db2": (X2, "ip")}


def _dbs():
    from tests.gpu_util import db
    raw = _raw()
    return {n: db(X, m, "bf16") for n, (X, m) in raw.items()}, \
        {"db1": (64, 64), "db2": (96, 64)}


def _alone(server, r):
    d = server.dbs[r.db]
    q = r.q.cuda()
    return d.search(q, r.K, L=server.bins_for(r.db, r.K), rerank=server.rerank,
                    bins=server.bins)


def _same(r, alone):
    """Every query of a batch is searched on its own (its bins, its rescoring,
    its re-rank), by the same kernels whatever the batch size: a request's
    result in the mix must equal its result alone, bit for bit."""
    av, ai = (t.cpu() for t in alone)
    assert torch.equal(r.idx, ai), r.rid
    assert torch.equal(r.val, av), r.rid
    return 0


@pytest.mark.gpu
def test_results_same_alone_and_in_mix():
    dbs, shapes = _dbs()
    # a burst: the first step fills every slot, later arrivals join as slots free up
    trace = synth.serving_trace(60, 2.0e5, shapes, m_max=256, seed=81)
    srv = SV.Server(dbs, hbm_budget=64 << 20, max_batch=512, slots=3)
    done = SV.run_trace(srv, [(t, n, torch.from_numpy(q).pin_memory(), K)
                              for t, n, q, K in trace])
    assert len(done) == 60 and all(r.error is None for r in done)
    assert srv.batches < 60                     # requests were batched together
    assert srv.max_in_flight >= 2               # several batches admitted at once
    for r in done:
        _same(r, _alone(srv, r))
    assert srv.arena.used == 0 and srv.arena.peak <= srv.arena.size


@pytest.mark.gpu
def test_served_results_match_the_oracle_per_class():
    """A mixed trace over both databases and both K; the first request of
    every (database, K) class, as the server returned it, against the FP64
    oracle's PartialReduce -> top-2K -> FP32 re-rank on the same queries
    (the parity rule of tests/parity.py with the BF16 kernel's tolerance)."""
    from tests.test_gpu_lowp import lowp_oracle_side, om
    from tests import parity as PT
    raw = _raw()
    dbs, shapes = _dbs()
    trace = synth.serving_trace(80, 2.0e5, shapes, m_max=256, seed=82)
    srv = SV.Server(dbs, hbm_budget=64 << 20, max_batch=512, slots=3)
    done = SV.run_trace(srv, [(t, n, torch.from_numpy(q).pin_memory(), K)
                              for t, n, q, K in trace])
    assert len(done) == 80 and all(r.error is None for r in done)
    assert srv.batches < 80
    first = {}
    for r in sorted(done, key=lambda r: r.rid):
        first.setdefault((r.db, r.K), r)
    assert len(first) == 4, sorted(first)
    for (name, K), r in sorted(first.items()):
        X, metric = raw[name]
        L = srv.bins_for(name, K)
        Q = r.q.numpy()
        o = lowp_oracle_side(X, Q, metric, "bf16", K, L, srv.rerank)
        gv, gi = r.val.numpy(), r.idx.numpy()
        frac = PT.check_search(gv, gi, o["ov"], o["oi"], o["S_lp"], o["S_f"], L, om(metric),
                               np.maximum(o["tol_d"], o["tol_df"]), o["dec2"])
        print("served %s K=%d L=%d m=%d: decided %.3f" % (name, K, L, Q.shape[0], frac))


@pytest.mark.gpu
def test_admission_by_memory_budget():
    dbs, shapes = _dbs()
    srv = SV.Server(dbs, hbm_budget=1 << 30, max_batch=4096, slots=4)
    srv_need = srv._need("db1", 10, 300)
    one = srv._need("db1", 10, 1000)
    # a budget that holds one 300-query batch but not two
    srv = SV.Server(dbs, hbm_budget=srv_need + srv_need // 2, max_batch=300, slots=4)
    g = np.random.Generator(np.random.PCG64(5))
    reqs = [srv.submit("db1", torch.from_numpy(g.standard_normal((300, 64)).astype(np.float32)),
                       10) for _ in range(4)]
    big = srv.submit("db1", torch.zeros((1000, 64)), 10)        # needs `one` > budget
    assert big.error and one > srv.arena.size
    srv.step()
    assert sum(b is not None for b in srv.busy) == 1            # memory admits one batch
    srv.drain()
    assert all(r.error is None and r.val.shape == (300, 10) for r in reqs)
    assert srv.max_in_flight == 1 and srv.arena.peak <= srv.arena.size
    for r in reqs:
        _same(r, _alone(srv, r))


@pytest.mark.gpu
def test_failed_call_fails_its_batch_only(monkeypatch):
    """Host-side fault injection: a fake knn_search that returns KNN_ECUDA for
    the db2 class; db1 requests still complete and memory is released."""
    dbs, shapes = _dbs()
    srv = SV.Server(dbs, hbm_budget=64 << 20, max_batch=512, slots=2)
    real = SV._lib.get()

    class Fake:
        def __getattr__(self, name):
            return getattr(real, name)

        def knn_search(self, *a):
            if a[5] == 96:              # D of db2
                return SV._lib.KNN_ECUDA
            return real.knn_search(*a)

    monkeypatch.setattr(SV._lib, "get", lambda: Fake())
    g = np.random.Generator(np.random.PCG64(6))
    r1 = [srv.submit("db1", torch.from_numpy(g.standard_normal((50, 64)).astype(np.float32)), 10)
          for _ in range(3)]
    r2 = [srv.submit("db2", torch.from_numpy(g.standard_normal((40, 96)).astype(np.float32)), 10)
          for _ in range(3)]
    srv.drain()
    assert all(r.error is None for r in r1)
    assert all(r.error and r.error.startswith("knn_search") for r in r2)
    assert srv.failed_batches >= 1 and srv.arena.used == 0
    monkeypatch.undo()
    for r in r1:
        _same(r, _alone(srv, r))
