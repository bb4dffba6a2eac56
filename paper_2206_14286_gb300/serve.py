"""Continuous-batching search server over device-resident databases.

Requests (a query set of any size m, a database, K) arrive at any time. The
server keeps one FIFO of pending requests and a fixed number of *slots*
(CUDA streams). Whenever a slot is free it forms a batch: the oldest pending
request fixes the class (database, K); every other pending request of that
class joins, in arrival order, while the batch stays within `max_batch`
queries and the device-memory budget. The batch's queries are copied
host -> device into one contiguous block, searched in ONE knn_search pass
(PartialReduce + ExactRescoring + FP32 re-rank, all queries of the batch
side by side), and the results are copied back and split per request.
Requests that arrive while batches run are admitted as soon as a slot and
memory free up, so batches of different classes overlap on the device.

Memory admission: every batch's device buffers (staged queries, outputs,
search workspace) are carved from one arena of `hbm_budget` bytes allocated
at start-up; a batch is admitted only if its block fits, so the server never
allocates device memory while serving and never exceeds its budget. A request
too large for the whole arena is rejected (its `error` is set).

Each query's result depends only on that query (bins, rescoring and re-rank
are per query), so a request gets the same answer alone and in a mix.
"""
import collections
import time

import torch

from . import _lib
from ._lib import BINS, DTYPE, METRIC
from .search import Database

_ALIGN = 256


def _al(n):
    return (int(n) + _ALIGN - 1) // _ALIGN * _ALIGN


class Arena:
    """First-fit allocator over one preallocated device buffer (offsets only)."""

    def __init__(self, nbytes, device):
        self.size = _al(nbytes)
        self.buf = torch.empty(self.size, dtype=torch.uint8, device=device)
        self.free = [(0, self.size)]          # sorted, coalesced (offset, length)
        self.used = 0
        self.peak = 0

    def alloc(self, n):
        n = _al(max(int(n), 1))
        for k, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(k)
                else:
                    self.free[k] = (off + n, ln - n)
                self.used += n
                self.peak = max(self.peak, self.used)
                return off, n
        return None

    def release(self, block):
        off, n = block
        self.used -= n
        self.free.append((off, n))
        self.free.sort()
        merged = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged

    def view(self, off, nbytes, dtype, shape):
        return self.buf[off:off + nbytes].view(dtype).view(shape)


class Request:
    __slots__ = ("rid", "db", "q", "K", "t_arrival", "t_done", "val", "idx", "error")

    def __init__(self, rid, db, q, K, t_arrival):
        self.rid, self.db, self.q, self.K = rid, db, q, K
        self.t_arrival = t_arrival
        self.t_done = None
        self.val = self.idx = None
        self.error = None

    @property
    def done(self):
        return self.t_done is not None

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.t_arrival


class _Batch:
    __slots__ = ("reqs", "block", "event", "val_h", "idx_h", "slot", "M")


def plan_batch(pending, max_batch, need, alloc):
    """The next batch from the FIFO `pending`: the oldest request fixes the
    class (db, K); later requests of that class join in arrival order while
    the batch stays within max_batch queries. The batch shrinks from its tail
    until need(db, K, M) bytes can be allocated; if even the oldest request
    alone does not fit, nothing launches (it waits for memory).
    Returns (requests, M, block) or None. Host logic only."""
    if not pending:
        return None
    head = pending[0]
    name, K = head.db, head.K
    take, M = [], 0
    for r in pending:
        if r.db != name or r.K != K:
            continue
        m = r.q.shape[0]
        if take and M + m > max_batch:
            break
        take.append(r)
        M += m
    while take:
        block = alloc(need(name, K, M))
        if block is not None:
            return take, M, block
        if len(take) == 1:
            return None
        M -= take.pop().q.shape[0]
    return None


class Server:
    """dbs: {name: Database}; hbm_budget: bytes of the serving arena."""

    def __init__(self, dbs, hbm_budget, max_batch=2048, slots=3, recall_target=0.95,
                 rerank=2, bins="mod", round_L=128, clock=time.perf_counter):
        if not dbs:
            raise ValueError("no database")
        self.dbs = dict(dbs)
        for name, d in self.dbs.items():
            if not isinstance(d, Database):
                raise TypeError("%s is not a Database" % name)
        self.device = next(iter(self.dbs.values())).device
        self.arena = Arena(hbm_budget, self.device)
        self.max_batch = int(max_batch)
        self.recall_target, self.rerank, self.bins = recall_target, rerank, bins
        self.round_L = round_L
        self.clock = clock
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        self.busy = [None] * slots
        self._pinned = [None] * slots           # per-slot pinned result buffers
        self.pending = collections.deque()
        self.finished = []
        self._next_id = 0
        self._L = {}
        self.batches = 0
        self.failed_batches = 0
        self.max_in_flight = 0

    # -- planning ----------------------------------------------------------------
    def bins_for(self, name, K):
        key = (name, K)
        if key not in self._L:
            d = self.dbs[name]
            L = _lib.get().knn_plan_bins(d.N, K, self.recall_target, self.round_L)
            if L < 1:
                raise ValueError("no bin count for K=%d on %s" % (K, name))
            self._L[key] = int(L)
        return self._L[key]

    def _bytes(self, name, K, M):
        d = self.dbs[name]
        L = self.bins_for(name, K)
        ws = _lib.get().knn_search_workspace(d.N, d.D, DTYPE[d.dtype], METRIC[d.metric], M, K, L,
                                             BINS[self.bins], self.recall_target, self.rerank)
        if ws == 0:
            raise ValueError("unsupported request (db %s, M=%d, K=%d)" % (name, M, K))
        return _al(M * d.D * 4), _al(M * K * 4), _al(ws)

    def _need(self, name, K, M):
        q, o, ws = self._bytes(name, K, M)
        return q + 2 * o + ws

    # -- requests ----------------------------------------------------------------
    def submit(self, db, q, K, t_arrival=None):
        """Queue a request: q is an m x D float32 CPU tensor (pinned is faster)."""
        if db not in self.dbs:
            raise KeyError(db)
        d = self.dbs[db]
        if q.dim() != 2 or q.shape[1] != d.D or q.dtype != torch.float32 or q.is_cuda:
            raise ValueError("q must be an m x %d float32 host tensor" % d.D)
        r = Request(self._next_id, db, q.contiguous(), int(K),
                    self.clock() if t_arrival is None else t_arrival)
        self._next_id += 1
        if q.shape[0] == 0:
            r.val = torch.empty((0, K), dtype=torch.float32)
            r.idx = torch.empty((0, K), dtype=torch.int32)
            r.t_done = r.t_arrival
            self.finished.append(r)
            return r
        try:
            if self._need(db, r.K, q.shape[0]) > self.arena.size:
                raise MemoryError("request needs more than the serving budget")
        except (ValueError, MemoryError) as e:
            r.error = str(e)
            r.t_done = r.t_arrival
            self.finished.append(r)
            return r
        self.pending.append(r)
        return r

    # -- the loop ----------------------------------------------------------------
    def _retire(self):
        for s, b in enumerate(self.busy):
            if b is None or not b.event.query():
                continue
            now = self.clock()
            row = 0
            for r in b.reqs:
                m = r.q.shape[0]
                r.val = b.val_h[row:row + m].clone()
                r.idx = b.idx_h[row:row + m].clone()
                row += m
                r.t_done = now
                self.finished.append(r)
            self.arena.release(b.block)
            self.busy[s] = None

    def _form(self):
        got = plan_batch(self.pending, self.max_batch, self._need, self.arena.alloc)
        if got is not None:
            for r in got[0]:
                self.pending.remove(r)
        return got

    def _launch(self, slot, take, M, block):
        name, K = take[0].db, take[0].K
        d = self.dbs[name]
        L = self.bins_for(name, K)
        qb, ob, wsb = self._bytes(name, K, M)
        off = block[0]
        a = self.arena
        qd = a.view(off, M * d.D * 4, torch.float32, (M, d.D))
        vd = a.view(off + qb, M * K * 4, torch.float32, (M, K))
        idd = a.view(off + qb + ob, M * K * 4, torch.int32, (M, K))
        ws = a.buf[off + qb + 2 * ob:off + qb + 2 * ob + wsb]
        st = self.streams[slot]
        b = _Batch()
        b.reqs, b.block, b.slot, b.M = take, block, slot, M
        pin = self._pinned[slot]
        if pin is None or pin.numel() < 2 * M * K:
            pin = torch.empty(2 * max(M * K, self.max_batch * 16), dtype=torch.int32,
                              pin_memory=True)
            self._pinned[slot] = pin
        b.val_h = pin[:M * K].view(torch.float32).view(M, K)
        b.idx_h = pin[M * K:2 * M * K].view(M, K)
        with torch.cuda.stream(st):
            row = 0
            for r in take:
                m = r.q.shape[0]
                qd[row:row + m].copy_(r.q, non_blocking=True)
                row += m
            with torch.cuda.device(self.device):
                status = _lib.get().knn_search(*d._args(), qd.data_ptr(), M, K, L,
                                               BINS[self.bins], self.recall_target, self.rerank,
                                               vd.data_ptr(), idd.data_ptr(), ws.data_ptr(), wsb,
                                               st.cuda_stream)
            if status != _lib.KNN_OK:
                # nothing of the search was enqueued (or a launch failed): fail
                # the batch's requests once the staged copies are done
                st.synchronize()
                now = self.clock()
                err = "knn_search: " + _lib.get().knn_status_string(status).decode()
                for r in take:
                    r.error = err
                    r.t_done = now
                    self.finished.append(r)
                self.arena.release(block)
                self.failed_batches += 1
                return
            b.val_h.copy_(vd, non_blocking=True)
            b.idx_h.copy_(idd, non_blocking=True)
            b.event = torch.cuda.Event()
            b.event.record(st)
        self.busy[slot] = b
        self.batches += 1
        self.max_in_flight = max(self.max_in_flight, sum(x is not None for x in self.busy))

    def step(self):
        """Retire finished batches, then fill every free slot. Returns the
        number of batches launched."""
        self._retire()
        launched = 0
        for s in range(len(self.busy)):
            if self.busy[s] is not None:
                continue
            got = self._form()
            if got is None:
                break
            self._launch(s, *got)
            launched += 1
        return launched

    def idle(self):
        return not self.pending and all(b is None for b in self.busy)

    def drain(self):
        while not self.idle():
            self.step()

    def take_finished(self):
        out, self.finished = self.finished, []
        return out


def run_trace(server, trace, spin=True):
    """Replay (t_offset_s, db, q, K) arrivals in real time against `server`.
    Returns the finished requests (latency = completion - arrival)."""
    trace = sorted(trace, key=lambda x: x[0])
    t0 = server.clock()
    k = 0
    done = []
    while k < len(trace) or not server.idle():
        now = server.clock() - t0
        while k < len(trace) and trace[k][0] <= now:
            t, name, q, K = trace[k]
            server.submit(name, q, K, t_arrival=t0 + t)
            k += 1
        server.step()
        done.extend(server.take_finished())
        if not spin and k < len(trace) and server.idle():
            time.sleep(max(0.0, trace[k][0] - (server.clock() - t0)))
    done.extend(server.take_finished())
    return done


def latency_summary(reqs, wall_s):
    lat = sorted(r.latency for r in reqs if r.error is None)
    if not lat:
        return {}
    q = sum(r.q.shape[0] for r in reqs if r.error is None)

    def pct(p):
        return lat[min(len(lat) - 1, int(round(p * (len(lat) - 1))))] * 1e3

    return {"requests": len(lat), "queries": q, "queries_per_s": q / wall_s,
            "p50_ms": pct(0.50), "p99_ms": pct(0.99), "max_ms": lat[-1] * 1e3}
