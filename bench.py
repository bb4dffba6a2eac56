#!/usr/bin/env python
"""Benchmark of the fused search: queries/s at recall@10 >= 0.95.

One step = one knn_search call over the whole query batch: query preparation,
fused BF16 contraction + PartialReduce (tcgen05), ExactRescoring top-2K, FP32
re-rank to the top K. Default workload: 1,000,000 x 128 database rows from a
256-centre Gaussian mixture, 1024 queries from the same mixture, L2 metric,
K = 10, L from the recall law for 0.95 rounded up to the 128-row tile.

Reported beside it:
  * the plain FP32 path (SIMT contraction, same workload) with its roofline;
  * recall@10 against the exact FP32 search, p50/p99 step latency, the
    end-to-end rate through the host-buffer entry point, CUDA-graph replay;
  * the dominant kernel's roofline, and the paper's three-roof bound (Eq. 6)
    with gamma and the FFMA rate measured by microbenchmarks and C from the
    kernel's ncu instruction count;
  * score errors against FP64 on the original FP32 data;
  * the other workloads: FP8-E4M3 cosine 10M x 96 (K = 100) and the
    1M x 256 BF16 forward + backward (K = 32);
  * the serving loop over two resident databases (p50/p99);
  * the unfused GEMM -> HBM -> approx_max_k comparison (App. A.6);
  * the FP64 CPU oracle timed on bounded samples (all cores and one core).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU (torchrun): every rank runs an independent replica (the search does
not shard on one box); the value is the total over ranks.
"""
import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "queries/s at recall@10≥0.95 (fused BF16 vs plain FP32) and % of roofline; p99 ms"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# nominal dense tensor rates per GPU (PFLOP/s): FP8 / BF16 = 4.5 / 2.25
FP8_PER_BF16 = 2.0
# nominal FP32 CUDA-core rate: 152 SMs x 128 FMA lanes x 2 FLOP x 2.07 GHz
FFMA_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
KERNEL_CLASSES = ["prep", "k1", "k2", "k3"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mix_l2_1m")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp32-steps", type=int, default=10)
    ap.add_argument("--bins", default="mod", choices=["mod", "contiguous"])
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-unfused", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the E4M3 10M and the 1M x 256 backward workloads")
    ap.add_argument("--config-steps", type=int, default=10)
    ap.add_argument("--config-list", default="small,e4m3,grad",
                    help="which of the other workloads to run (comma list of small, e4m3, grad)")
    ap.add_argument("--config-scale", type=float, default=1.0,
                    help="shrink N and M of the e4m3 and grad workloads (small profiling runs)")
    ap.add_argument("--shard", action="store_true",
                    help="N-sharded search: the rows split over the ranks, two all-reduce MAX "
                         "exchanges per step (strong scaling); default: independent replicas")
    ap.add_argument("--serving-requests", type=int, default=1200)
    ap.add_argument("--serving-rates", default="1500,6000",
                    help="offered requests/s, one trace per rate")
    return ap.parse_args()


def job_rate(world, units_per_rank, local_ms, device=None):
    """Whole-job rate of independent replicas: every rank processed
    units_per_rank units in local_ms; the job took as long as the slowest
    rank (max over ranks). Returns (units/s over all ranks, job ms)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    job_ms = float(t.item())
    return world * units_per_rank / (job_ms / 1e3), job_ms


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


# ----------------------------------------------------------------------------
# nvidia-smi clock sampling during the timed region
# ----------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.2)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return None
        mx = max(r[1] for r in rows)
        loaded = [r for r in rows if r[0] > 0.5 * mx] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[2][k].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# CPU oracle (baseline and the reference arm)
# ----------------------------------------------------------------------------
class OracleRunner:
    """The FP64 oracle running the same method (PartialReduce, top-rerank*K,
    FP32-data re-rank) on a bounded sample of the workload's queries. The rows
    are stored as the library stores them (BF16 rounding or per-row E4M3, unit
    rows for cosine) and converted to float64 once, outside the timed runs."""

    def __init__(self, w, L, K, bins="mod", rerank=2):
        import oracle
        self.o = oracle
        self.bins, self.rerank = bins, rerank
        self.Q, self.L, self.K = w["Q"], L, K
        self.cos = w["metric"] == "cos"
        self.metric = "ip" if self.cos else w["metric"]
        self.dtype = w["dtype"]
        self.Xf, self.Xs = self._stored(w["X"])
        self.cursor = 0

    def _stored(self, A):
        o = self.o
        f = o.normalize_rows(A) if self.cos else np.asarray(A, np.float64)
        f = np.ascontiguousarray(f, np.float64)
        if self.dtype == "bf16":
            return f, o.bf16_round(f.astype(np.float32))
        if self.dtype == "e4m3":
            return f, o.e4m3_rows(f.astype(np.float32))[0]
        return f, f

    def run(self, n):
        o = self.o
        q = np.take(self.Q, np.arange(self.cursor, self.cursor + n) % self.Q.shape[0], axis=0)
        self.cursor = (self.cursor + n) % self.Q.shape[0]
        qf, qs = self._stored(q)
        t0 = time.perf_counter()
        V, A = o.partial_reduce(qs, self.Xs, self.L, self.metric, bins=self.bins)
        if self.rerank == 0:
            o.topk_pairs(V, A, self.K)
        else:
            _, cand = o.topk_pairs(V, A, min(self.rerank * self.K, self.L))
            o.rerank(qf, self.Xf, cand, self.K, self.metric)
        return time.perf_counter() - t0

    def size_for(self, seconds, cap):
        t = self.run(8)
        return int(max(8, min(cap, seconds / max(t / 8, 1e-6))))


def cpu_baseline(w, L, K, bins, seconds=4.0, rerank=2):
    """The oracle on all host cores and on one core: three runs each on a
    bounded sample of the queries (about `seconds` each), median."""
    import oracle
    oracle.build()
    runner = OracleRunner(w, L, K, bins, rerank)
    M, N = w["Q"].shape[0], w["X"].shape[0]
    cores = oracle.set_threads(0)
    try:
        n_all = runner.size_for(seconds, M)
        t_all = statistics.median(runner.run(n_all) for _ in range(3))
        oracle.set_threads(1)
        n_one = runner.size_for(seconds, M)
        t_one = statistics.median(runner.run(n_one) for _ in range(3))
    finally:
        oracle.set_threads(cores)
    return {"value": n_all / t_all, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": "%d of the %d queries against the full %d-row database (FP64), "
                      "median of 3 runs of %.1f s" % (n_all, M, N, t_all),
            "single_thread": {"value": n_one / t_one, "unit": "queries/s", "cores": 1,
                              "sample": "%d queries, median of 3 runs of %.1f s"
                                        % (n_one, t_one)}}


# ----------------------------------------------------------------------------
# helpers on the GPU side
# ----------------------------------------------------------------------------
def timed(fn, steps, warmup=2):
    """Mean ms per call of fn over `steps` calls, CUDA events on the current stream."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def profiled(lib, fn, reps):
    """Per kernel class of the library (query prep, K1, K2, K3): mean ms per
    launch and launches, from the library's event profiler on fn's stream."""
    import torch
    from paper_2206_14286_gb300 import _lib
    _lib.check(lib.knn_profile_enable(1))
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    _lib.check(lib.knn_profile_enable(0))
    out = {}
    for c, name in enumerate(KERNEL_CLASSES):
        tot = ctypes.c_double()
        n = ctypes.c_int64()
        _lib.check(lib.knn_profile_read(c, ctypes.byref(tot), ctypes.byref(n)))
        out[name] = {"ms_avg": tot.value / max(1, n.value), "launches": n.value}
    return out


def measure_rates(lib):
    """gamma (compare/select COPs per second) and the FP32 FFMA rate of this
    GPU, from the library's issue-rate microbenchmarks."""
    from paper_2206_14286_gb300 import _lib
    out = {}
    for name in ("minmax", "ffma"):
        r, ms = ctypes.c_double(), ctypes.c_double()
        _lib.check(lib.knn_measure_rate(_lib.RATE[name], 4096, ctypes.byref(r), ctypes.byref(ms),
                                        None))
        out[name] = {"ops_per_s": r.value, "ms": ms.value}
    return {"gamma_cops": out["minmax"]["ops_per_s"],
            "ffma_tflops": 2.0 * out["ffma"]["ops_per_s"] / 1e12,
            "how": "knn_measure_rate: FP32 min/max (gamma) and FFMA issue rates, 16 chains per "
                   "thread, 2048 threads per SM, CUDA events",
            "kernel_ms": {k: v["ms"] for k, v in out.items()}}


def scaled_mm_tflops():
    """Dense E4M3 GEMM rate of the library GEMM at 8192^3 (context for the
    FP8 roof; the roof itself is the measured BF16 peak x the nominal ratio)."""
    import torch
    try:
        n = 8192
        a = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device="cuda").to(torch.float8_e4m3fn).t()
        one = torch.ones((), device="cuda")
        ms = timed(lambda: torch._scaled_mm(a, b, scale_a=one, scale_b=one,
                                            out_dtype=torch.bfloat16), 10, 3)
        del a, b
        return 2.0 * n ** 3 / (ms / 1e3) / 1e12
    except (RuntimeError, TypeError, AttributeError) as e:
        return "unavailable: " + str(e)[:120]


def prepared_rows(d, rows):
    """FP64 values the contraction sees for the rows `rows` (CUDA int64
    tensor) of a prepared Database: BF16, E4M3 x scale, or FP32, decoded from
    the stored bytes."""
    import torch
    esz = {"f32": 4, "bf16": 2, "e4m3": 1, "e4m3t": 1}[d.dtype]
    b = d.lp.view(d.N, d.pitch * esz)[rows][:, :d.D * esz].contiguous()
    if d.dtype == "bf16":
        return b.view(torch.bfloat16).double()
    if d.dtype in ("e4m3", "e4m3t"):
        return b.view(torch.float8_e4m3fn).float().double() * d.scale[rows].double()[:, None]
    return b.view(torch.float32).double()


def score_errors(d, Xd, Qd, val, idx, metric, n=64, seed=7):
    """Errors against FP64 on the original FP32 data, over n sampled queries
    and their returned rows: of the low-precision score the contraction
    computes (FP64 on the stored values), and of the returned value. Both in
    the reported form (IP <q,x>, L2 |q-x|^2, COS cosine); `scaled` divides by
    the natural scale |q||x| (IP, COS) or |q|^2 + |x|^2 (L2)."""
    import torch
    from paper_2206_14286_gb300 import search as S
    M, K = idx.shape
    samp = np.random.Generator(np.random.PCG64(seed)).choice(M, size=min(n, M), replace=False)
    st = torch.from_numpy(samp).cuda()
    qsel = Qd[st].contiguous()
    # queries are stored per row (E4M3 per-row scales with either E4M3 database)
    qdt = "e4m3" if d.dtype == "e4m3t" else d.dtype
    dq = S.Database(qsel, metric=metric, dtype=qdt, keep_f32=False)
    qlp = prepared_rows(dq, torch.arange(len(samp), device="cuda"))
    rows = idx[st].long()
    xlp = prepared_rows(d, rows.reshape(-1)).view(len(samp), K, -1)
    xf = Xd[rows.reshape(-1)].double().view(len(samp), K, -1)
    qf = qsel.double()

    def score(q, x):
        if metric == "l2":
            return ((q[:, None, :] - x) ** 2).sum(-1)
        if metric == "cos":
            x = x / x.norm(dim=-1, keepdim=True)
            q = q / q.norm(dim=-1, keepdim=True)
        return (q[:, None, :] * x).sum(-1)

    exact = score(qf, xf)
    lowp = score(qlp, xlp) if metric != "cos" else (qlp[:, None, :] * xlp).sum(-1)
    ret = val[st].double()
    if metric == "l2":
        scale = (qf * qf).sum(-1)[:, None] + (xf * xf).sum(-1)
    elif metric == "cos":
        scale = torch.ones_like(exact)
    else:
        scale = qf.norm(dim=-1)[:, None] * xf.norm(dim=-1)

    def stats(e):
        a = e.abs()
        s = a / scale
        return {"max_abs": a.max().item(), "mean_abs": a.mean().item(),
                "max_scaled": s.max().item(), "mean_scaled": s.mean().item()}

    out = {"queries": len(samp), "rows_per_query": K,
           "contraction_%s" % d.dtype: stats(lowp - exact), "returned_fp32": stats(ret - exact),
           "reference": "FP64 on the original FP32 rows and queries (torch, float64)"}
    del dq
    return out


def recall_of(gi, ei):
    K = gi.shape[1]
    return float(np.mean([len(set(gi[i]) & set(ei[i])) / K for i in range(gi.shape[0])]))


def eq6(M, N, D, seconds, pi, beta, bytes_moved, gamma, C_design, C_measured=None):
    """The paper's three-roof bound (Eq. 6) for one launch of a fused
    contraction over M x N scores of length D, with C COPs per score."""
    from paper_2206_14286_gb300 import roofline as RF
    out = {"gamma_tcops": gamma / 1e12,
           "cop_budget_per_score": RF.cop_budget(D, gamma, pi)}
    for tag, C in (("design", C_design), ("measured", C_measured)):
        if C is None:
            continue
        r = RF.report(M, N, D, seconds, pi, beta, gamma, C, bytes_moved)
        out[tag] = {"C_cops_per_score": C, "I_MEM_flop_per_byte": r["I_MEM"],
                    "I_COP_flop_per_cop": r["I_COP"],
                    "roofs_tflops": {k: v / 1e12 for k, v in r["roofs"].items()},
                    "binding": r["binding"],
                    "fraction_of_attainable": r["fraction_of_attainable"]}
    return out


# ----------------------------------------------------------------------------
def main():
    args = parse()
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_2206_14286_gb300 import synth

    if args.impl == "reference":
        return reference_arm(args, rank)

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2206_14286_gb300 import search as S
    from paper_2206_14286_gb300 import _lib
    lib = _lib.get()
    if args.shard:
        return shard_main(args, world, rank, local)

    w = synth.workload(args.workload)
    X, Q, K, metric = w["X"], w["Q"], w["K"], w["metric"]
    N, D = X.shape
    M = Q.shape[0]
    L = S.plan_bins(N, K, w["recall"], round_to=128)
    L_min = S.plan_bins(N, K, w["recall"])
    rerank = w.get("rerank", 2)
    Xd = torch.from_numpy(X).cuda()
    Qd = torch.from_numpy(Q).cuda()
    db = S.Database(Xd, metric=metric, dtype=w["dtype"], keep_f32=True)
    val = torch.empty((M, K), dtype=torch.float32, device="cuda")
    idx = torch.empty((M, K), dtype=torch.int32, device="cuda")

    bins = args.bins

    def step():
        db.search(Qd, K, L=L, rerank=rerank, out=(val, idx), bins=bins)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    S.sync_status()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()

    # The timed region: K searches, two in flight on two streams (a workspace
    # slot and outputs each), as a serving loop runs them: one search's query
    # prep and rescoring run beside the other's contraction. Events on the
    # launching stream bracket all K; both streams join it before the end.
    streams2 = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs2 = [(val, idx), (torch.empty_like(val), torch.empty_like(idx))]

    def run2(n):
        cur = torch.cuda.current_stream()
        for st_ in streams2:
            st_.wait_stream(cur)
        for t in range(n):
            db.search(Qd, K, L=L, rerank=rerank, out=outs2[t % 2], bins=bins,
                      stream=streams2[t % 2], slot=t % 2)
        for st_ in streams2:
            cur.wait_stream(st_)

    run2(4)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    t_a, t_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_a.record()
    run2(args.steps)
    t_b.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = t_a.elapsed_time(t_b)
    value, total_ms = job_rate(world, M * args.steps, total_ms, device="cuda")
    # the same K searches one after another on one stream
    t_a.record()
    for _ in range(args.steps):
        step()
    t_b.record()
    torch.cuda.synchronize()
    single_value, single_ms = job_rate(world, M * args.steps, t_a.elapsed_time(t_b),
                                       device="cuda")
    # step latency (p50 / p99): a separate pass of at least 100 searches with
    # an event pair around each
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(max(100, args.steps))]
    for a, b in evs:
        a.record()
        step()
        b.record()
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in evs]

    # per-kernel times from the library's event profiler, in a separate pass
    # (its events are not part of the timed steps above)
    prof = profiled(lib, step, min(args.steps, 20))
    # prep, K1 (plus the ragged-row kernel when N mod L != 0), then K2 and K3,
    # or one launch of both when the library fuses them (no K3 launches)
    fused23 = prof["k3"]["launches"] == 0
    kernels = {"prep": prof["prep"], "k1_partial_reduce": prof["k1"]}
    if fused23:
        kernels["k2_k3_rescoring_rerank_fused"] = prof["k2"]
    else:
        kernels["k2_rescoring"], kernels["k3_rerank"] = prof["k2"], prof["k3"]
    launches_per_step = (3 if fused23 else 4) + (1 if bins == "mod" and N % L else 0)
    S.sync_status()

    # the same step replayed from a CUDA graph (knn_search allocates nothing,
    # so a caller can capture it once and replay it)
    graph = None
    try:
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr):
            step()
        g_ms = timed(gr.replay, args.steps, 3)
        graph = {"value": world * M / (g_ms / 1e3), "unit": "queries/s", "ms_per_step": g_ms}
        del gr
    except RuntimeError as e:  # capture refused: report why
        graph = {"unavailable": str(e)[:200]}
    S.sync_status()

    # recall@10 against the exact FP32 search on the same data, score errors
    dbx = S.Database(Xd, metric=metric, dtype="f32", keep_f32=True)
    _, ei = dbx.search_exact(Qd, K)
    ei = ei.cpu().numpy()
    recall = recall_of(idx.cpu().numpy(), ei)
    errors = score_errors(db, Xd, Qd, val, idx, metric)

    # the same BF16 search with the other bin map, same workload
    other = "mod" if bins == "contiguous" else "contiguous"
    vo = torch.empty_like(val)
    io = torch.empty_like(idx)
    ms_other = timed(lambda: db.search(Qd, K, L=L, rerank=rerank, bins=other, out=(vo, io)),
                     args.steps)
    recall_other = recall_of(io.cpu().numpy(), ei)

    # the plain FP32 path on the same workload (j mod L bins)
    v32 = torch.empty_like(val)
    i32 = torch.empty_like(idx)

    def step32():
        dbx.search(Qd, K, L=L, rerank=rerank, out=(v32, i32))
    ms32 = timed(step32, args.fp32_steps)
    prof32 = profiled(lib, step32, 3)
    recall32 = recall_of(i32.cpu().numpy(), ei)
    del dbx

    # end to end through the host-buffer entry point (pinned buffers): every
    # step copies its queries in and its results out. Two steps are in flight
    # on two streams (knn_search_host_async, a workspace and outputs each), so
    # one step's copies overlap the other's kernels; the clock stops once both
    # streams have finished. The synchronous call is timed beside it.
    qh = torch.from_numpy(Q).pin_memory()
    outs = [(torch.empty((M, K), dtype=torch.float32, pin_memory=True),
             torch.empty((M, K), dtype=torch.int32, pin_memory=True)) for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    e2e_steps = max(5, args.steps)

    def e2e_run(n, wait):
        for t in range(n):
            db.search_host(qh, K, L=L, rerank=rerank, out=outs[t % 2], bins=bins,
                           stream=streams[t % 2], wait=wait, slot=t % 2)
        for st_ in streams:
            st_.synchronize()
    e2e_run(4, False)
    e2e_run(3, True)
    t0 = time.perf_counter()
    e2e_run(e2e_steps, False)
    e2e_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    e2e_run(e2e_steps, True)
    e2e_sync_s = time.perf_counter() - t0
    S.sync_status()
    # whole-job rates: the slowest rank's wall clock
    e2e_value, _ = job_rate(world, M * e2e_steps, e2e_s * 1e3, device="cuda")
    e2e_sync_value, _ = job_rate(world, M * e2e_steps, e2e_sync_s * 1e3, device="cuda")
    e2e = {"value": e2e_value, "unit": "queries/s",
           "h2d_bytes_per_step": int(M * D * 4), "d2h_bytes_per_step": int(M * K * 8),
           "mode": "knn_search_host_async, two steps in flight on two streams",
           "synchronous": {"value": e2e_sync_value,
                           "mode": "knn_search_host, one step at a time"}}

    # roofline of the dominant kernel (K1), and of the FP32 path's K1
    pk, pk_kind = peaks()
    rates = measure_rates(lib)
    k1_ms = prof["k1"]["ms_avg"]
    flops = 2.0 * M * N * D
    achieved = flops / (k1_ms / 1e3) / 1e12
    peak = pk["bf16_tflops"]
    k1_bytes = N * D * 2 + (N * 4 if metric == "l2" else 0) + M * D * 2
    fields = profile_fields("k1_tcs_mix_l2_1m.md", "k1_tcs.cu", M, N, D, bins)
    traffic = int(fields["dram bytes per launch"]) if fields else None
    alu = float(fields["alu warp instructions per launch"]) if fields and \
        "alu warp instructions per launch" in fields else None
    C_meas = 32.0 * alu / (M * N) if alu else None
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": "%s bf16 dense burst (MEASURED_PEAKS.json)" % pk_kind,
            "kernel": ("k1_tcs_kernel: fused BF16 contraction + PartialReduce, contiguous bins"
                       if bins == "contiguous" else
                       "k1_tcs_kernel (+ k1_tcs_tail for the N mod L ragged rows): fused BF16 "
                       "contraction + PartialReduce, j mod L bins"),
            "algorithmic": "2*M*N*D = %.4g FLOP per launch" % flops,
            "eq6": dict(eq6(M, N, D, k1_ms / 1e3, peak * 1e12, pk["hbm_gbs"] * 1e9,
                            traffic or k1_bytes, rates["gamma_cops"], 1.0 / 16.0, C_meas),
                        C_note="design: one ALU compare per 16-score maximum (tcgen05.ld.red); "
                               "measured: 32 x ALU-pipe warp instructions per score from the "
                               "kernel's ncu capture, which also counts the polling of "
                               "its barrier waits"),
            "hbm_context": {"algorithmic_bytes": k1_bytes,
                            "achieved_gbs": k1_bytes / (k1_ms / 1e3) / 1e9,
                            "peak_gbs": pk["hbm_gbs"]}}
    k1_32 = prof32["k1"]["ms_avg"]
    fp32_roof = {"bound": "alu", "kernel": "k1_simt_kernel (FP32 FFMA contraction + PartialReduce)",
                 "achieved": flops / (k1_32 / 1e3) / 1e12, "unit": "TFLOP/s",
                 "peak_measured_ffma": rates["ffma_tflops"],
                 "peak_nominal_ffma": FFMA_NOMINAL_TFLOPS,
                 "frac": flops / (k1_32 / 1e3) / 1e12 / rates["ffma_tflops"],
                 "k1_ms": k1_32}

    serving = None if args.no_serving else serving_leg(args, db, w)
    unfused = None if args.no_unfused else unfused_leg(Xd, Qd, K, L)
    configs = None
    if not args.no_configs:
        del Xd, Qd
        torch.cuda.empty_cache()
        wanted = set(args.config_list.split(","))
        # the oracle baselines of the legs: rank 0 of a single-GPU run only
        args.leg_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
        configs = {}
        if "small" in wanted:
            configs["f32_ip_16k"] = small_leg(args, lib)
        if "e4m3" in wanted:
            configs["fp8_e4m3_cos_10m"] = e4m3_leg(args, lib, pk, rates)
        if "grad" in wanted:
            configs["bf16_ip_grad_1m"] = grad_leg(args, lib, pk)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, L, K, bins)

    if rank == 0:
        sm = sorted(step_ms)
        line = {"metric": METRIC,
                "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16", "data": "synthetic", "config": config_of(w, L, L_min, bins),
                "recall_at_10": recall,
                "score_error": errors,
                "other_bins": {"bins": other, "value": world * M / (ms_other / 1e3),
                               "unit": "queries/s", "ms_per_step": ms_other,
                               "recall_at_10": recall_other},
                "p50_ms": sm[len(sm) // 2], "p99_ms": sm[min(len(sm) - 1, int(0.99 * len(sm)))],
                "latency_samples": len(sm),
                "streams": 2,
                "single_stream": {"value": single_value, "unit": "queries/s",
                                  "ms_per_step": single_ms / args.steps},
                "fp32_path": {"value": world * M / (ms32 / 1e3), "unit": "queries/s",
                              "ms_per_step": ms32, "recall_at_10": recall32,
                              "roofline": fp32_roof},
                "kernels": kernels, "roofline": roof, "e2e": e2e,
                "rates": dict(rates, fp8_scaled_mm_tflops=scaled_mm_tflops()),
                "graph_replay": graph,
                "configs": configs,
                "serving": serving,
                "unfused_baseline": unfused,
                "gpu_launches": launches_per_step * args.steps, "clocks": clk,
                "cpu_baseline": cpu}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def shard_main(args, world, rank, local):
    """The N-sharded search (knn_shard_*): rank r holds rows
    shard_bounds(N, world, L)[r] of the workload's database, every rank takes
    the whole query batch, and a step is PartialReduce on the shard, an
    all-reduce MAX of the M x L keys, rescoring of the candidates the shard
    holds, an all-reduce MAX of the M x Kp keys and the top K. Total work is
    fixed as the ranks grow (strong scaling); value = queries / step time
    (max over ranks)."""
    import torch
    import torch.distributed as dist
    from paper_2206_14286_gb300 import search as S, shard as SH, synth
    w = synth.workload(args.workload)
    X, Q, K, metric = w["X"], w["Q"], w["K"], w["metric"]
    N, D = X.shape
    M = Q.shape[0]
    L = S.plan_bins(N, K, w["recall"], round_to=128)
    rerank = w.get("rerank", 2)
    row0, n = SH.shard_bounds(N, world, L)[rank]
    part = SH.DatabaseShard(torch.from_numpy(X[row0:row0 + n]).cuda(), row0, N, metric,
                            w["dtype"])
    Qd = torch.from_numpy(Q).cuda()
    ar = SH.dist_allreduce_max()
    out = {}

    def step():
        out["r"] = SH.sharded_search(part, Qd, K, L, rerank, ar)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    S.sync_status()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        step()
    b.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    t = torch.tensor([a.elapsed_time(b)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    job_ms = float(t.item())
    value = M * args.steps / (job_ms / 1e3)
    recall = None
    if world == 1:
        dbx = S.Database(torch.from_numpy(X).cuda(), metric=metric, dtype="f32")
        _, ei = dbx.search_exact(Qd, K)
        recall = recall_of(out["r"][1].cpu().numpy(), ei.cpu().numpy())
    if rank == 0:
        cfg = config_of(w, L, bins="mod")
        cfg["parallelism"] = "shard%d" % world
        cfg["shard_rows"] = n
        print(json.dumps({"metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": job_ms / args.steps, "higher_is_better": True,
                          "scaling": "strong", "vs_baseline": None, "dtype": w["dtype"],
                          "data": "synthetic", "config": cfg, "recall_at_10": recall,
                          # per step: prep, K1 (+ ragged rows), bin merge, key conversion;
                          # key conversion, K2, FP32 scoring; key conversion, K2, pairs
                          "gpu_launches": args.steps * (10 + (1 if n % L else 0) +
                                                        (1 if metric == "cos" else 0)),
                          "clocks": clk}))
    if world > 1:
        dist.destroy_process_group()
    return 0


def reference_arm(args, rank):
    """The FP64 oracle on the host cores, on the bench's workload and metric."""
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    from oracle import recall as R
    from paper_2206_14286_gb300 import synth
    w = synth.workload(args.workload)
    K = w["K"]
    L = min(w["X"].shape[0], -(-R.min_bins(K, w["recall"]) // 128) * 128)
    runner = OracleRunner(w, L, K, args.bins)
    n = runner.size_for(max(0.5, 120.0 / max(1, args.steps + args.warmup)), 256)
    per = []
    nq = 0
    for s in range(args.warmup + args.steps):
        t = runner.run(n)
        if s >= args.warmup:
            per.append((n, t))
            nq += n
    tot = sum(t for _, t in per)
    value = nq / tot
    cores = oracle.set_threads(0)
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(per),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(w, L, bins=args.bins),
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores,
                             "kind": "oracle",
                             "sample": "%d queries per step of the %d-query batch, full %d-row "
                                       "database" % (per[0][0], w["Q"].shape[0],
                                                     w["X"].shape[0])},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def small_leg(args, lib):
    """The plain FP32 case: 16,384 x 128 i.i.d. N(0,1) rows, M = 64 queries,
    inner product, K = 10, L = 1024 (no re-rank: the rows are FP32), and the
    exact search beside it; a launch-latency case, timed over 200 calls, with
    the oracle's full run (all 64 queries) as its CPU baseline."""
    import torch
    from paper_2206_14286_gb300 import search as S, synth
    w = synth.workload("iid_ip_16k")
    X, Q, K, L = w["X"], w["Q"], w["K"], w["L"]
    M = Q.shape[0]
    Xd = torch.from_numpy(X).cuda()
    Qd = torch.from_numpy(Q).cuda()
    d = S.Database(Xd, metric="ip", dtype="f32")
    v = torch.empty((M, K), dtype=torch.float32, device="cuda")
    i = torch.empty((M, K), dtype=torch.int32, device="cuda")
    ms = timed(lambda: d.search(Qd, K, L=L, rerank=0, out=(v, i)), 200, 10)
    ms_exact = timed(lambda: d.search_exact(Qd, K), 200, 10)
    _, ei = d.search_exact(Qd, K)
    S.sync_status()
    out = {"workload": "iid N(0,1) inner product N=%d D=%d M=%d K=%d, FP32" % (X.shape + (M, K)),
           "L": L, "value": M / (ms / 1e3), "unit": "queries/s", "ms_per_step": ms,
           "recall_at_10": recall_of(i.cpu().numpy(), ei.cpu().numpy()),
           "exact": {"value": M / (ms_exact / 1e3), "ms_per_step": ms_exact},
           "bound": "launch latency (0.27 GFLOP per call)"}
    if args.leg_cpu:
        import oracle
        oracle.build()
        runner = OracleRunner(w, L, K, "mod", rerank=0)
        cores = oracle.set_threads(0)
        try:
            t_all = statistics.median(runner.run(M) for _ in range(3))
            oracle.set_threads(1)
            t_one = statistics.median(runner.run(M) for _ in range(3))
        finally:
            oracle.set_threads(cores)
        out["cpu_baseline"] = {"value": M / t_all, "unit": "queries/s", "cores": cores,
                               "kind": "oracle", "sample": "all %d queries, median of 3" % M,
                               "single_thread": {"value": M / t_one, "unit": "queries/s",
                                                 "cores": 1}}
    del d, Xd, Qd
    torch.cuda.empty_cache()
    return out


def e4m3_leg(args, lib, pk, rates):
    """FP8-E4M3 with per-row scales, cosine, 10,000,000 x 96 rows from a
    1024-centre mixture, M = 10,000 queries, K = 100, L = 8192, FP32 re-rank
    of 8K bin winners; recall@100 against exact FP32 search on 2000 sampled
    queries; the BF16 path on the same workload beside it."""
    import torch
    from paper_2206_14286_gb300 import search as S, synth
    w = synth.workload("mix_cos_10m", scale=args.config_scale)
    X, Q, K = w["X"], w["Q"], w["K"]
    N, D = X.shape
    M = Q.shape[0]
    L, rr = w["L"], w["rerank"]
    Xd = torch.from_numpy(X).cuda()
    Qd = torch.from_numpy(Q).cuda()
    del X
    d8 = S.Database(Xd, metric="cos", dtype="e4m3")
    v = torch.empty((M, K), dtype=torch.float32, device="cuda")
    i = torch.empty((M, K), dtype=torch.int32, device="cuda")

    def step():
        d8.search(Qd, K, L=L, rerank=rr, out=(v, i))
    ms = timed(step, args.config_steps, 3)
    prof = profiled(lib, step, 3)
    S.sync_status()
    samp = np.random.Generator(np.random.PCG64(11)).choice(M, min(2000, M), replace=False)
    st = torch.from_numpy(samp).cuda()
    dx = S.Database(Xd, metric="cos", dtype="f32")
    _, ei = dx.search_exact(Qd[st].contiguous(), K)
    del dx
    torch.cuda.empty_cache()
    ei = ei.cpu().numpy()
    rec = recall_of(i[st].cpu().numpy(), ei)
    errors = score_errors(d8, Xd, Qd, v, i, "cos", n=32)
    flops = 2.0 * M * N * D
    k1 = prof["k1"]["ms_avg"]
    fp8_peak = FP8_PER_BF16 * pk["bf16_tflops"]
    out = {"workload": "gaussian-mixture-1024c cosine N=%d D=%d M=%d K=%d, FP8-E4M3 per-row "
                       "scales" % (N, D, M, K),
           "L": L, "rerank": "FP32 top-%dK" % rr, "value": M / (ms / 1e3),
           "unit": "queries/s", "ms_per_step": ms, "recall_at_100": rec,
           "recall_sample": "%d queries vs exact FP32 search" % len(samp),
           "kernels": {"prep": prof["prep"], "k1_partial_reduce": prof["k1"],
                       "k2_rescoring": prof["k2"], "k3_rerank": prof["k3"]},
           "roofline": {"bound": "tensor", "kernel": "k1_tc_kernel (E4M3 tcgen05 kind::f8f6f4, "
                                                    "packed-key PartialReduce)",
                        "achieved": flops / (k1 / 1e3) / 1e12, "unit": "TFLOP/s",
                        "peak": fp8_peak,
                        "peak_source": "measured BF16 burst x 2 (nominal FP8/BF16 ratio)",
                        "frac": flops / (k1 / 1e3) / 1e12 / fp8_peak,
                        "eq6": eq6(M, N, D, k1 / 1e3, fp8_peak * 1e12, pk["hbm_gbs"] * 1e9,
                                   N * (D + 4) + M * D, rates["gamma_cops"], 2.0)},
           "score_error": errors}
    # E4M3 with one database-wide scale: raw dot products of different rows
    # compare directly, so the BF16 kernel's design (one compare per 16 rows)
    # runs with E4M3 MMAs; same L and re-rank
    del d8
    torch.cuda.empty_cache()
    dt = S.Database(Xd, metric="cos", dtype="e4m3t")

    def step_t():
        dt.search(Qd, K, L=L, rerank=rr, out=(v, i))
    ms_t = timed(step_t, args.config_steps, 3)
    prof_t = profiled(lib, step_t, 3)
    S.sync_status()
    k1_t = prof_t["k1"]["ms_avg"]
    out["e4m3_database_scale"] = {
        "workload": "the same rows, FP8-E4M3 with one database-wide scale (max |x| / 448)",
        "L": L, "rerank": "FP32 top-%dK" % rr, "value": M / (ms_t / 1e3), "unit": "queries/s",
        "ms_per_step": ms_t, "recall_at_100": recall_of(i[st].cpu().numpy(), ei),
        "kernels": {"prep": prof_t["prep"], "k1_partial_reduce": prof_t["k1"],
                    "k2_rescoring": prof_t["k2"], "k3_rerank": prof_t["k3"]},
        "roofline": {"bound": "tensor", "kernel": "k1_tcs_kernel (E4M3 tcgen05 kind::f8f6f4, "
                                                 "tcgen05.ld.red.max PartialReduce)",
                     "achieved": flops / (k1_t / 1e3) / 1e12, "unit": "TFLOP/s",
                     "peak": fp8_peak,
                     "peak_source": "measured BF16 burst x 2 (nominal FP8/BF16 ratio)",
                     "frac": flops / (k1_t / 1e3) / 1e12 / fp8_peak},
        "score_error": score_errors(dt, Xd, Qd, v, i, "cos", n=32)}
    del dt
    torch.cuda.empty_cache()
    # the BF16 path on the same rows: L from the recall law, 2K re-rank
    d16 = S.Database(Xd, metric="cos", dtype="bf16")
    L16 = S.plan_bins(N, K, w["recall"], round_to=128)

    def step16():
        d16.search(Qd, K, L=L16, rerank=2, out=(v, i))
    ms16 = timed(step16, args.config_steps, 3)
    k1_16 = profiled(lib, step16, 3)["k1"]["ms_avg"]
    out["bf16_same_workload"] = {"L": L16, "rerank": "FP32 top-2K", "value": M / (ms16 / 1e3),
                                 "ms_per_step": ms16, "unit": "queries/s",
                                 "recall_at_100": recall_of(i[st].cpu().numpy(), ei),
                                 "k1_ms": k1_16,
                                 "k1_frac_of_bf16_peak": flops / (k1_16 / 1e3) / 1e12 /
                                 pk["bf16_tflops"]}
    S.sync_status()
    del d16, Xd, Qd
    torch.cuda.empty_cache()
    if args.leg_cpu:
        out["cpu_baseline"] = cpu_baseline(w, L, K, "mod", seconds=2.0, rerank=rr)
    return out


def grad_leg(args, lib, pk):
    """The differentiation workload: BF16 inner product, 1,000,000 x 256
    N(0, 1/D) rows, M = 4096, K = 32; forward search, then knn_backward of
    seeded weights on the K values (dQ gather, dX scatter-add; dX dense and
    zero-filled as torch's autograd needs it, and added into an existing dX)."""
    import torch
    from paper_2206_14286_gb300 import search as S, synth
    w = synth.workload("iid_ip_grad_1m", scale=args.config_scale)
    X, Q, K = w["X"], w["Q"], w["K"]
    N, D = X.shape
    M = Q.shape[0]
    L = S.plan_bins(N, K, w["recall"], round_to=128)
    Xd = torch.from_numpy(X).cuda()
    Qd = torch.from_numpy(Q).cuda()
    d = S.Database(Xd, metric="ip", dtype="bf16", keep_f32=True)
    v = torch.empty((M, K), dtype=torch.float32, device="cuda")
    i = torch.empty((M, K), dtype=torch.int32, device="cuda")

    def fwd():
        d.search(Qd, K, L=L, rerank=2, out=(v, i))
    ms_f = timed(fwd, args.config_steps, 3)
    prof = profiled(lib, fwd, 3)
    g = torch.from_numpy(synth.targets(M, K)).cuda()
    dxb = torch.zeros((N, D), dtype=torch.float32, device="cuda")
    ms_b = timed(lambda: d.backward(Qd, i, g, dx=dxb, zero_dx=True), args.config_steps, 2)
    ms_b_acc = timed(lambda: d.backward(Qd, i, g, dx=dxb, zero_dx=False), args.config_steps, 2)
    ms_dq = timed(lambda: d.backward(Qd, i, g, want_dx=False), args.config_steps, 2)
    ms_b_at = timed(lambda: d.backward(Qd, i, g, dx=dxb, zero_dx=True, atomic=True),
                    args.config_steps, 2)
    ms_b_acc_det = timed(lambda: d.backward(Qd, i, g, dx=dxb, zero_dx=False, deterministic=True),
                         args.config_steps, 2)
    S.sync_status()
    touched = int(torch.unique(i).numel())
    flops = 2.0 * M * N * D
    k1 = prof["k1"]["ms_avg"]
    gather = M * K * D * 4 + 2 * M * D * 4 + M * K * 8
    sparse = gather + 2 * touched * D * 4
    dense = N * D * 4
    out = {"workload": "iid N(0,1/D) inner product N=%d D=%d M=%d K=%d, BF16" % (N, D, M, K),
           "L": L, "forward": {"value": M / (ms_f / 1e3), "unit": "queries/s",
                               "ms_per_step": ms_f, "k1_ms": k1,
                               "roofline": {"bound": "tensor",
                                            "achieved": flops / (k1 / 1e3) / 1e12,
                                            "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                                            "frac": flops / (k1 / 1e3) / 1e12 /
                                            pk["bf16_tflops"]}},
           "backward": {"ms_dense_dx": ms_b, "ms_accumulate_dx": ms_b_acc, "ms_dq_only": ms_dq,
                        "ms_dense_dx_atomic": ms_b_at,
                        "ms_accumulate_dx_deterministic": ms_b_acc_det,
                        "touched_rows": touched,
                        "algorithmic_bytes": {"dense": dense + gather, "accumulate": sparse},
                        "roofline": {"bound": "hbm", "unit": "GB/s", "peak": pk["hbm_gbs"],
                                     "achieved_dense": (dense + gather) / (ms_b / 1e3) / 1e9,
                                     "frac_dense": (dense + gather) / (ms_b / 1e3) / 1e9 /
                                     pk["hbm_gbs"],
                                     "achieved_accumulate": sparse / (ms_b_acc / 1e3) / 1e9,
                                     "frac_accumulate": sparse / (ms_b_acc / 1e3) / 1e9 /
                                     pk["hbm_gbs"]},
                        "bytes_model": "dense: every dX row written once N*D*4, gathered rows "
                                       "M*K*D*4, q read + dq write 2*M*D*4, idx + g M*K*8; "
                                       "accumulate: the same without the N*D*4, plus read and "
                                       "write of the touched dX rows 2*rows*D*4",
                        "dx_modes": "ms_dense_dx: the row path (each dX row written once, "
                                    "entries in order; deterministic); ms_dense_dx_atomic: zero "
                                    "fill + FP32 atomics; ms_accumulate_dx: FP32 atomics into "
                                    "the existing dX; ms_accumulate_dx_deterministic: the row "
                                    "path adding into it"},
           "score_error": score_errors(d, Xd, Qd, v, i, "ip", n=64)}
    del d, Xd, Qd, dxb
    torch.cuda.empty_cache()
    if args.leg_cpu:
        out["forward"]["cpu_baseline"] = cpu_baseline(w, L, K, "mod", seconds=2.0)
    return out


def unfused_leg(Xd, Qd, K, L):
    """The fusion argument (App. A.6) on this GPU: the same inner-product
    search done unfused -- a cuBLAS BF16 GEMM writes the M x N score matrix
    to HBM, then approx_max_k reads it back (bins, top-K) -- against the fused
    search (PartialReduce inside the contraction, ExactRescoring, re-rank of
    the K winners). Same rows and queries as the main workload, BF16, K, L."""
    import torch
    from paper_2206_14286_gb300 import search as S
    M, N = Qd.shape[0], Xd.shape[0]
    db_ip = S.Database(Xd, metric="ip", dtype="bf16", keep_f32=True)
    Xb, Qb = Xd.to(torch.bfloat16), Qd.to(torch.bfloat16)
    scores = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
    gemm_ms = timed(lambda: torch.matmul(Qb, Xb.t(), out=scores), 5)
    amk_ms = timed(lambda: S.approx_max_k(scores, K, L=L), 5)
    unfused_ms = timed(lambda: S.approx_max_k(torch.matmul(Qb, Xb.t(), out=scores), K, L=L), 5)
    fused_ms = timed(lambda: db_ip.search(Qd, K, L=L, rerank=1), 5)
    sbytes = M * N * 2
    out = {"workload": "IP, BF16, N=%d x D=%d, M=%d, K=%d, L=%d" % (N, Xd.shape[1], M, K, L),
           "gemm_ms": gemm_ms, "approx_max_k_ms": amk_ms,
           "approx_max_k_gbs": sbytes / (amk_ms / 1e3) / 1e9,
           "score_matrix_bytes": sbytes, "unfused_ms": unfused_ms, "fused_ms": fused_ms,
           "fused_speedup": unfused_ms / fused_ms,
           "paper": "24.9 ms unfused vs 2.6 ms fused (9.6x) on one TPU v4 core, App. A.6"}
    del scores, Xb, Qb, db_ip
    torch.cuda.empty_cache()
    return out


def serving_leg(args, db1, w1):
    """Continuous batching over two resident databases: the bench's own
    (1,000,000 x 128, L2) and a 4,000,000 x 768 inner-product Gaussian mixture
    (256 centres, drawn on the device from a fixed seed). Seeded Poisson
    arrivals, m log-uniform in [1, 512], K in {10, 100}, a 4 GiB serving arena.
    Latency = completion - arrival, wall clock."""
    import torch
    from paper_2206_14286_gb300 import search as S, serve as SV, synth
    X2 = synth.mixture_device(4_000_000, 768, 256, 11, "cuda")
    db2 = S.Database(X2, metric="ip", dtype="bf16")
    n1, n2 = "db1_1m_x128_l2", "db2_4m_x768_ip"
    dbs = {n1: db1, n2: db2}
    shapes = {n1: (128, 256), n2: (768, 256)}
    runs = []
    for rate in [float(r) for r in args.serving_rates.split(",") if r]:
        trace = synth.serving_trace(args.serving_requests, rate, shapes)
        trace = [(t, n, torch.from_numpy(q).pin_memory(), K) for t, n, q, K in trace]
        srv = SV.Server(dbs, hbm_budget=4 << 30, max_batch=4096, slots=3)
        # warm-up: one request of every class, then the timed trace
        for n in dbs:
            for K in (10, 100):
                srv.submit(n, torch.zeros((8, shapes[n][0])), K)
        srv.drain()
        srv.take_finished()
        srv.batches = srv.max_in_flight = 0
        t0 = time.perf_counter()
        done = SV.run_trace(srv, trace)
        wall = time.perf_counter() - t0
        out = SV.latency_summary(done, wall)
        out.update({"offered_requests_per_s": rate, "batches": srv.batches,
                    "max_in_flight": srv.max_in_flight,
                    "errors": sum(r.error is not None for r in done)})
        runs.append(out)
    S.sync_status()
    del db2, X2
    torch.cuda.empty_cache()
    return {"databases": "1M x 128 L2 and 4M x 768 IP, BF16, FP32 re-rank of 2K",
            "arrivals": "seeded Poisson, m log-uniform in [1, 512], K in {10, 100}",
            "runs": runs}


def config_of(w, L, L_min=None, bins="mod"):
    X, Q = w["X"], w["Q"]
    return {"workload": "gaussian-mixture-256c L2 N=%d D=%d M=%d K=%d" % (X.shape[0], X.shape[1],
                                                                          Q.shape[0], w["K"]),
            "N": X.shape[0], "D": X.shape[1], "global_batch": Q.shape[0], "K": w["K"],
            "L": L, "L_min_eq14": L_min, "bins": bins, "metric": w["metric"],
            "rerank": "FP32 top-%dK" % w.get("rerank", 2),
            "l2_flush": "inputs larger than L2 (database %d MB in BF16 streamed every step)"
                        % (X.shape[0] * X.shape[1] * 2 // 2 ** 20),
            "parallelism": "replicas"}


def profile_fields(name, source, M, N, D, bins="mod"):
    """Fields of a committed ncu summary under profiles/ when it was taken on
    the current kernel source (sha256 prefix) and the same launch shape, else
    None. The summary holds lines "- <field>: <value>", among them
    "kernel source sha256", "bins", "M", "N", "D", "dram bytes per launch"
    and "alu warp instructions per launch"."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    fields = {}
    for line in open(p):
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    h = hashlib.sha256(open(os.path.join(ROOT, "paper_2206_14286_gb300", "csrc", source),
                            "rb").read()).hexdigest()[:16]
    try:
        if (fields.get("kernel source sha256") != h or fields.get("bins") != bins
                or int(fields.get("M", -1)) != M or int(fields.get("N", -1)) != N
                or int(fields.get("D", -1)) != D or "dram bytes per launch" not in fields):
            return None
    except ValueError:
        return None
    return fields


if __name__ == "__main__":
    sys.exit(main())
