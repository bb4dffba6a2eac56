#!/usr/bin/env python
"""Benchmark of the fused search: queries/s at recall@10 >= 0.95.

One step = one knn_search call over the whole query batch: query preparation,
fused BF16 contraction + PartialReduce (tcgen05), ExactRescoring top-2K, FP32
re-rank to the top K. Default workload: 1,000,000 x 128 database rows from a
256-centre Gaussian mixture, 1024 queries from the same mixture, L2 metric,
K = 10, L from the recall law for 0.95 rounded up to the 128-row tile.

Reported beside it: the plain FP32 path (SIMT contraction, same workload),
recall@10 against the exact FP32 search, p50/p99 step latency, the end-to-end
rate through the host-buffer entry point, the dominant kernel's roofline and
the FP64 CPU oracle timed on a bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU (torchrun): every rank runs an independent replica (the search does
not shard on one box); the value is the total over ranks.
"""
import argparse
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

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}


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
    ap.add_argument("--serving-requests", type=int, default=1200)
    ap.add_argument("--serving-rates", default="1500,6000",
                    help="offered requests/s, one trace per rate")
    return ap.parse_args()


def eq6_block(M, N, D, k1_ms, pk, bytes_moved):
    """The paper's three-roof bound (Eq. 6) for K1 on this GPU: pi and beta
    measured, gamma from unit counts x clock (ALU pipe), C from the kernel's
    design: one compare per 16-score maximum (tcgen05.ld.red), plus the
    searches of new bests, which depend on the data and are not counted."""
    from paper_2206_14286_gb300 import roofline as RF
    C = 1.0 / 16.0
    r = RF.report(M, N, D, k1_ms / 1e3, pk["bf16_tflops"] * 1e12, pk["hbm_gbs"] * 1e9,
                  RF.gb300_gamma("alu"), C, bytes_moved)
    return {"C_design_alu_cops_per_score": C, "I_MEM_flop_per_byte": r["I_MEM"],
            "I_COP_flop_per_cop": r["I_COP"],
            "roofs_tflops": {k: v / 1e12 for k, v in r["roofs"].items()},
            "binding": r["binding"], "fraction_of_attainable": r["fraction_of_attainable"],
            "gamma_alu_tcops": RF.gb300_gamma("alu") / 1e12,
            "cop_budget_per_score": RF.cop_budget(D, RF.gb300_gamma("alu"),
                                                  pk["bf16_tflops"] * 1e12)}


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
    """The FP64 oracle running the same method (PartialReduce, top-2K, re-rank)
    on a bounded sample of the workload's queries."""

    def __init__(self, w, L, K, bins="mod"):
        import oracle
        self.o = oracle
        self.bins = bins
        self.X, self.Q, self.L, self.K, self.metric = w["X"], w["Q"], L, K, w["metric"]
        self.lowp = w["dtype"] == "bf16"
        self.Xs = oracle.bf16_round(self.X) if self.lowp else self.X.astype(np.float64)
        self.cursor = 0

    def run(self, n):
        o = self.o
        q = np.take(self.Q, np.arange(self.cursor, self.cursor + n) % self.Q.shape[0], axis=0)
        self.cursor = (self.cursor + n) % self.Q.shape[0]
        Qs = o.bf16_round(q) if self.lowp else q.astype(np.float64)
        t0 = time.perf_counter()
        V, A = o.partial_reduce(Qs, self.Xs, self.L, self.metric, bins=self.bins)
        _, cand = o.topk_pairs(V, A, 2 * self.K)
        o.rerank(q, self.X, cand, self.K, self.metric)
        return time.perf_counter() - t0

    def size_for(self, seconds, cap):
        t = self.run(8)
        return int(max(8, min(cap, seconds / max(t / 8, 1e-6))))


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
        if rank != 0:
            return 0
        import oracle
        oracle.build()
        from oracle import recall as R
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
        cores = os.cpu_count()
        line = {"impl": "reference", "metric": "queries/s at recall@10>=0.95", "value": value,
                "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(per),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": config_of(w, L, bins=args.bins),
                "cpu_baseline": {"value": value, "unit": "queries/s", "cores": cores,
                                 "kind": "oracle",
                                 "sample": "%d queries per step of the %d-query batch, full %d-row database"
                                           % (per[0][0], w["Q"].shape[0], w["X"].shape[0])},
                "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return 0

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    from paper_2206_14286_gb300 import search as S
    from paper_2206_14286_gb300 import _lib
    lib = _lib.get()

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

    clocks = Clocks(local)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for a, b in evs:
        a.record()
        step()
        b.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = evs[0][0].elapsed_time(evs[-1][1])
    value, total_ms = job_rate(world, M * args.steps, total_ms, device="cuda")

    # per-kernel times from the library's event profiler, in a separate pass
    # (its events are not part of the timed steps above)
    _lib.check(lib.knn_profile_enable(1))
    for _ in range(min(args.steps, 20)):
        step()
    torch.cuda.synchronize()
    _lib.check(lib.knn_profile_enable(0))
    prof = {}
    import ctypes
    for c, name in enumerate(["prep", "k1_partial_reduce", "k2_rescoring", "k3_rerank"]):
        tot = ctypes.c_double()
        n = ctypes.c_int64()
        _lib.check(lib.knn_profile_read(c, ctypes.byref(tot), ctypes.byref(n)))
        prof[name] = {"ms_avg": tot.value / max(1, n.value), "launches": n.value}
    # prep, K1 (plus the ragged-row kernel when N mod L != 0), then K2 and K3,
    # or one launch of both when the library fuses them (no K3 launches)
    fused23 = prof["k3_rerank"]["launches"] == 0
    if fused23:
        prof["k2_k3_rescoring_rerank_fused"] = prof.pop("k2_rescoring")
        prof.pop("k3_rerank")
    launches_per_step = (3 if fused23 else 4) + (1 if bins == "mod" and N % L else 0)
    S.sync_status()

    # the same step replayed from a CUDA graph (knn_search allocates nothing,
    # so a caller can capture it once and replay it)
    graph = None
    try:
        gr = torch.cuda.CUDAGraph()
        with torch.cuda.graph(gr):
            step()
        for _ in range(3):
            gr.replay()
        torch.cuda.synchronize()
        ga, gb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ga.record()
        for _ in range(args.steps):
            gr.replay()
        gb.record()
        torch.cuda.synchronize()
        g_ms = ga.elapsed_time(gb) / args.steps
        graph = {"value": world * M / (g_ms / 1e3), "unit": "queries/s", "ms_per_step": g_ms}
        del gr
    except RuntimeError as e:  # capture refused: report why
        graph = {"unavailable": str(e)[:200]}
    S.sync_status()

    # recall@10 against the exact FP32 search on the same data
    dbx = S.Database(Xd, metric=metric, dtype="f32", keep_f32=True)
    _, ei = dbx.search_exact(Qd, K)
    gi = idx.cpu().numpy()
    ei = ei.cpu().numpy()
    recall = float(np.mean([len(set(gi[i]) & set(ei[i])) / K for i in range(M)]))

    # the same BF16 search with the other bin map (j mod L), same workload
    other = "mod" if bins == "contiguous" else "contiguous"
    for _ in range(2):
        db.search(Qd, K, L=L, rerank=rerank, bins=other)
    torch.cuda.synchronize()
    ao, bo = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ao.record()
    for _ in range(args.steps):
        db.search(Qd, K, L=L, rerank=rerank, bins=other, out=(val, idx))
    bo.record()
    torch.cuda.synchronize()
    ms_other = ao.elapsed_time(bo) / args.steps
    io = idx.cpu().numpy()
    recall_other = float(np.mean([len(set(io[i]) & set(ei[i])) / K for i in range(M)]))

    # the plain FP32 path on the same workload (j mod L bins)
    def step32():
        dbx.search(Qd, K, L=L, rerank=rerank)
    for _ in range(2):
        step32()
    torch.cuda.synchronize()
    a32, b32 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a32.record()
    for _ in range(args.fp32_steps):
        step32()
    b32.record()
    torch.cuda.synchronize()
    ms32 = a32.elapsed_time(b32) / args.fp32_steps
    v32, i32 = dbx.search(Qd, K, L=L, rerank=rerank)
    i32 = i32.cpu().numpy()
    recall32 = float(np.mean([len(set(i32[i]) & set(ei[i])) / K for i in range(M)]))
    del dbx

    # end to end through the host-buffer entry point (pinned buffers)
    qh = torch.from_numpy(Q).pin_memory()
    vh = torch.empty((M, K), dtype=torch.float32, pin_memory=True)
    ih = torch.empty((M, K), dtype=torch.int32, pin_memory=True)
    for _ in range(3):
        db.search_host(qh, K, L=L, rerank=rerank, out=(vh, ih), bins=bins)
    e2e_steps = max(5, args.steps)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        db.search_host(qh, K, L=L, rerank=rerank, out=(vh, ih), bins=bins)
    e2e_s = time.perf_counter() - t0
    e2e = {"value": world * M * e2e_steps / e2e_s, "unit": "queries/s",
           "h2d_bytes_per_step": int(M * D * 4), "d2h_bytes_per_step": int(M * K * 8)}

    # roofline of the dominant kernel (K1)
    pk, pk_kind = peaks()
    k1_ms = prof["k1_partial_reduce"]["ms_avg"]
    flops = 2.0 * M * N * D
    achieved = flops / (k1_ms / 1e3) / 1e12
    peak = pk["bf16_tflops"]
    k1_bytes = N * D * 2 + (N * 4 if metric == "l2" else 0) + M * D * 2
    traffic = k1_traffic(M, N, D, bins)
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": "%s bf16 dense burst (MEASURED_PEAKS.json)" % pk_kind,
            "kernel": ("k1_tcs_kernel: fused BF16 contraction + PartialReduce, contiguous bins"
                       if bins == "contiguous" else
                       "k1_tcs_kernel (+ k1_tcs_tail for the N mod L ragged rows): fused BF16 "
                       "contraction + PartialReduce, j mod L bins"),
            "algorithmic": "2*M*N*D = %.4g FLOP per launch" % flops,
            "eq6": eq6_block(M, N, D, k1_ms, pk, traffic or k1_bytes),
            "hbm_context": {"algorithmic_bytes": k1_bytes,
                            "achieved_gbs": k1_bytes / (k1_ms / 1e3) / 1e9,
                            "peak_gbs": pk["hbm_gbs"]}}

    serving = None if args.no_serving else serving_leg(args, db, w)
    unfused = None if args.no_unfused else unfused_leg(Xd, Qd, K, L)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        runner = OracleRunner(w, L, K, bins)
        n = runner.size_for(12.0, M)
        tt = runner.run(n)
        rate = n / tt
        cpu = {"value": rate, "unit": "queries/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "%d of the %d queries against the full %d-row database (FP64), %.1f s"
                         % (n, M, N, tt)}

    if rank == 0:
        sm = sorted(step_ms)
        line = {"metric": "queries/s at recall@10>=0.95 (fused BF16; plain FP32 alongside)",
                "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16", "data": "synthetic", "config": config_of(w, L, L_min, bins),
                "recall_at_10": recall,
                "other_bins": {"bins": other, "value": world * M / (ms_other / 1e3),
                               "unit": "queries/s", "ms_per_step": ms_other,
                               "recall_at_10": recall_other},
                "p50_ms": sm[len(sm) // 2], "p99_ms": sm[min(len(sm) - 1, int(0.99 * len(sm)))],
                "fp32_path": {"value": world * M / (ms32 / 1e3), "unit": "queries/s",
                              "ms_per_step": ms32, "recall_at_10": recall32},
                "kernels": prof, "roofline": roof, "e2e": e2e,
                "graph_replay": graph,
                "serving": serving,
                "unfused_baseline": unfused,
                "gpu_launches": launches_per_step * args.steps, "clocks": clk,
                "cpu_baseline": cpu}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


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

    def events(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    gemm_ms = events(lambda: torch.matmul(Qb, Xb.t(), out=scores))
    amk_ms = events(lambda: S.approx_max_k(scores, K, L=L))
    unfused_ms = events(lambda: S.approx_max_k(torch.matmul(Qb, Xb.t(), out=scores), K, L=L))
    fused_ms = events(lambda: db_ip.search(Qd, K, L=L, rerank=1))
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
            "L": L, "L_min_eq14": L_min, "bins": bins, "metric": w["metric"], "rerank": "FP32 top-%dK" % w.get("rerank", 2),
            "l2_flush": "inputs larger than L2 (database %d MB in BF16 streamed every step)"
                        % (X.shape[0] * X.shape[1] * 2 // 2 ** 20),
            "parallelism": "replicas"}


def k1_traffic(M, N, D, bins="mod"):
    """DRAM bytes per K1 launch from the committed ncu summary of the same
    kernel source and launch shape (else None). The summary holds lines
    "- kernel source sha256: <16 hex>", "- bins: ...", "- M: ...", "- N: ...",
    "- D: ..." and "- dram bytes per launch: <int>"."""
    name = "k1_tcs_mix_l2_1m.md"
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    fields = {}
    for line in open(p):
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    h = hashlib.sha256(open(os.path.join(ROOT, "paper_2206_14286_gb300", "csrc", "k1_tcs.cu"),
                            "rb").read()).hexdigest()[:16]
    try:
        if (fields.get("kernel source sha256") != h or fields.get("bins") != bins
                or int(fields.get("M", -1)) != M or int(fields.get("N", -1)) != N
                or int(fields.get("D", -1)) != D):
            return None
        return int(fields["dram bytes per launch"])
    except (KeyError, ValueError):
        return None


if __name__ == "__main__":
    sys.exit(main())
