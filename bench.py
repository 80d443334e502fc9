#!/usr/bin/env python
"""Benchmark: solved DoFs/s of the adaptive local-smoothing GMG-CG solver.

One step = one full solve gmg_solve(b -> x) to relative residual 1e-8 of
-lap u = f on the 3D Q2 sphere-refined mesh of [0,1]^3 (4^3 coarse cells,
5 global refinements, 2 refinements of the cells meeting the sphere
|x - c| = 0.25; about 23M unknowns), FP32 V-cycle inside FP64 CG, with the
right-hand side already resident on the device.  The same solve with an
FP64 V-cycle is timed beside it, and the end-to-end variant copies b from
pinned host memory and x back every step.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gmg|reference]
Under torchrun each rank solves its own replica (no data-path collective).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "solved DoFs/s to rel. residual 1e-8 (FP32-vcycle vs FP64); GB/s vs HBM; p99 latency"
TOL = 1e-8
GLOBAL_REF, ADAPTIVE_REF = 5, 2
SAMPLE_GLOBAL, SAMPLE_ADAPTIVE = 2, 2  # bounded CPU sample of the same generator


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "src": "measured"}
    return {"hbm_gbs": 6800.0, "src": "fallback"}


# FP64 arithmetic peak of the part: 1.25 TFLOP/s nominal (dense FP64, incl. FMA = 2 flops)
FP64_PEAK_TFLOPS = 1.25



class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def over_ranks(dist, torch, value: float, op: str, device: str = "cuda") -> float:
    """Whole-job reduction of a per-rank number for replica runs: "max" for
    the timed seconds (the slowest rank sets the job time), "sum" for the
    unknowns solved; the value itself on a single process."""
    if dist is None:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def _oracle_worker(conn, g, a):
    """One oracle process: build the sample hierarchy once, then solve it on
    every request and report the solve time."""
    from oracle import gmg as ogmg
    from paper_1904_03317_gb300 import inputs
    w = inputs.poisson3d_sphere(g, a)
    H = ogmg.setup(w)
    b = H.disc.rhs_sine()
    conn.send(H.disc.n)
    while conn.recv() == "solve":
        t0 = time.perf_counter()
        res = ogmg.solve(H, b, TOL)
        conn.send((time.perf_counter() - t0, res.iterations))


class OraclePool:
    """The oracle (FP64, scipy sparse; one thread per process) on every host
    core of this process's affinity mask: one spawned process per core, each
    holding its own copy of the bounded sample of the headline generator.  A
    step is one solve in every process at once; its wall time is the
    slowest.  Spawned, not forked: the parent may already hold a CUDA
    context."""

    def __init__(self, g=SAMPLE_GLOBAL, a=SAMPLE_ADAPTIVE, cores=None):
        import multiprocessing as mp
        self.cores = cores or len(os.sched_getaffinity(0))
        self.g, self.a = g, a
        ctx = mp.get_context("spawn")
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"  # each process computes on one core
        try:
            self.conns, self.procs = [], []
            for _ in range(self.cores):
                mine, theirs = ctx.Pipe()
                pr = ctx.Process(target=_oracle_worker, args=(theirs, g, a), daemon=True)
                pr.start()
                self.conns.append(mine)
                self.procs.append(pr)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.n = [c.recv() for c in self.conns][0]

    def step(self):
        t0 = time.perf_counter()
        for c in self.conns:
            c.send("solve")
        its = [c.recv()[1] for c in self.conns]
        return time.perf_counter() - t0, its[0]

    def close(self):
        for c in self.conns:
            c.send("stop")
        for pr in self.procs:
            pr.join(timeout=30)

    def describe(self, steps, its):
        return (f"oracle FP64 local-smoothing GMG-CG (scipy sparse), {self.cores} processes x one core, each solving "
                f"the same sphere generator with {self.g} global + {self.a} adaptive refinements ({self.n} unknowns, "
                f"{its} its to 1e-8; the headline workload has {GLOBAL_REF} + {ADAPTIVE_REF} rounds, 21.9M unknowns, "
                f"which the assembled-matrix oracle cannot hold), {steps} rounds of {self.cores} concurrent solves")


def cpu_baseline(min_seconds=10.0):
    """The oracle on all host cores (OraclePool) for at least min_seconds of
    solves; returns (DoFs/s, sample description, cores)."""
    pool = OraclePool()
    try:
        pool.step()  # first solve of every process untimed
        t = 0.0
        steps = 0
        while t < min_seconds:
            dt, its = pool.step()
            t += dt
            steps += 1
    finally:
        pool.close()
    return pool.n * pool.cores * steps / t, pool.describe(steps, its), pool.cores


def run_reference(args, rank, world):
    """Reference arm: the oracle on the host cores (rank 0 only); a step is
    one solve of the bounded sample in every process of the pool."""
    if rank != 0:
        return
    pool = OraclePool()
    try:
        for _ in range(args.warmup):
            pool.step()
        t = 0.0
        for _ in range(args.steps):
            dt, its = pool.step()
            t += dt
    finally:
        pool.close()
    v = pool.n * pool.cores * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "DoFs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"poisson3d_q2_sphere_g{SAMPLE_GLOBAL}_a{SAMPLE_ADAPTIVE} x {pool.cores} "
                                   f"(bounded CPU sample of the g{GLOBAL_REF}_a{ADAPTIVE_REF} workload, one per core)",
                       "unknowns": pool.n, "tol": TOL, "cheb_degree": 4},
            "cpu_baseline": {"value": v, "unit": "DoFs/s", "cores": pool.cores, "kind": "oracle",
                             "sample": pool.describe(args.steps, its)},
            "e2e": {"value": v, "unit": "DoFs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_solves(torch, H, b, x, steps, stream, tol=TOL):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    st = None
    for _ in range(steps):
        st = H.solve(b, x, tol=tol)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, st


def serve_measure(torch, G, inputs, local, requests, warm_requests, rate):
    """Request loop: Poisson arrivals of 3D Q2 sphere-surface problems of
    log-uniform size, served with continuous batching (serve.Server); latency
    is arrival to result, throughput counts the measured requests only.  The
    same requests one at a time with the plain FP64 V-cycle (a sample) are
    timed beside it.  Returns (record, clocks)."""
    from paper_1904_03317_gb300 import serve
    total = warm_requests + requests
    arrivals, ws = inputs.serving_requests(total, rate=rate)
    sampler = ClockSampler(local)
    sampler.start()
    srv = serve.Server(torch, device=local)
    res = srv.run(arrivals, ws)
    clocks = sampler.stop()
    meas = res[warm_requests:]
    assert all(r.status == G.OK for r in meas), [r.status for r in meas]
    lat = [r.latency for r in meas]
    span = max(r.ready for r in meas) - min(r.arrival for r in meas)
    dofs = float(sum(r.n for r in meas))
    setup = [r.setup_done - r.admitted for r in meas]
    solve = [r.ready - r.setup_done for r in meas]
    queue = [r.admitted - r.arrival for r in meas]
    # the same requests one at a time with the plain FP64 V-cycle (a sample)
    k = min(16, len(meas))
    ctx = G.Context(local, torch.cuda.current_stream().cuda_stream)
    t_setup64 = t_solve64 = 0.0
    n64 = 0
    for r in meas[:k]:
        w = ws[r.rid]
        a = time.perf_counter()
        h = G.Hierarchy(ctx, G.build_mesh(w), w.degree, w.coeff, cheb_degree=w.cheb_degree,
                        vcycle_prec=G.PREC_FP64)
        b = torch.empty(h.n, dtype=torch.float64, device="cuda")
        h.assemble_rhs(b, "random", w.seed)
        x = torch.zeros_like(b)
        torch.cuda.synchronize()
        m = time.perf_counter()
        h.solve(b, x, tol=TOL)
        torch.cuda.synchronize()
        e = time.perf_counter()
        t_setup64 += m - a
        t_solve64 += e - m
        n64 += h.n
        h.close()
    ns = [r.n for r in meas]
    rec = {"value": dofs / span, "unit": "DoFs/s (served, setup included)", "requests": len(meas),
           "warm_requests": warm_requests, "rate_per_s": rate, "span_s": span,
           "unknowns_min": int(min(ns)), "unknowns_median": int(np.median(ns)), "unknowns_max": int(max(ns)),
           "setup_workers": srv.workers, "memory_budget_gb": round(srv.budget / 1e9, 1),
           "hierarchy_cache_hits": srv.cache_hits,
           "latency_s": {"p50": serve.percentile(lat, 50), "p99": serve.percentile(lat, 99),
                         "queue_p50": serve.percentile(queue, 50), "setup_p50": serve.percentile(setup, 50),
                         "solve_p50": serve.percentile(solve, 50), "solve_p99": serve.percentile(solve, 99)},
           "serial_fp64": {"sample": k, "solve_dofs_per_s": n64 / t_solve64,
                           "setup_and_solve_dofs_per_s": n64 / (t_setup64 + t_solve64)}}
    return rec, clocks


def run_serve(args, torch, G, inputs, local, rank, world):
    rec, clocks = serve_measure(torch, G, inputs, local, args.requests, args.warm_requests, args.rate)
    if rank == 0:
        line = {
            "metric": METRIC, "value": rec["value"], "unit": "DoFs/s", "n_gpus": world, "steps": rec["requests"],
            "warmup": rec["warm_requests"], "ms_per_step": 1e3 * rec["span_s"] / rec["requests"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 V-cycle / f64 CG",
            "data": "synthetic",
            "config": {"workload": "serving_3d_q2_sphere_surface_requests", "tol": TOL,
                       **{k: rec[k] for k in ("requests", "warm_requests", "rate_per_s", "unknowns_min",
                                              "unknowns_median", "unknowns_max", "setup_workers",
                                              "memory_budget_gb")}},
            "latency_s": rec["latency_s"], "serial_fp64": rec["serial_fp64"],
            "hierarchy_cache_hits": rec["hierarchy_cache_hits"], "clocks": clocks,
        }
        print(json.dumps(line), flush=True)


def batch_measure(torch, G, inputs, local, count, steps, warmup, serial_sample, barrier, max_over_ranks,
                  sum_over_ranks):
    """Independent problems solved together (gmg_solve_batch): each step solves
    every problem of the list once; the stream count is tuned in the warm-up.
    The same problems one at a time (FP32 V-cycle, graph mode) and a sample
    with the plain FP64 V-cycle are timed beside it.  Returns (record,
    clocks)."""
    from concurrent.futures import ThreadPoolExecutor
    from paper_1904_03317_gb300 import batch
    ws = inputs.batched_problems(count)
    stream = torch.cuda.current_stream()
    ctx = G.Context(local, stream.cuda_stream)
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=8) as ex:  # host setup in parallel (the ABI releases the GIL)
        meshes = list(ex.map(G.build_mesh, ws))
    t_mesh = time.perf_counter() - t0
    # tile shape per problem class, timed on each class's median problem
    t0 = time.perf_counter()
    tun = batch.tune_tiles(torch, ctx, ws, meshes, tol=TOL, vcycle_prec=G.PREC_FP32)
    t_tune = time.perf_counter() - t0
    t0 = time.perf_counter()
    hs = [G.Hierarchy(ctx, m, w.degree, w.coeff, cheb_degree=w.cheb_degree, vcycle_prec=G.PREC_FP32,
                      brick_min_members=batch.tile_for(tun, w.coarse.dim, w.degree, m.num_leaves()))
          for m, w in zip(meshes, ws)]
    t_setup = time.perf_counter() - t0
    ns = [h.n for h in hs]
    bs = [torch.empty(n, dtype=torch.float64, device="cuda") for n in ns]
    for h, b, w in zip(hs, bs, ws):
        h.assemble_rhs(b, "random", w.seed)
    xs = [torch.zeros_like(b) for b in bs]
    # warm-up, and pick the stream count
    nst = batch.tune_streams(torch, tun, hs, bs, xs, tol=TOL)
    for _ in range(max(0, warmup - 1)):
        G.solve_batch(hs, bs, xs, tol=TOL, n_streams=nst)
    sampler = ClockSampler(local)
    sampler.start()
    for h in hs:
        h.profile_reset(timing=False)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        stats, status = G.solve_batch(hs, bs, xs, tol=TOL, n_streams=nst)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    secs = max_over_ranks(e0.elapsed_time(e1) / 1e3)
    launches = int(sum(sum(v["launches"] for v in h.profile_read().values()) for h in hs))
    total = sum_over_ranks(float(sum(ns)) * steps)
    value = total / secs
    its = [s.iterations for s in stats]
    # the same problems one at a time (graph mode, FP32 V-cycle), and a sample
    # with the plain FP64 V-cycle
    torch.cuda.synchronize()
    a = time.perf_counter()
    for h, b, x in zip(hs, bs, xs):
        h.solve(b, x, tol=TOL)
    torch.cuda.synchronize()
    serial32 = float(sum(ns)) / (time.perf_counter() - a)
    k = min(serial_sample, len(ws))
    h64 = [G.Hierarchy(ctx, meshes[i], ws[i].degree, ws[i].coeff, cheb_degree=ws[i].cheb_degree,
                       vcycle_prec=G.PREC_FP64) for i in range(k)]
    x64 = [torch.zeros_like(bs[i]) for i in range(k)]
    for i in range(k):
        h64[i].solve(bs[i], x64[i], tol=TOL)  # builds the graphs
    torch.cuda.synchronize()
    a = time.perf_counter()
    for i in range(k):
        h64[i].solve(bs[i], x64[i], tol=TOL)
    torch.cuda.synchronize()
    serial64 = float(sum(ns[:k])) / (time.perf_counter() - a)
    diff = max(float(torch.linalg.vector_norm(xs[i] - x64[i]) / torch.linalg.vector_norm(x64[i])) for i in range(k))
    for h in h64:
        h.close()
    dims = [w.coarse.dim for w in ws]
    rec = {"value": value, "unit": "DoFs/s", "steps": steps, "ms_per_step": 1e3 * secs / steps,
           "workload": f"batched_{len(ws)}_poisson_2d3d_q1q2_random_rounds",
           "problems": len(ws), "unknowns_total": int(sum(ns)), "unknowns_min": int(min(ns)),
           "unknowns_median": int(np.median(ns)), "unknowns_max": int(max(ns)),
           "problems_3d": int(sum(1 for d in dims if d == 3)),
           "cg_iterations_min_max": [int(min(its)), int(max(its))], "n_streams": nst,
           "setup_s": {"mesh": round(t_mesh, 2), "tuning": round(t_tune, 2), "hierarchies": round(t_setup, 2)},
           "tuning": dict(tun.record(), problems_per_class={
               batch.class_name(c): v for c, v in sorted(batch.class_counts(ws, meshes).items())}),
           "gpu_launches": launches,
           "serial_fp32_graph": {"value": serial32, "unit": "DoFs/s"},
           "serial_fp64": {"value": serial64, "unit": "DoFs/s", "sample": f"first {k} problems",
                           "max_rel_diff_vs_batched": diff}}
    for h in hs:
        h.close()
    return rec, clocks


def run_batch(args, torch, G, inputs, local, barrier, max_over_ranks, sum_over_ranks, rank, world):
    rec, clocks = batch_measure(torch, G, inputs, local, args.batch_count, args.steps, args.warmup,
                                args.serial_sample, barrier, max_over_ranks, sum_over_ranks)
    if rank == 0:
        line = {
            "metric": METRIC, "value": rec["value"], "unit": "DoFs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rec["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 V-cycle / f64 CG", "data": "synthetic",
            "config": {"tol": TOL, "parallelism": f"replicas x{world}",
                       **{k: rec[k] for k in ("workload", "problems", "unknowns_total", "unknowns_min",
                                              "unknowns_median", "unknowns_max", "problems_3d",
                                              "cg_iterations_min_max", "n_streams", "setup_s")}},
            "gpu_launches": rec["gpu_launches"], "serial_fp32_graph": rec["serial_fp32_graph"],
            "serial_fp64": rec["serial_fp64"], "clocks": clocks,
        }
        print(json.dumps(line), flush=True)


def run_levels(args, torch, G, inputs, local):
    """Level smoother alone: on each level of the headline workload, the
    Chebyshev smoothing of the V-cycle (m updates from a nonzero start,
    gmg_level_smooth) timed with CUDA events, with its algorithmic bytes
    (s B x (4 n_S + n_I) per update, s = 4 in FP32 and 8 in FP64; the call
    also copies the level vector once, 2 s B per slot)."""
    w = inputs.poisson3d_sphere(args.global_ref, args.adaptive_ref)
    stream = torch.cuda.current_stream()
    ctx = G.Context(local, stream.cuda_stream)
    fp64 = args.level_prec == "fp64"
    dt, sb = (torch.float64, 8.0) if fp64 else (torch.float32, 4.0)
    H = G.Hierarchy(ctx, G.build_mesh(w), w.degree, cheb_degree=w.cheb_degree,
                    vcycle_prec=G.PREC_FP64 if fp64 else G.PREC_FP32)
    info, m = H.info, w.cheb_degree
    wanted = [int(v) for v in args.levels.split(",")] if args.levels else list(range(1, info.n_levels))
    out = []
    for lvl in wanted:
        n = int(info.slots[lvl])
        g = torch.rand(n, dtype=dt, device="cuda")
        u, tmp = torch.zeros_like(g), torch.zeros_like(g)
        for _ in range(args.warmup):
            H.level_smooth(lvl, g, u, tmp, False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            H.level_smooth(lvl, g, u, tmp, False)
        e1.record(stream)
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) / 1e3 / args.steps
        nbytes = m * sb * (4 * int(info.n_S[lvl]) + int(info.n_I[lvl])) + 2 * sb * n
        out.append({"level": lvl, "slots": n, "n_S": int(info.n_S[lvl]), "n_I": int(info.n_I[lvl]),
                    "bricks": int(info.bricks[lvl]), "bricks_partial": int(info.bricks_partial[lvl]),
                    "us_per_smoothing": round(1e6 * secs, 2), "GB/s": round(nbytes / secs / 1e9, 1)})
    print(json.dumps({"metric": "level smoothing time (m Chebyshev updates)", "workload": w.name,
                      "precision": args.level_prec,
                      "cheb_degree": m, "steps": args.steps, "warmup": args.warmup, "levels": out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gmg", choices=["gmg", "reference"])
    ap.add_argument("--global-ref", type=int, default=GLOBAL_REF)
    ap.add_argument("--adaptive-ref", type=int, default=ADAPTIVE_REF)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--fichera-rounds", type=int, default=13,
                    help="fichera workload: adaptive rounds (13: 3.4M unknowns, the paper's cycle 13)")
    ap.add_argument("--levels", default="", help="levels workload: comma-separated levels (default all)")
    ap.add_argument("--level-prec", default="fp32", choices=["fp32", "fp64"],
                    help="levels workload: precision of the level vectors")
    ap.add_argument("--brick-min-members", type=int, default=0,
                    help="smoother tile shape (gmg_params.brick_min_members; 0 = library default)")
    ap.add_argument("--deterministic", action="store_true", help="bitwise-repeatable solves (gmg_params)")
    ap.add_argument("--workload", default="sphere",
                    choices=["sphere", "checker", "fichera", "batch", "serve", "levels"],
                    help="sphere: 3D Q2 Poisson refined at a sphere (the headline); checker: 3D Q2 with the "
                         "{1, 100} subcube checkerboard coefficient refined at the subcube planes; fichera: "
                         "the Laplace example of Sec. 4.3 with its MF solver settings; batch: "
                         "512 independent 2D/3D Q1/Q2 problems solved together")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--requests", type=int, default=200, help="serve workload: measured requests")
    ap.add_argument("--warm-requests", type=int, default=20, help="serve workload: requests before them")
    ap.add_argument("--rate", type=float, default=200.0, help="serve workload: arrivals per second")
    ap.add_argument("--serial-sample", type=int, default=64,
                    help="batch workload: problems timed one by one with plain FP64 V-cycles")
    ap.add_argument("--finest-level", type=int, default=9, help="checker workload: finest level")
    ap.add_argument("--no-batch", action="store_true",
                    help="sphere workload: skip the batched sub-record")
    ap.add_argument("--no-serve", action="store_true",
                    help="sphere workload: skip the serving sub-record")
    ap.add_argument("--sub-requests", type=int, default=60,
                    help="sphere workload: measured requests of the serving sub-record")
    ap.add_argument("--sub-warm-requests", type=int, default=10,
                    help="sphere workload: requests before them")
    ap.add_argument("--solve-mode", default="graph", choices=["graph", "stream"],
                    help="graph: each solve is one CUDA-graph launch; stream: one launch per kernel")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        return over_ranks(dist, torch, v, "max")

    def sum_over_ranks(v):
        return over_ranks(dist, torch, v, "sum")

    import __graft_entry__
    __graft_entry__.build()
    from paper_1904_03317_gb300 import gmg as G
    from paper_1904_03317_gb300 import inputs
    if args.workload == "serve":
        run_serve(args, torch, G, inputs, local, rank, world)
        if dist:
            dist.destroy_process_group()
        return
    if args.workload == "levels":
        run_levels(args, torch, G, inputs, local)
        return
    if args.workload == "batch":
        run_batch(args, torch, G, inputs, local, barrier, max_over_ranks, sum_over_ranks, rank, world)
        if dist:
            dist.destroy_process_group()
        return

    if args.workload == "sphere":
        w = inputs.poisson3d_sphere(args.global_ref, args.adaptive_ref)
    elif args.workload == "fichera":
        w = inputs.fichera(args.fichera_rounds)
    else:
        w = inputs.checkerboard3d(args.global_ref, args.finest_level)
    tol = w.tol
    solver = {"cheb_degree": w.cheb_degree, "brick_min_members": args.brick_min_members,
              "deterministic": args.deterministic,
              "smoother": G.SMOOTHER_JACOBI if w.smoother == "jacobi" else G.SMOOTHER_CHEBYSHEV,
              "coarse_solver": {"cholesky": G.COARSE_CHOLESKY, "chebyshev": G.COARSE_CHEBYSHEV,
                                "cg": G.COARSE_CG}[w.coarse_solver]}
    t0 = time.perf_counter()
    mesh = G.build_mesh(w)
    t_mesh = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    ctx = G.Context(local, stream.cuda_stream)
    t0 = time.perf_counter()
    H = G.Hierarchy(ctx, mesh, w.degree, w.coeff, vcycle_prec=G.PREC_FP32, solve_graph=args.solve_mode == "graph",
                    **solver)
    t_setup = time.perf_counter() - t0
    info = H.info
    n = H.n
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    H.assemble_rhs(b, w.rhs, w.seed)  # manufactured, or seeded U[-1, 1) per unknown
    x = torch.zeros_like(b)
    for _ in range(args.warmup):
        H.solve(b, x, tol=tol)

    # ---- timed region: K solves, each one CUDA-graph launch whose CG loop
    # runs on the device (--solve-mode graph; launches counted by the
    # library's accounting)
    sampler = ClockSampler(local)
    sampler.start()
    H.profile_reset(timing=False)
    barrier()
    secs, st = time_solves(torch, H, b, x, args.steps, stream, tol)
    barrier()
    launches = int(sum(v["launches"] for v in H.profile_read().values()))
    t_max = max_over_ranks(secs)
    total_dofs = sum_over_ranks(float(n) * args.steps)
    value = total_dofs / t_max
    iters = st.iterations

    # ---- per-kernel times: the same K solves in stream mode, every launch
    # bracketed by CUDA events on the solve stream (graph mode has no
    # per-launch events)
    H.profile_reset(timing=True)
    barrier()
    secs_stream, _ = time_solves(torch, H, b, x, args.steps, stream, tol)
    barrier()
    kern = H.profile_read()
    H.profile_reset(timing=False)
    clocks = sampler.stop()
    stream_ms = 1e3 * max_over_ranks(secs_stream) / args.steps

    # ---- end to end through host buffers: every step copies its b from
    # pinned host memory and its x back; serially, and pipelined (step i+1's
    # input and step i's result move on a copy stream while a solve runs)
    hb = b.cpu().pin_memory()
    hx = [torch.empty_like(hb).pin_memory() for _ in range(2)]
    db = [torch.empty_like(b) for _ in range(2)]
    dx = [torch.zeros_like(b) for _ in range(2)]
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        db[0].copy_(hb, non_blocking=True)
        H.solve(db[0], dx[0], tol=tol)
        hx[0].copy_(dx[0], non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_serial = total_dofs / max_over_ranks(e0.elapsed_time(e1) / 1e3)
    copy_s = torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    ev_done = torch.cuda.Event()
    barrier()
    e0.record(stream)
    copy_s.wait_stream(stream)
    with torch.cuda.stream(copy_s):
        db[0].copy_(hb, non_blocking=True)
        ev_in[0].record(copy_s)
    for i in range(args.steps):
        j = i % 2
        if i + 1 < args.steps:
            with torch.cuda.stream(copy_s):
                db[1 - j].copy_(hb, non_blocking=True)
                ev_in[1 - j].record(copy_s)
        stream.wait_event(ev_in[j])
        if i >= 2:
            stream.wait_event(ev_out[j])  # x of step i-2 has left the device
        H.solve(db[j], dx[j], tol=tol)
        ev_done.record(stream)
        copy_s.wait_event(ev_done)
        with torch.cuda.stream(copy_s):
            hx[j].copy_(dx[j], non_blocking=True)
            ev_out[j].record(copy_s)
    stream.wait_stream(copy_s)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_secs = max_over_ranks(e0.elapsed_time(e1) / 1e3)
    e2e_value = total_dofs / e2e_secs
    assert torch.equal(hx[(args.steps - 1) % 2], dx[(args.steps - 1) % 2].cpu())
    x32 = dx[(args.steps - 1) % 2].clone()

    # ---- the FP64 V-cycle path on the same problem
    fp64 = None
    if not args.no_fp64:
        H64 = G.Hierarchy(ctx, mesh, w.degree, w.coeff, vcycle_prec=G.PREC_FP64, **solver)
        x64 = torch.zeros_like(b)
        H64.solve(b, x64, tol=tol)
        s64, st64 = time_solves(torch, H64, b, x64, max(1, min(args.steps, 3)), stream, tol)
        s64 = max_over_ranks(s64)
        steps64 = max(1, min(args.steps, 3))
        diff = float(torch.linalg.vector_norm(x32 - x64) / torch.linalg.vector_norm(x64))
        fp64 = {"value": sum_over_ranks(float(n) * steps64) / s64, "unit": "DoFs/s",
                "ms_per_step": 1e3 * s64 / steps64, "iterations": st64.iterations,
                "rel_diff_fp32_vs_fp64_solution": diff}
        H64.close()

    # ---- the batched and served workloads, measured in the same run (one
    # process; replicas run the headline only)
    batch = serve_rec = None
    if world == 1 and not args.no_batch and args.workload == "sphere":
        H.close()
        rec, bclocks = batch_measure(torch, G, inputs, local, args.batch_count, 2, 2, args.serial_sample,
                                     barrier, max_over_ranks, sum_over_ranks)
        batch = dict(rec, clocks=bclocks)
    if world == 1 and not args.no_serve and args.workload == "sphere":
        rec, sclocks = serve_measure(torch, G, inputs, local, args.sub_requests, args.sub_warm_requests, args.rate)
        serve_rec = dict(rec, clocks=sclocks)

    # ---- roofline of the dominant kernel (largest share of the timed region)
    pk = peaks()
    dom = max(kern, key=lambda k: kern[k]["ms"])
    kd = kern[dom]
    if dom == "active_apply":
        achieved = kd["flops"] / (kd["ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s (FP64)", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_src": "nominal FP64 (152 SMs x 2 FP64 FMA/clk x 2070 MHz x 2)"}
    else:
        achieved = kd["bytes"] / (kd["ms"] / 1e3) / 1e9
        # DRAM traffic needs a profiler, which this timed run does not use:
        # the measured per-launch traffic of the same kernels is in profiles/
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / pk["hbm_gbs"], "traffic": None,
                "algorithmic_bytes_per_launch": kd["bytes"] / max(kd["launches"], 1), "peak_src": pk["src"]}
    t_all = sum(v["ms"] for v in kern.values())
    kernels = {}
    for k, v in kern.items():
        if v["launches"] == 0:
            continue
        kernels[k] = {"launches": v["launches"], "ms": round(v["ms"], 3),
                      "share": round(v["ms"] / t_all, 4) if t_all else None,
                      "GB/s": round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1) if v["ms"] else None,
                      "TFLOP/s": round(v["flops"] / (v["ms"] / 1e3) / 1e12, 3) if v["ms"] else None}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc, ncores = cpu_baseline()
        cpu = {"value": v, "unit": "DoFs/s", "cores": ncores, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "DoFs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 V-cycle / f64 CG",
            "data": "synthetic",
            "config": {"workload": w.name,
                       "unknowns": n, "leaves": int(info.n_leaves), "levels": int(info.n_levels),
                       "tol": tol, "cheb_degree": w.cheb_degree, "smoother": w.smoother,
                       "coarse_solver": w.coarse_solver, "cg_iterations": iters,
                       "brick_min_members": args.brick_min_members or 4, "deterministic": args.deterministic,
                       "parallelism": f"replicas x{world}", "solve_mode": args.solve_mode,
                       "l2": f"inputs larger than L2 (active vector {8 * n / 1e6:.0f} MB)",
                       "setup_s": {"mesh": round(t_mesh, 3), "hierarchy_host": round(info.setup_host_s, 3),
                                   "hierarchy_device": round(info.setup_device_s, 3),
                                   "total": round(t_setup, 3)}},
            "gpu_launches": launches,
            "e2e": {"value": e2e_value, "unit": "DoFs/s", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
                    "copies": "pipelined: step i+1's b in and step i's x out on a copy stream during solves",
                    "serial_value": e2e_serial},
            "roofline": roof,
            "kernels": kernels,
            "kernel_timing": {"mode": "stream (one launch per kernel, CUDA events per launch)",
                              "ms_per_step": stream_ms, "steps": args.steps},
            "fp64_vcycle": fp64,
            "batch": batch,
            "serve": serve_rec,
            "cpu_baseline": cpu,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
