"""Request loop with continuous batching for independent solves.

Requests arrive over time; each brings its own adaptive mesh and right-hand
side.  The loop admits a request as soon as it has arrived, a setup slot is
free and its estimated device memory fits in the budget; setup workers build
the mesh and hierarchy (host, then device) on the request's own stream, and
the solve is enqueued at once with ``gmg_solve_async`` (one CUDA graph per
solve), so requests that arrive while others are on the GPU overlap with
them there.  Finished solves are polled without blocking; their hierarchy is
released, which frees memory for the next admissions.  Latency is measured
from arrival to the result being ready on the device.
"""
from __future__ import annotations

import collections
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from . import gmg as G
from . import inputs

# device bytes per unknown of a Q2 3D hierarchy with FP32 V-cycle (level
# vectors, tables, leaf tables, CG vectors), with margin; measured ~170
BYTES_PER_UNKNOWN = 230.0


@dataclass
class Result:
    rid: int
    n: int = 0
    arrival: float = 0.0
    admitted: float = 0.0
    setup_done: float = 0.0
    ready: float = 0.0
    iterations: int = 0
    converged: bool = False
    status: int = -1
    x: object = None
    device_bytes: int = 0

    @property
    def latency(self) -> float:
        return self.ready - self.arrival


@dataclass
class _Live:
    res: Result
    hier: object
    mesh: object
    ctx: object
    b: object
    x: object
    stream: object
    reserved: float


class Server:
    def __init__(self, torch, device: int = 0, mem_budget: Optional[float] = None, setup_workers: int = 8,
                 max_live: int = 64, tol: float = 1e-8, vcycle_prec: int = G.PREC_FP32, keep_x: bool = False):
        self.torch = torch
        self.device = device
        if mem_budget is None:
            free, _ = torch.cuda.mem_get_info(device)
            mem_budget = 0.6 * free
        self.budget = float(mem_budget)
        self.workers = setup_workers
        self.max_live = max_live
        self.tol = tol
        self.prec = vcycle_prec
        self.keep_x = keep_x
        self._streams = collections.deque(torch.cuda.Stream(device=device) for _ in range(max_live))

    def _setup(self, req_id, w, stream, t0):
        torch = self.torch
        m = G.build_mesh(w)
        ctx = G.Context(self.device, stream.cuda_stream)
        h = G.Hierarchy(ctx, m, w.degree, w.coeff, cheb_degree=w.cheb_degree, vcycle_prec=self.prec)
        host_b = inputs.random_rhs(w.seed, h.n)
        with torch.cuda.stream(stream):
            b = torch.from_numpy(host_b).to(device=f"cuda:{self.device}")
            x = torch.empty_like(b)
        return m, ctx, h, b, x, time.perf_counter() - t0

    def run(self, arrivals: np.ndarray, workloads: List[inputs.Workload]) -> List[Result]:
        """Serve the requests (arrival times in seconds from the start)."""
        torch = self.torch
        order = np.argsort(arrivals, kind="stable")
        pending = collections.deque(int(i) for i in order)
        results = [Result(rid=i, arrival=float(arrivals[i])) for i in range(len(workloads))]
        setups = {}
        live: List[_Live] = []
        reserved = 0.0
        done = 0
        t0 = time.perf_counter()
        with ThreadPoolExecutor(max_workers=self.workers) as pool:
            while done < len(workloads):
                now = time.perf_counter() - t0
                progressed = False
                # admission: arrived, a setup slot and a stream free, memory fits
                while pending and arrivals[pending[0]] <= now and len(setups) < self.workers and self._streams:
                    i = pending[0]
                    est = BYTES_PER_UNKNOWN * 8 * self._leaves_estimate(workloads[i])
                    if reserved + est > self.budget and (live or setups):
                        break
                    pending.popleft()
                    stream = self._streams.popleft()
                    results[i].admitted = now
                    reserved += est
                    setups[pool.submit(self._setup, i, workloads[i], stream, t0)] = (i, stream, est)
                    progressed = True
                # finished setups: enqueue their solves
                for fut in [f for f in setups if f.done()]:
                    i, stream, est = setups.pop(fut)
                    m, ctx, h, b, x, t_done = fut.result()
                    res = results[i]
                    res.setup_done = t_done
                    res.n = h.n
                    res.device_bytes = int(h.info.device_bytes)
                    h.solve_async(b, x, tol=self.tol)
                    live.append(_Live(res, h, m, ctx, b, x, stream, est))
                    progressed = True
                # finished solves: record and release
                still = []
                for lv in live:
                    ready, st, status = lv.hier.solve_poll(False)
                    if not ready:
                        still.append(lv)
                        continue
                    res = lv.res
                    res.ready = time.perf_counter() - t0
                    res.iterations, res.converged, res.status = st.iterations, bool(st.converged), status
                    if self.keep_x:
                        res.x = lv.x
                    lv.hier.close()
                    reserved -= lv.reserved
                    self._streams.append(lv.stream)
                    done += 1
                    progressed = True
                live = still
                if not progressed:
                    time.sleep(0.0002)
        return results

    @staticmethod
    def _leaves_estimate(w: inputs.Workload) -> float:
        """Leaves of a request's mesh before it is built, for admission: the
        requests refine uniformly g times and then twice at a surface, which
        adds a thin layer (a factor 1.6 covers it at every size)."""
        n0 = float(np.prod([w.coarse.n0[d] for d in range(w.coarse.dim)]))
        return n0 * float(2 ** w.coarse.dim) ** max(len(w.rounds) - 2, 0) * 1.6


def percentile(values, q):
    return float(np.percentile(np.asarray(values, dtype=np.float64), q))
