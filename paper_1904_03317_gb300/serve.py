"""Request loop with continuous batching for independent solves.

Requests arrive over time; each brings its own adaptive mesh and right-hand
side.  A request goes through two setup phases on a pool of host workers,
then a device solve:

1. mesh: as soon as it has arrived and a worker and a stream are free, its
   forest is refined and closed on the host, and the leaf set is hashed;
2. hierarchy: an idle hierarchy of an identical mesh (same leaves, degree,
   coefficients and solver parameters) is taken from the cache, or a new
   one is built once its device memory fits in the budget.  The memory a
   hierarchy needs is predicted from its leaf count with the largest
   bytes-per-leaf ratio seen so far, and the reservation is corrected to the
   hierarchy's measured device bytes as soon as it exists;
3. solve: the right-hand side is formed on the request's stream and the
   solve enqueued at once with ``gmg_solve_async`` (one CUDA graph per
   solve), so requests that arrive while others are on the GPU overlap with
   them there.  Finished solves are polled without blocking.

A finished hierarchy stays in a least-recently-used cache while memory and
streams allow; it is released when an admission needs either.  Latency is
measured from arrival to the result being ready on the device.
"""
from __future__ import annotations

import collections
import hashlib
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from . import gmg as G
from . import inputs

# device bytes per leaf cell assumed until the first hierarchy has been
# measured (a Q2 3D hierarchy with FP32 V-cycle holds about 1,200 per leaf)
INITIAL_BYTES_PER_LEAF = 2000.0


@dataclass
class Result:
    rid: int
    n: int = 0
    leaves: int = 0
    arrival: float = 0.0
    admitted: float = 0.0
    meshed: float = 0.0
    hier_start: float = 0.0
    setup_done: float = 0.0
    ready: float = 0.0
    iterations: int = 0
    converged: bool = False
    status: int = -1
    cache_hit: bool = False
    x: object = None
    device_bytes: int = 0

    @property
    def latency(self) -> float:
        return self.ready - self.arrival


@dataclass
class _Entry:
    """A hierarchy with its mesh, context, stream and reserved bytes."""
    key: bytes
    mesh: object
    ctx: object
    hier: object
    stream: object
    reserved: float


@dataclass
class _Live:
    res: Result
    entry: _Entry
    b: object
    x: object


class Server:
    def __init__(self, torch, device: int = 0, mem_budget: Optional[float] = None, setup_workers: int = 8,
                 max_live: int = 64, tol: float = 1e-8, vcycle_prec: int = G.PREC_FP32, keep_x: bool = False,
                 cache: bool = True, deterministic: bool = False):
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
        self.use_cache = cache
        self.deterministic = deterministic  # bitwise-repeatable solves (gmg_params.deterministic)
        self.bytes_per_leaf = INITIAL_BYTES_PER_LEAF
        self.cache_hits = 0
        self._measured = False
        self._streams = collections.deque(torch.cuda.Stream(device=device) for _ in range(max_live))

    # ----------------------------------------------------------- setup work
    def mesh_key(self, w: inputs.Workload, leaves) -> bytes:
        """Identity of a request's hierarchy: the leaf set of its mesh, its
        degree, coefficients and solver parameters."""
        lv, co = leaves
        h = hashlib.sha256()
        for a in (np.ascontiguousarray(lv), np.ascontiguousarray(co)):
            h.update(a.tobytes())
        coeff = b"" if w.coeff is None else np.ascontiguousarray(w.coeff, dtype=np.float64).tobytes()
        h.update(repr((w.coarse.dim, tuple(w.coarse.n0), tuple(w.coarse.lo), tuple(w.coarse.hi), w.degree,
                       w.cheb_degree, self.prec, self.deterministic)).encode())
        h.update(coeff)
        return h.digest()

    def _mesh(self, w: inputs.Workload, t0: float):
        """Phase 1 (host): the request's mesh, its leaf count and key."""
        m = G.build_mesh(w)
        leaves = m.leaves()
        return m, len(leaves[0]), self.mesh_key(w, leaves), time.perf_counter() - t0

    def _hierarchy(self, w: inputs.Workload, m, stream, t0: float):
        """Phase 2 (host, then device on the request's stream): the hierarchy."""
        ctx = G.Context(self.device, stream.cuda_stream)
        h = G.Hierarchy(ctx, m, w.degree, w.coeff, cheb_degree=w.cheb_degree, vcycle_prec=self.prec,
                        deterministic=self.deterministic)
        return ctx, h, time.perf_counter() - t0

    def _vectors(self, w: inputs.Workload, h, stream):
        """Right-hand side and solution of a request, on its stream."""
        torch = self.torch
        with torch.cuda.stream(stream):
            b = torch.empty(h.n, dtype=torch.float64, device=f"cuda:{self.device}")
            x = torch.empty_like(b)
        h.assemble_rhs(b, "random", w.seed)
        return b, x

    # ------------------------------------------------------------ the loop
    def run(self, arrivals: np.ndarray, workloads: List[inputs.Workload]) -> List[Result]:
        """Serve the requests (arrival times in seconds from the start)."""
        order = np.argsort(arrivals, kind="stable")
        pending = collections.deque(int(i) for i in order)
        results = [Result(rid=i, arrival=float(arrivals[i])) for i in range(len(workloads))]
        meshing = {}        # future -> (rid, stream)
        meshed = collections.deque()  # (rid, stream, mesh, leaves, key) waiting for a hierarchy
        building = {}       # future -> (rid, stream, mesh, key, reserved)
        live: List[_Live] = []
        cache: "collections.OrderedDict[bytes, _Entry]" = collections.OrderedDict()  # idle hierarchies
        reserved = 0.0
        done = 0
        t0 = time.perf_counter()

        def release(entry: _Entry):
            nonlocal reserved
            entry.hier.close()
            reserved -= entry.reserved
            self._streams.append(entry.stream)

        def busy() -> bool:
            return bool(live or building)

        with ThreadPoolExecutor(max_workers=self.workers) as pool:
            while done < len(workloads):
                now = time.perf_counter() - t0
                progressed = False
                # phase 1: arrived requests get a stream and a worker for their mesh
                while pending and arrivals[pending[0]] <= now and len(meshing) + len(building) < self.workers:
                    if not self._streams and cache:
                        release(cache.popitem(last=False)[1])  # an idle hierarchy gives up its stream
                    if not self._streams:
                        break
                    i = pending.popleft()
                    stream = self._streams.popleft()
                    results[i].admitted = now
                    meshing[pool.submit(self._mesh, workloads[i], t0)] = (i, stream)
                    progressed = True
                for fut in [f for f in meshing if f.done()]:
                    i, stream = meshing.pop(fut)
                    m, nleaves, key, t_done = fut.result()
                    results[i].meshed = t_done
                    results[i].leaves = nleaves
                    meshed.append((i, stream, m, nleaves, key))
                    progressed = True
                # phase 2: a cached hierarchy, or a new one once its memory fits
                while meshed:
                    i, stream, m, nleaves, key = meshed[0]
                    res = results[i]
                    if self.use_cache and key in cache:
                        entry = cache.pop(key)
                        self._streams.append(stream)  # the cached hierarchy brings its own stream
                        meshed.popleft()
                        res.cache_hit = True
                        self.cache_hits += 1
                        res.hier_start = res.setup_done = time.perf_counter() - t0
                        self._start_solve(res, entry, workloads[i], live)
                        progressed = True
                        continue
                    if len(building) >= self.workers:
                        break
                    est = self.bytes_per_leaf * nleaves
                    while reserved + est > self.budget and cache:
                        release(cache.popitem(last=False)[1])
                    if reserved + est > self.budget and busy():
                        break  # waits for memory (a request larger than the budget runs alone)
                    meshed.popleft()
                    reserved += est
                    res.hier_start = time.perf_counter() - t0
                    building[pool.submit(self._hierarchy, workloads[i], m, stream, t0)] = (i, stream, m, key, est)
                    progressed = True
                for fut in [f for f in building if f.done()]:
                    i, stream, m, key, est = building.pop(fut)
                    ctx, h, t_done = fut.result()
                    res = results[i]
                    res.setup_done = t_done
                    actual = float(h.info.device_bytes) + 16.0 * h.n  # hierarchy, b and x
                    reserved += actual - est  # the measured size replaces the prediction
                    self.bytes_per_leaf = self._learn(actual, res.leaves)
                    self._start_solve(res, _Entry(key, m, ctx, h, stream, actual), workloads[i], live)
                    progressed = True
                # finished solves: record, keep the hierarchy for an identical mesh
                still = []
                for lv in live:
                    ready, st, status = lv.entry.hier.solve_poll(False)
                    if not ready:
                        still.append(lv)
                        continue
                    res = lv.res
                    res.ready = time.perf_counter() - t0
                    res.iterations, res.converged, res.status = st.iterations, bool(st.converged), status
                    if self.keep_x:
                        res.x = lv.x
                    if self.use_cache and lv.entry.key not in cache:
                        cache[lv.entry.key] = lv.entry
                    else:
                        release(lv.entry)
                    done += 1
                    progressed = True
                live = still
                if not progressed:
                    time.sleep(0.0002)
            for entry in cache.values():
                entry.hier.close()
                self._streams.append(entry.stream)
        return results

    def _learn(self, actual_bytes: float, leaves: int) -> float:
        """Bytes per leaf for the next predictions: the largest ratio measured
        so far, with 5% margin (the initial guess only until the first
        measurement)."""
        ratio = 1.05 * actual_bytes / max(leaves, 1)
        if not self._measured:
            self._measured = True
            return ratio
        return max(self.bytes_per_leaf, ratio)

    def _start_solve(self, res: Result, entry: _Entry, w: inputs.Workload, live: List[_Live]):
        b, x = self._vectors(w, entry.hier, entry.stream)
        res.n = entry.hier.n
        res.device_bytes = int(entry.hier.info.device_bytes)
        entry.hier.solve_async(b, x, tol=self.tol)
        live.append(_Live(res, entry, b, x))


def percentile(values, q):
    return float(np.percentile(np.asarray(values, dtype=np.float64), q))
