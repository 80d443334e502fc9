"""Batched solves of independent problems with measured launch parameters.

`gmg_solve_batch` launches every problem's solve graph on a pool of streams.
Two launch parameters are chosen by measurement and recorded:

* per problem class (dimension, degree, half-decade of the leaf count): the
  smoother's tile shape, `gmg_params.brick_min_members` (a 2x2x2 block of
  sibling groups becomes a partial brick when at least this many of its
  groups are smoothed; 8 = full bricks only).  It is timed on the class's
  median problem with a few graph-mode solves per candidate.  Bricks exist
  in 3D only, so 2D classes keep the library default;
* for the whole batch: the number of streams.

Tuning runs on the caller's device and costs a few hierarchy builds per
class; its record says what was tried and what was chosen.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field
from typing import Dict, List, Sequence, Tuple

from . import gmg as G

TILE_CANDIDATES = (2, 4, 8)
STREAM_CANDIDATES = (8, 16, 32, 64)

Class = Tuple[int, int, int]


def problem_class(dim: int, degree: int, leaves: int) -> Class:
    """(dimension, degree, half-decade of the leaf count)."""
    return (int(dim), int(degree), int(math.floor(2.0 * math.log10(max(leaves, 1)))))


def class_name(c: Class) -> str:
    return f"{c[0]}d_q{c[1]}_leaves_1e{c[2] / 2:g}"


@dataclass
class Tuning:
    tile: Dict[Class, int] = field(default_factory=dict)                  # chosen brick_min_members
    tile_ms: Dict[Class, Dict[int, float]] = field(default_factory=dict)  # per candidate, ms per solve
    sample: Dict[Class, int] = field(default_factory=dict)                # index of the timed problem
    streams: int = 16
    streams_ms: Dict[int, float] = field(default_factory=dict)

    def record(self) -> dict:
        return {"tile_brick_min_members": {class_name(c): v for c, v in sorted(self.tile.items())},
                "tile_ms_per_solve": {class_name(c): {str(k): round(t, 3) for k, t in v.items()}
                                      for c, v in sorted(self.tile_ms.items())},
                "streams": self.streams,
                "streams_ms_per_batch": {str(k): round(t, 2) for k, t in self.streams_ms.items()}}


def _time_solves(torch, h, b, x, tol: float, reps: int) -> float:
    h.solve(b, x, tol=tol)  # builds the solve graph
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        h.solve(b, x, tol=tol)
    torch.cuda.synchronize()
    return 1e3 * (time.perf_counter() - t0) / reps


def tune_tiles(torch, ctx, workloads: Sequence, meshes: Sequence, tol: float = 1e-8, reps: int = 3,
               candidates: Sequence[int] = TILE_CANDIDATES, **params) -> Tuning:
    """Per 3D class, time the median problem with each tile candidate."""
    tun = Tuning()
    classes: Dict[Class, List[Tuple[int, int]]] = {}
    for i, (w, m) in enumerate(zip(workloads, meshes)):
        n = m.num_leaves()
        classes.setdefault(problem_class(w.coarse.dim, w.degree, n), []).append((n, i))
    for c, members in sorted(classes.items()):
        if c[0] != 3:
            continue
        members.sort()
        i = members[len(members) // 2][1]
        w = workloads[i]
        times = {}
        for cand in candidates:
            h = G.Hierarchy(ctx, meshes[i], w.degree, w.coeff, cheb_degree=w.cheb_degree,
                            brick_min_members=cand, **params)
            b = torch.empty(h.n, dtype=torch.float64, device="cuda")
            h.assemble_rhs(b, "random", w.seed)
            x = torch.zeros_like(b)
            times[cand] = _time_solves(torch, h, b, x, tol, reps)
            h.close()
        tun.tile[c] = min(times, key=times.get)
        tun.tile_ms[c] = times
        tun.sample[c] = i
    return tun


def tile_for(tun: Tuning, dim: int, degree: int, leaves: int) -> int:
    """The tuned brick_min_members of a problem (0: library default)."""
    return tun.tile.get(problem_class(dim, degree, leaves), 0)


def tune_streams(torch, tun: Tuning, hiers, bs, xs, tol: float = 1e-8,
                 candidates: Sequence[int] = STREAM_CANDIDATES) -> int:
    """Time one batched solve per stream count; keep the fastest."""
    for nst in candidates:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, status = G.solve_batch(hiers, bs, xs, tol=tol, n_streams=nst)
        torch.cuda.synchronize()
        tun.streams_ms[nst] = 1e3 * (time.perf_counter() - t0)
        if any(rc != G.OK for rc in status):
            raise RuntimeError(f"batched solve failed while tuning: {status}")
    tun.streams = min(tun.streams_ms, key=tun.streams_ms.get)
    return tun.streams


def class_counts(workloads: Sequence, meshes: Sequence) -> Dict[Class, int]:
    out: Dict[Class, int] = {}
    for w, m in zip(workloads, meshes):
        c = problem_class(w.coarse.dim, w.degree, m.num_leaves())
        out[c] = out.get(c, 0) + 1
    return out
