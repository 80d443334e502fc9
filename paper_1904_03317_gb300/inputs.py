"""Seeded synthetic inputs: which leaves to refine, coefficients, random values.

This module is shared by the CUDA path's callers (tests, bench, smoke) and by
the CPU oracle.  It holds none of the multigrid method's arithmetic: no mesh
closure, no degrees of freedom, no element integrals.  It only answers
"which of these leaf cells does this refinement round flag?", "what is the
coefficient of this coarse cell?" and "which uniform random numbers does this
seed give?".  Every function takes plain integer cell descriptions
(level, lattice coordinates) and returns numpy arrays, so each side can call
it on the leaves of its own mesh.

Mesh shapes follow the refinement rules of Sec. 3.5 of the paper (uniform,
circle, quadrant, sine curve, annulus; each round followed by closure) and
the configurations of the solver experiments in Sec. 4.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x) -> np.ndarray:
    """SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014).

    Maps each 64-bit input to a well-mixed 64-bit output.  Used with
    ``x = seed + counter * golden_gamma`` as a counter-based generator.
    """
    z = np.asarray(x, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counters) -> np.ndarray:
    """Uniform doubles in [0, 1) from (seed, counter) pairs, 53 random bits each."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ (c * np.uint64(0xD1B54A32D192ED03))
    bits = splitmix64(x) >> np.uint64(11)
    return bits.astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_pm1(seed: int, counters) -> np.ndarray:
    """Uniform doubles in [-1, 1) from (seed, counter) pairs."""
    return 2.0 * uniform01(seed, counters) - 1.0


def cell_hash_key(level, coords) -> np.ndarray:
    """A 64-bit counter that names a cell (level, lattice coordinates) uniquely.

    ``coords`` has shape (n, 3); unused dimensions are 0.  Coordinates must be
    below 2**20, levels below 16.
    """
    level = np.asarray(level, dtype=np.uint64)
    c = np.asarray(coords, dtype=np.uint64)
    return ((level << np.uint64(60)) | (c[:, 2] << np.uint64(40))
            | (c[:, 1] << np.uint64(20)) | c[:, 0])


@dataclasses.dataclass(frozen=True)
class CoarseMesh:
    """A Cartesian brick [lo, hi] split into n0[0] x n0[1] (x n0[2]) coarse cells.

    ``present`` (optional) lists, per coarse cell in lexicographic order (x
    fastest), whether the cell belongs to the domain; the domain is the
    union of the present cells (for instance the Fichera corner, a brick with
    one octant removed).  None: every cell is present.
    """

    dim: int
    n0: Sequence[int]
    lo: Sequence[float]
    hi: Sequence[float]
    present: Optional[Tuple[bool, ...]] = None

    def cell_present(self, coords) -> np.ndarray:
        """Whether the coarse cells with the given coordinates (n, 3) are in the domain."""
        c = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
        if self.present is None:
            return np.ones(len(c), dtype=bool)
        n = [int(self.n0[d]) if d < self.dim else 1 for d in range(3)]
        mask = np.asarray(self.present, dtype=bool)
        return mask[c[:, 0] + n[0] * (c[:, 1] + n[1] * c[:, 2])]

    def cells_per_dim(self, level: int) -> np.ndarray:
        n = np.ones(3, dtype=np.int64)
        n[: self.dim] = np.asarray(self.n0[: self.dim], dtype=np.int64) << level
        return n

    def boxes(self, level, coords):
        """Lower and upper corners (n, dim) of the cells given by level and lattice coords."""
        level = np.asarray(level, dtype=np.int64)
        coords = np.asarray(coords, dtype=np.int64)
        lo = np.asarray(self.lo[: self.dim], dtype=np.float64)
        hi = np.asarray(self.hi[: self.dim], dtype=np.float64)
        n0 = np.asarray(self.n0[: self.dim], dtype=np.float64)
        h = (hi - lo)[None, :] / (n0[None, :] * np.ldexp(1.0, level)[:, None])
        blo = lo[None, :] + coords[:, : self.dim] * h
        return blo, blo + h


# A refinement round: (coarse, level, coords, finest_level) -> bool flags.
RoundFn = Callable[[CoarseMesh, np.ndarray, np.ndarray, int], np.ndarray]


def round_uniform() -> RoundFn:
    """Flag every leaf (one global refinement)."""

    def fn(cm, level, coords, finest):
        return np.ones(len(level), dtype=bool)

    return fn


def round_sphere_surface(center, radius, finest_only: bool = True) -> RoundFn:
    """Flag leaves whose closed box meets the sphere (circle in 2D) |x - center| = radius.

    A closed box meets the sphere iff its nearest point to the centre lies
    inside (or on) the sphere and its farthest point lies outside (or on) it.
    With ``finest_only`` only leaves on the current finest level are flagged.
    """
    center = np.asarray(center, dtype=np.float64)
    r2 = float(radius) ** 2

    def meets(cm, level, coords):
        blo, bhi = cm.boxes(level, coords)
        c = center[None, : cm.dim]
        near = np.clip(c, blo, bhi) - c
        far = np.maximum(np.abs(blo - c), np.abs(bhi - c))
        dmin = np.sum(near * near, axis=1)
        dmax = np.sum(far * far, axis=1)
        return (dmin <= r2) & (dmax >= r2)

    def fn(cm, level, coords, finest):
        if not finest_only:
            return meets(cm, level, coords)
        level = np.asarray(level)
        sel = np.nonzero(level == finest)[0]  # only these can be flagged
        hit = np.zeros(len(level), dtype=bool)
        hit[sel] = meets(cm, level[sel], np.asarray(coords)[sel])
        return hit

    return fn


def round_shell(center, r_in, r_out) -> RoundFn:
    """Flag leaves whose closed box meets the shell r_in <= |x - center| <= r_out."""
    center = np.asarray(center, dtype=np.float64)

    def fn(cm, level, coords, finest):
        blo, bhi = cm.boxes(level, coords)
        c = center[None, : cm.dim]
        near = np.clip(c, blo, bhi) - c
        far = np.maximum(np.abs(blo - c), np.abs(bhi - c))
        dmin = np.sum(near * near, axis=1)
        dmax = np.sum(far * far, axis=1)
        return (dmin <= r_out * r_out) & (dmax >= r_in * r_in)

    return fn


def round_random_interface(seed: int, round_index: int, prob: float,
                           planes_per_unit: int = 4) -> RoundFn:
    """Flag, with probability ``prob``, each finest-level leaf that has a face on an
    interior plane x_i = m / planes_per_unit (m = 1 .. planes_per_unit-1) of the
    unit brick.  The draw is keyed by (seed, round, cell), so it does not depend
    on the order in which the leaves are listed.
    """

    def fn(cm, level, coords, finest):
        level = np.asarray(level, dtype=np.int64)
        coords = np.asarray(coords, dtype=np.int64)
        on_plane = np.zeros(len(level), dtype=bool)
        for d in range(cm.dim):
            cells = np.asarray(cm.n0[d], dtype=np.int64) << level
            # plane spacing in level-l lattice units; requires n0 * 2^l divisible
            step = cells // planes_per_unit
            ok = step * planes_per_unit == cells
            lo_face = coords[:, d]
            hi_face = coords[:, d] + 1
            for face in (lo_face, hi_face):
                m = np.where(ok, face // np.maximum(step, 1), 0)
                hit = ok & (face % np.maximum(step, 1) == 0) & (m > 0) & (m < planes_per_unit)
                on_plane |= hit
        key = cell_hash_key(level, coords) ^ (np.uint64(round_index) << np.uint64(56))
        u = uniform01(seed, key)
        return on_plane & (level == finest) & (u < prob)

    return fn


def round_random(seed: int, round_index: int, prob: float) -> RoundFn:
    """Flag each current leaf with probability ``prob``; the draw is keyed by
    (seed, round, cell), independent of the order of the leaves."""

    def fn(cm, level, coords, finest):
        level = np.asarray(level, dtype=np.int64)
        coords = np.asarray(coords, dtype=np.int64)
        key = cell_hash_key(level, coords) ^ (np.uint64(round_index + 1) << np.uint64(56))
        return uniform01(seed, key) < prob

    return fn


# ------------------------------------------------ refinement sequences of Sec. 3.5
# The meshes of the partition-efficiency study: a coarse mesh of [-1, 1]^d,
# then L rounds of one selection rule, each followed by closure.

def round_vertex_in_ball(radius: float) -> RoundFn:
    """Flag leaves with at least one vertex strictly inside |x| < radius, and
    the leaves whose closed box contains the centre (a cell around the centre
    whose vertices all lie outside the small ball, such as the single coarse
    cell [-1, 1]^d, would otherwise never be refined)."""
    r2 = float(radius) ** 2

    def fn(cm, level, coords, finest):
        blo, bhi = cm.boxes(level, coords)
        hit = np.all((blo <= 0.0) & (bhi >= 0.0), axis=1)
        for b in range(1 << cm.dim):
            v = np.where([(b >> d) & 1 for d in range(cm.dim)], bhi, blo)
            hit |= np.sum(v * v, axis=1) < r2
        return hit

    return fn


def round_negative_orthant() -> RoundFn:
    """Flag leaves whose centre has no positive coordinate (the negative
    quadrant, octant in 3D; the single coarse cell [-1, 1]^d has its centre at
    the origin, so the first round refines it)."""

    def fn(cm, level, coords, finest):
        blo, bhi = cm.boxes(level, coords)
        return np.all(0.5 * (blo + bhi) <= 0.0, axis=1)

    return fn


def sine_curve(x):
    """The curve of the "sine curve" sequence: y = 3/4 sin(3x - 5/2) + 1/5."""
    return 0.75 * np.sin(3.0 * np.asarray(x, dtype=np.float64) - 2.5) + 0.2


def round_sine_curve() -> RoundFn:
    """Flag leaves whose closed box meets the curve y = sine_curve(x) (in 3D the
    surface of all z over that curve)."""

    def fn(cm, level, coords, finest):
        blo, bhi = cm.boxes(level, coords)
        x0, x1 = blo[:, 0], bhi[:, 0]
        fmin = np.minimum(sine_curve(x0), sine_curve(x1))
        fmax = np.maximum(sine_curve(x0), sine_curve(x1))
        # interior extrema at 3x - 5/2 = pi/2 + j pi (sine = +-1)
        for j in range(-3, 3):
            xc = (2.5 + np.pi / 2 + j * np.pi) / 3.0
            inside = (x0 < xc) & (xc < x1)
            fc = float(sine_curve(xc))
            fmin = np.where(inside, np.minimum(fmin, fc), fmin)
            fmax = np.where(inside, np.maximum(fmax, fc), fmax)
        return (fmin <= bhi[:, 1]) & (fmax >= blo[:, 1])

    return fn


def round_centre_in_shell(r_in: float, r_out: float) -> RoundFn:
    """Flag leaves whose centre lies strictly between the radii r_in < |x| < r_out
    (r_in = 0: strictly inside the ball of radius r_out)."""

    def fn(cm, level, coords, finest):
        blo, bhi = cm.boxes(level, coords)
        c = 0.5 * (blo + bhi)
        d2 = np.sum(c * c, axis=1)
        return (d2 > r_in * r_in) & (d2 < r_out * r_out)

    return fn


# the "annulus" sequence's three steps after L - 3 uniform rounds: centres in
# the ball of radius 0.55, then in the shells 0.3-0.42 and 0.335-0.39 (the
# text gives 0.43 for the first shell; the per-level cell counts of the
# paper's 3D annulus table come out exactly with 0.42)
ANNULUS_STEPS = ((0.0, 0.55), (0.3, 0.42), (0.335, 0.39))


def paper_sequence(name: str, dim: int, L: int) -> List[RoundFn]:
    """Refinement rounds of the sequences of Sec. 3.5 ("uniform", "circle",
    "quadrant", "sine", "annulus") up to finest level L."""
    if name == "uniform":
        return [round_uniform()] * L
    if name == "circle":
        return [round_vertex_in_ball(1.0 / (4.0 * np.pi))] * L
    if name == "quadrant":
        return [round_negative_orthant()] * L
    if name == "sine":
        return [round_sine_curve()] * L
    if name == "annulus":
        if L < 3:
            raise ValueError("the annulus sequence needs L >= 3")
        return [round_uniform()] * (L - 3) + [round_centre_in_shell(a, b) for a, b in ANNULUS_STEPS]
    raise ValueError(f"unknown sequence {name!r}")


def paper_sequence_coarse(dim: int, n: int = 1) -> CoarseMesh:
    """[-1, 1]^d split into n^d coarse cells (n = 1: the single cell of the
    sequences; the 3D annulus table of Sec. 3.6 starts from 5^3 cells)."""
    return CoarseMesh(dim, (n, n, n if dim == 3 else 1), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0))


def checkerboard_coefficients(cm: CoarseMesh, low: float = 1.0, high: float = 100.0) -> np.ndarray:
    """Coefficient per coarse cell: ``high`` where the coarse-cell index sum is odd.

    Coarse cells are listed lexicographically with x fastest.
    """
    n = [cm.n0[d] if d < cm.dim else 1 for d in range(3)]
    iz, iy, ix = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    odd = ((ix + iy + iz) % 2 == 1).ravel()
    return np.where(odd, high, low).astype(np.float64)


def random_rhs(seed: int, n: int) -> np.ndarray:
    """Right-hand side entries U[-1, 1) for unknowns 0..n-1 in canonical order."""
    return uniform_pm1(seed, np.arange(n, dtype=np.uint64))


@dataclasses.dataclass
class Workload:
    """A synthetic problem: brick, degree, refinement rounds, coefficient, rhs."""

    name: str
    coarse: CoarseMesh
    degree: int
    rounds: List[RoundFn]
    coeff: Optional[np.ndarray]  # per coarse cell, None = 1
    rhs: str  # "sine" (manufactured u = prod sin(pi x_i)), "random" or "one" (f = 1)
    cheb_degree: int
    seed: int = 0
    tol: float = 1e-8
    smoother: str = "chebyshev"     # or "jacobi" (undamped, cheb_degree steps)
    coarse_solver: str = "cholesky"  # or "cg" / "chebyshev"


def poisson2d_circle(global_refinements: int = 3, adaptive_rounds: int = 3) -> Workload:
    """2D Poisson on [0,1]^2, Q1, 4x4 coarse quads, refined near the circle
    |x - (0.5, 0.5)| = 0.3; manufactured u = sin(pi x) sin(pi y)."""
    cm = CoarseMesh(2, (4, 4, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    rounds = [round_uniform()] * global_refinements
    rounds += [round_sphere_surface((0.5, 0.5), 0.3)] * adaptive_rounds
    return Workload(f"poisson2d_q1_circle_g{global_refinements}_a{adaptive_rounds}", cm, 1,
                    rounds, None, "sine", 2)


def poisson3d_sphere(global_refinements: int = 5, adaptive_rounds: int = 2,
                     degree: int = 2) -> Workload:
    """3D Poisson on [0,1]^3, Q2, 4^3 coarse hexes, refined near the sphere
    |x - (0.5, 0.5, 0.5)| = 0.25; manufactured u = prod sin(pi x_i)."""
    cm = CoarseMesh(3, (4, 4, 4), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    rounds = [round_uniform()] * global_refinements
    rounds += [round_sphere_surface((0.5, 0.5, 0.5), 0.25)] * adaptive_rounds
    return Workload(f"poisson3d_q{degree}_sphere_g{global_refinements}_a{adaptive_rounds}", cm,
                    degree, rounds, None, "sine", 4)


def checkerboard3d(global_refinements: int = 5, finest_level: int = 9, seed: int = 20190403,
                   prob: float = 0.3) -> Workload:
    """3D variable coefficient on [0,1]^3, Q2: a in {1, 100} on the 4x4x4 subcube
    checkerboard, refined near the subcube interfaces by seeded random rounds."""
    cm = CoarseMesh(3, (4, 4, 4), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
    rounds = [round_uniform()] * global_refinements
    for r in range(finest_level - global_refinements):
        rounds.append(round_random_interface(seed, r, prob))
    return Workload(f"checkerboard3d_q2_g{global_refinements}_L{finest_level}", cm, 2, rounds,
                    checkerboard_coefficients(cm), "random", 4, seed=seed)


def fichera_coarse() -> CoarseMesh:
    """The Fichera corner [-1, 1]^3 minus [0, 1]^3 (Sec. 4.3) as 56 coarse
    cells of size 1/2: the brick's 4^3 cells without the 8 in the removed
    octant.  (The paper's coarse mesh is the 7 unit cells; one global
    refinement of it gives these 56, on which the coefficient below is
    constant per cell.)"""
    present = tuple(not (x >= 2 and y >= 2 and z >= 2) for z in range(4) for y in range(4) for x in range(4))
    return CoarseMesh(3, (4, 4, 4), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), present)


def fichera_coefficients(cm: CoarseMesh, low: float = 1.0, high: float = 100.0) -> np.ndarray:
    """epsilon = 1 where min(x, y, z) > -1/2, else 100 (Sec. 4.3): per coarse
    cell of the Fichera mesh, ``high`` on the cells with an index 0 (they
    cover min(x, y, z) < -1/2), ``low`` elsewhere."""
    iz, iy, ix = np.meshgrid(np.arange(cm.n0[2]), np.arange(cm.n0[1]), np.arange(cm.n0[0]), indexing="ij")
    low_side = ((ix == 0) | (iy == 0) | (iz == 0)).ravel()
    return np.where(low_side, high, low).astype(np.float64)


def round_reentrant_fraction(fraction: float = 0.142) -> RoundFn:
    """Flag the given fraction of the leaves with the largest indicator
    h_K^3 / (h_K + d_K), d_K the distance from the cell centre to the
    re-entrant edges of the Fichera corner (the segments from the origin to
    (1,0,0), (0,1,0), (0,0,1)); ties go to the smaller (level, key).  It
    stands in for the a-posteriori estimator of Sec. 4.3, whose largest
    contributions sit at those edges, and refines a fixed fraction per round
    as the paper does (14.2%, which roughly doubles the cells)."""

    def fn(cm, level, coords, finest):
        blo, bhi = cm.boxes(level, coords)
        c = 0.5 * (blo + bhi)
        h = bhi[:, 0] - blo[:, 0]
        d = np.full(len(c), np.inf)
        for axis in range(3):
            t = np.clip(c[:, axis], 0.0, 1.0)
            q = np.zeros_like(c)
            q[:, axis] = t
            d = np.minimum(d, np.linalg.norm(c - q, axis=1))
        eta = h ** 3 / (h + d)
        m = int(round(fraction * len(c)))
        key = cell_hash_key(level, coords)
        order = np.lexsort((key, -eta))  # eta descending, then key ascending
        flags = np.zeros(len(c), dtype=bool)
        flags[order[:m]] = True
        return flags

    return fn


def fichera(adaptive_rounds: int = 2, global_refinements: int = 0) -> Workload:
    """The Laplace example of Sec. 4.3: -div(eps grad u) = 1 on the Fichera
    corner, u = 0 on the boundary, Q2, eps = 100 where min(x, y, z) <= -1/2;
    global refinements of the 56 coarse cells, then rounds of the
    re-entrant-edge fraction rule (closure after each).  Solver settings of
    the paper's "MF" column: one undamped Jacobi step, CG coarse solver,
    tolerance 1e-10."""
    cm = fichera_coarse()
    rounds = [round_uniform()] * global_refinements + [round_reentrant_fraction()] * adaptive_rounds
    return Workload(f"fichera_q2_g{global_refinements}_a{adaptive_rounds}", cm, 2, rounds,
                    fichera_coefficients(cm), "one", 1, tol=1e-10, smoother="jacobi", coarse_solver="cg")


# Leaf growth of r random rounds (p = 0.2, closure after each) on a uniform
# mesh, measured with this generator: the closure multiplies the count far
# beyond the (1 + p (2^d - 1))^r of the flags alone.
RANDOM_ROUND_GROWTH = {2: {3: 6.5, 4: 13.1, 5: 26.8, 6: 55.1}, 3: {3: 34.1, 4: 124.2, 5: 470.8, 6: 1732.9}}


def batched_problems(count: int = 512, seed: int = 20190404, n_min: float = 1e4, n_max: float = 5e5,
                     prob: float = 0.2):
    """Independent Poisson problems of mixed dimension, degree and size: per
    problem d in {2, 3}, k in {1, 2}, a target size N log-uniform in
    [n_min, n_max], 3..6 rounds that flag every leaf with probability prob,
    and the global level g whose expected size k^d (4 2^g)^d G(d, rounds) is
    closest to N in ratio, G the measured growth of the random rounds with
    closure (RANDOM_ROUND_GROWTH; sizes are counted, not assumed).  Coarse
    mesh 4^d on the unit brick, seeded random right-hand side, Chebyshev
    degree 2 (2D) / 4 (3D).  All draws are keyed by (seed, problem index), so
    the list does not depend on how it is consumed."""
    out = []
    for i in range(count):
        key = np.arange(6, dtype=np.uint64) + np.uint64(8 * i)
        u = uniform01(seed, key)
        dim = 2 if u[0] < 0.5 else 3
        k = 1 if u[1] < 0.5 else 2
        target = float(np.exp(np.log(n_min) + u[2] * (np.log(n_max) - np.log(n_min))))
        rounds = 3 + int(u[3] * 4)
        growth = RANDOM_ROUND_GROWTH[dim][rounds]
        sizes = [(k ** dim) * (4 * 2 ** gg) ** dim * growth for gg in range(12)]
        g = int(np.argmin([abs(np.log(sz / target)) for sz in sizes]))
        cm = CoarseMesh(dim, (4, 4, 4) if dim == 3 else (4, 4, 1), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
        rs = [round_uniform()] * g + [round_random(seed + i, r, prob) for r in range(rounds)]
        out.append(Workload(f"batch{i}_d{dim}_q{k}_g{g}_r{rounds}", cm, k, rs, None, "random",
                            2 if dim == 2 else 4, seed=seed + i))
    return out


def serving_requests(count: int, seed: int = 20190405, n_min: float = 1e4, n_max: float = 2e7,
                     rate: float = 200.0):
    """Solve requests for a request loop: Poisson arrivals at ``rate`` per
    second (exponential gaps) and, per request, a 3D Q2 problem on the unit
    cube (4^3 coarse cells) refined twice at the surface of a sphere with
    centre U[0.3, 0.7]^3 and radius U[0.15, 0.35], a random right-hand side,
    and a target size N log-uniform in [n_min, n_max] met by the choice of the
    global level g (the one whose estimated size is closest to N; sizes are
    counted, not assumed).  Returns (arrival times in s, workloads)."""
    out, times = [], []
    t = 0.0
    for i in range(count):
        key = np.arange(8, dtype=np.uint64) + np.uint64(8 * i)
        u = uniform01(seed, key)
        t += -np.log(max(1.0 - u[0], 1e-300)) / rate
        times.append(t)
        target = float(np.exp(np.log(n_min) + u[1] * (np.log(n_max) - np.log(n_min))))
        c = tuple(0.3 + 0.4 * float(v) for v in u[2:5])
        r = 0.15 + 0.2 * float(u[5])

        def est(g):
            # uniform cells, plus 7 new leaves per refined surface cell in
            # each of the two rounds (about 1.5 cells per h^2 of sphere area)
            cells = 64 * 8 ** g
            surf = lambda lvl: 1.5 * 4 * np.pi * r * r * (4 * 2 ** lvl) ** 2
            return 8 * (cells + 7 * surf(g) + 7 * surf(g + 1))

        g = int(np.argmin([abs(np.log(est(gg) / target)) for gg in range(8)]))
        cm = CoarseMesh(3, (4, 4, 4), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))
        rs = [round_uniform()] * g + [round_sphere_surface(c, r)] * 2
        out.append(Workload(f"request{i}_g{g}", cm, 2, rs, None, "random", 4, seed=seed + 1000 + i))
    return np.asarray(times), out

