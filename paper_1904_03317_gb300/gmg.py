"""Thin ctypes binding of libgmg (include/gmg.h).

Argument marshalling only: every step of the solver runs in the library.
PyTorch tensors are accepted for device vectors (their data_ptr() is passed);
PyTorch is used for device memory and streams, nothing else.  The library is
loaded from the package's lib/ directory; if it is missing this module raises
instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

from .inputs import CoarseMesh, Workload

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libgmg.so")

MAX_LEVELS = 24
OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, EBREAKDOWN, ENAN, ETIMEOUT, EUNSUPPORTED = range(9)
PREC_FP64, PREC_FP32 = 0, 1
SMOOTHER_CHEBYSHEV, SMOOTHER_JACOBI = 0, 1
COARSE_CHOLESKY, COARSE_CHEBYSHEV, COARSE_CG = 0, 1, 2
RHS_SINE, RHS_RANDOM, RHS_ONE = 0, 1, 2
EXPORT_UNKNOWN_KEYS, EXPORT_HOME_LEVEL, EXPORT_HANGING, EXPORT_LEVEL_KEYS, EXPORT_LEVEL_CLASS, \
    EXPORT_HOME_SLOT = range(6)

STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOTCONV", 5: "EBREAKDOWN",
                6: "ENAN", 7: "ETIMEOUT", 8: "EUNSUPPORTED"}

# every symbol include/gmg.h declares
EXPORTED = [
    "gmg_create", "gmg_destroy", "gmg_last_error", "gmg_build_info",
    "gmg_mesh_create", "gmg_mesh_destroy", "gmg_mesh_num_leaves", "gmg_mesh_num_levels",
    "gmg_mesh_leaves", "gmg_mesh_refine", "gmg_mesh_partition_model",
    "gmg_params_default", "gmg_hier_build", "gmg_build_hierarchy", "gmg_hier_destroy", "gmg_hier_info",
    "gmg_hier_export",
    "gmg_assemble_rhs", "gmg_apply", "gmg_vcycle", "gmg_solve", "gmg_solve_batch", "gmg_solve_async", "gmg_solve_poll",
    "gmg_level_apply", "gmg_level_residual_restrict", "gmg_level_prolongate", "gmg_level_smooth",
    "gmg_level_inv_diag", "gmg_coarse_solve", "gmg_profile_reset", "gmg_profile_read",
    "gmg_level_smooth_noalloc",
]

KERNEL_KINDS = ["cheb", "smooth_first", "residual_restrict", "prolongate", "coarse", "copy_to_mg",
                "copy_from_mg", "active_apply", "cg_update_xr", "cg_update_p", "other"]


class GmgError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class CoarseMeshC(C.Structure):
    _fields_ = [("dim", C.c_int), ("n0", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("present", C.c_void_p)]


def _coarse_struct(coarse: CoarseMesh):
    """gmg_coarse_mesh of an inputs.CoarseMesh, and the mask array it points to
    (kept alive by the caller for the duration of the call)."""
    cm = CoarseMeshC()
    cm.dim = coarse.dim
    for d in range(3):
        cm.n0[d] = int(coarse.n0[d]) if d < coarse.dim else 1
        cm.lo[d] = float(coarse.lo[d])
        cm.hi[d] = float(coarse.hi[d])
    mask = None
    if getattr(coarse, "present", None) is not None:
        mask = np.ascontiguousarray(np.asarray(coarse.present, dtype=np.uint8))
        cm.present = mask.ctypes.data
    return cm, mask


# gmg_refine_fn: (user, round, n_leaves, level*, coords*, flags*) -> int
REFINE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.c_uint64, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                        C.POINTER(C.c_uint8))


class ParamsC(C.Structure):
    _fields_ = [("cheb_degree", C.c_int), ("eig_lo", C.c_double), ("eig_hi", C.c_double),
                ("eig_iters", C.c_int), ("vcycle_prec", C.c_int),
                ("fixed_lambda", C.POINTER(C.c_double)), ("smoother", C.c_int), ("coarse_solver", C.c_int),
                ("coarse_tol", C.c_double), ("solve_graph", C.c_int), ("deterministic", C.c_int),
                ("brick_min_members", C.c_int)]


class PartitionModelC(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("n_cells", C.c_double * MAX_LEVELS), ("w_level", C.c_double * MAX_LEVELS),
                ("w_opt", C.c_double), ("w_sync", C.c_double), ("w", C.c_double), ("efficiency", C.c_double)]


class InfoC(C.Structure):
    _fields_ = [("dim", C.c_int), ("degree", C.c_int), ("n_levels", C.c_int), ("vcycle_prec", C.c_int),
                ("n_unknowns", C.c_uint64), ("n_leaves", C.c_uint64), ("n_hanging", C.c_uint64),
                ("n_leaf_nodes", C.c_uint64),
                ("cells", C.c_uint64 * MAX_LEVELS), ("leaves", C.c_uint64 * MAX_LEVELS),
                ("groups", C.c_uint64 * MAX_LEVELS), ("ghosts", C.c_uint64 * MAX_LEVELS),
                ("slots", C.c_uint64 * MAX_LEVELS), ("n_S", C.c_uint64 * MAX_LEVELS),
                ("n_I", C.c_uint64 * MAX_LEVELS), ("n_home", C.c_uint64 * MAX_LEVELS),
                ("bricks", C.c_uint64 * MAX_LEVELS), ("groups_jump", C.c_uint64 * MAX_LEVELS),
                ("lambda_max", C.c_double * MAX_LEVELS), ("device_bytes", C.c_uint64),
                ("setup_host_s", C.c_double), ("setup_device_s", C.c_double),
                ("leaf_patches", C.c_uint64), ("leaf_groups", C.c_uint64), ("leaf_single_cells", C.c_uint64),
                ("coarse_degree", C.c_int), ("coarse_range", C.c_double * 2), ("setup_phase_s", C.c_double * 8),
                ("bricks_partial", C.c_uint64 * MAX_LEVELS)]


class KernelStatsC(C.Structure):
    _fields_ = [("launches", C.c_uint64 * 11), ("ms", C.c_double * 11), ("bytes", C.c_double * 11),
                ("flops", C.c_double * 11)]


class StatsC(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("rel_residual", C.c_double),
                ("norm_b", C.c_double)]


_lib = None


def load_library(path: Optional[str] = None) -> C.CDLL:
    """Load libgmg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"{p} is missing: build it with paper_1904_03317_gb300.build.build()")
    lib = C.CDLL(p)
    vp, i32, u64, dp = C.c_void_p, C.c_int, C.c_uint64, C.POINTER(C.c_double)
    sig = {
        "gmg_create": [i32, vp, C.POINTER(vp)],
        "gmg_destroy": [vp],
        "gmg_last_error": [],
        "gmg_build_info": [C.POINTER(i32), C.POINTER(i32)],
        "gmg_mesh_create": [C.POINTER(CoarseMeshC), C.POINTER(vp)],
        "gmg_mesh_destroy": [vp],
        "gmg_mesh_num_leaves": [vp, C.POINTER(u64)],
        "gmg_mesh_num_levels": [vp, C.POINTER(i32)],
        "gmg_mesh_leaves": [vp, vp, vp],
        "gmg_mesh_refine": [vp, vp, u64],
        "gmg_mesh_partition_model": [vp, C.c_int64, C.POINTER(PartitionModelC)],
        "gmg_params_default": [C.POINTER(ParamsC)],
        "gmg_hier_build": [vp, vp, i32, vp, C.POINTER(ParamsC), C.POINTER(vp)],
        "gmg_build_hierarchy": [vp, C.POINTER(CoarseMeshC), i32, REFINE_FN, vp, i32, vp, C.POINTER(ParamsC),
                                C.POINTER(vp)],
        "gmg_hier_destroy": [vp],
        "gmg_hier_info": [vp, C.POINTER(InfoC)],
        "gmg_hier_export": [vp, i32, i32, vp, C.POINTER(u64)],
        "gmg_assemble_rhs": [vp, i32, u64, vp],
        "gmg_apply": [vp, vp, vp],
        "gmg_vcycle": [vp, vp, vp],
        "gmg_solve": [vp, vp, vp, C.c_double, i32, i32, C.POINTER(StatsC)],
        "gmg_solve_batch": [vp, vp, vp, i32, C.c_double, i32, i32, vp, vp],
        "gmg_solve_async": [vp, vp, vp, C.c_double, i32],
        "gmg_solve_poll": [vp, i32, C.POINTER(i32), C.POINTER(StatsC), C.POINTER(i32)],
        "gmg_level_apply": [vp, i32, vp, vp],
        "gmg_level_residual_restrict": [vp, i32, vp, vp, vp],
        "gmg_level_prolongate": [vp, i32, vp, vp, vp],
        "gmg_level_smooth": [vp, i32, vp, vp, vp, i32],
        "gmg_level_smooth_noalloc": [vp, i32, vp, vp, i32],
        "gmg_level_inv_diag": [vp, i32, vp],
        "gmg_coarse_solve": [vp, vp, vp],
        "gmg_profile_reset": [vp, i32],
        "gmg_profile_read": [vp, C.POINTER(KernelStatsC)],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = None if name in ("gmg_destroy", "gmg_mesh_destroy", "gmg_hier_destroy",
                                      "gmg_params_default") else C.c_int
    lib.gmg_last_error.restype = C.c_char_p
    if path is None:
        _lib = lib
    return lib


def _check(status: int, where: str) -> None:
    if status != OK:
        raise GmgError(status, where, load_library().gmg_last_error().decode())


def _ptr(t) -> C.c_void_p:
    """Device or host address of a torch tensor or numpy array."""
    if t is None:
        return C.c_void_p(0)
    if isinstance(t, np.ndarray):
        return C.c_void_p(t.ctypes.data)
    return C.c_void_p(t.data_ptr())


class Context:
    """Device (or host-only, device=-1) context with the CUDA stream all work goes to."""

    def __init__(self, device: int = 0, stream: Optional[int] = None):
        lib = load_library()
        if device >= 0 and stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        h = C.c_void_p()
        _check(lib.gmg_create(device, C.c_void_p(stream or 0), C.byref(h)), "gmg_create")
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            load_library().gmg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    """Forest of a Cartesian brick with 2:1-balanced refinement (gmg_mesh_*)."""

    def __init__(self, coarse: CoarseMesh):
        lib = load_library()
        cm, mask = _coarse_struct(coarse)
        self.coarse = coarse
        h = C.c_void_p()
        _check(lib.gmg_mesh_create(C.byref(cm), C.byref(h)), "gmg_mesh_create")
        self.handle = h

    def num_leaves(self) -> int:
        n = C.c_uint64()
        _check(load_library().gmg_mesh_num_leaves(self.handle, C.byref(n)), "gmg_mesh_num_leaves")
        return n.value

    def num_levels(self) -> int:
        n = C.c_int()
        _check(load_library().gmg_mesh_num_levels(self.handle, C.byref(n)), "gmg_mesh_num_levels")
        return n.value

    def leaves(self):
        n = self.num_leaves()
        level = np.zeros(n, dtype=np.int32)
        coords = np.zeros((n, 3), dtype=np.int32)
        _check(load_library().gmg_mesh_leaves(self.handle, _ptr(level), _ptr(coords)), "gmg_mesh_leaves")
        return level, coords

    def partition_model(self, n_parts: int) -> dict:
        """Partitioning efficiency model (W_opt, W_sync, W, E) for n_parts parts."""
        m = PartitionModelC()
        _check(load_library().gmg_mesh_partition_model(self.handle, int(n_parts), C.byref(m)),
               "gmg_mesh_partition_model")
        L = m.n_levels
        return {"n_cells": [int(v) for v in m.n_cells[:L]], "w_level": [int(v) for v in m.w_level[:L]],
                "w_opt": m.w_opt, "w_sync": m.w_sync, "w": m.w, "efficiency": m.efficiency}

    def refine(self, flags) -> None:
        f = np.ascontiguousarray(np.asarray(flags, dtype=np.uint8))
        _check(load_library().gmg_mesh_refine(self.handle, _ptr(f), C.c_uint64(len(f))), "gmg_mesh_refine")

    def apply_rounds(self, rounds) -> None:
        for fn in rounds:
            level, coords = self.leaves()
            self.refine(fn(self.coarse, level.astype(np.int64), coords.astype(np.int64), int(level.max())))

    def close(self):
        if self.handle:
            load_library().gmg_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_params(cheb_degree: int = 5, vcycle_prec: int = PREC_FP32, eig_lo: float = 0.08, eig_hi: float = 1.2,
                 eig_iters: int = 10, fixed_lambda: Optional[Sequence[float]] = None, solve_graph: bool = True,
                 smoother: int = 0, coarse_solver: int = 0, coarse_tol: float = 1e-3, deterministic: bool = False,
                 brick_min_members: int = 0):
    """gmg_params from keyword arguments; returns (params, array to keep alive)."""
    p = ParamsC()
    load_library().gmg_params_default(C.byref(p))
    p.cheb_degree, p.eig_lo, p.eig_hi, p.eig_iters, p.vcycle_prec = cheb_degree, eig_lo, eig_hi, eig_iters, vcycle_prec
    p.solve_graph = int(solve_graph)
    p.deterministic, p.brick_min_members = int(deterministic), int(brick_min_members)
    p.smoother, p.coarse_solver, p.coarse_tol = smoother, coarse_solver, coarse_tol
    lam = None
    if fixed_lambda is not None:
        lam = np.ascontiguousarray(np.asarray(fixed_lambda, dtype=np.float64))
        p.fixed_lambda = lam.ctypes.data_as(C.POINTER(C.c_double))
    return p, lam


class Hierarchy:
    """Multigrid hierarchy of a mesh (gmg_hier_*), with the solve-path calls."""

    def __init__(self, ctx: Context, mesh: Mesh, degree: int, coarse_coeff=None, **params):
        """params: cheb_degree (5), vcycle_prec (PREC_FP32), eig_lo (0.08), eig_hi (1.2),
        eig_iters (10), fixed_lambda (None), solve_graph (True), smoother (0),
        coarse_solver (0), coarse_tol (1e-3), deterministic (False),
        brick_min_members (0: default 4) -- the fields of gmg_params."""
        p, keep = _make_params(**params)
        coeff = None if coarse_coeff is None else np.ascontiguousarray(np.asarray(coarse_coeff, dtype=np.float64))
        h = C.c_void_p()
        _check(load_library().gmg_hier_build(ctx.handle, mesh.handle, degree, _ptr(coeff), C.byref(p), C.byref(h)),
               "gmg_hier_build")
        self._attach(ctx, h, p.vcycle_prec, keep)

    def _attach(self, ctx: Context, handle: C.c_void_p, prec: int, keep) -> None:
        self.handle = handle
        self.ctx = ctx
        self._lam = keep
        self.info = self.get_info()
        self.n = int(self.info.n_unknowns)
        self.prec = prec

    def get_info(self) -> InfoC:
        info = InfoC()
        _check(load_library().gmg_hier_info(self.handle, C.byref(info)), "gmg_hier_info")
        return info

    def export(self, what: int, level: int = 0) -> np.ndarray:
        lib = load_library()
        n = C.c_uint64(0)
        _check(lib.gmg_hier_export(self.handle, what, level, None, C.byref(n)), "gmg_hier_export")
        if what == EXPORT_HANGING:
            out = np.zeros(n.value, dtype=[("key", "<i8"), ("master", "<i8"), ("w", "<f8")])
        else:
            dt = {EXPORT_UNKNOWN_KEYS: np.int64, EXPORT_HOME_LEVEL: np.int32, EXPORT_LEVEL_KEYS: np.int64,
                  EXPORT_LEVEL_CLASS: np.int8, EXPORT_HOME_SLOT: np.int64}[what]
            out = np.zeros(n.value, dtype=dt)
        _check(lib.gmg_hier_export(self.handle, what, level, _ptr(out), C.byref(n)), "gmg_hier_export")
        return out

    # ---- solve path (device FP64 active vectors)
    def assemble_rhs(self, b, kind: str = "sine", seed: int = 0) -> None:
        """gmg_assemble_rhs: kind "sine" (manufactured solution), "one" (f = 1)
        or "random" (U[-1, 1) per unknown from `seed`, as inputs.random_rhs)."""
        k = {"sine": RHS_SINE, "random": RHS_RANDOM, "one": RHS_ONE}[kind]
        _check(load_library().gmg_assemble_rhs(self.handle, k, C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), _ptr(b)),
               "gmg_assemble_rhs")

    def apply(self, x, y) -> None:
        _check(load_library().gmg_apply(self.handle, _ptr(x), _ptr(y)), "gmg_apply")

    def vcycle(self, r, z) -> None:
        _check(load_library().gmg_vcycle(self.handle, _ptr(r), _ptr(z)), "gmg_vcycle")

    def solve(self, b, x, tol: float = 1e-8, max_iter: int = 1000, fixed_iterations: int = 0,
              raise_on_error: bool = True) -> StatsC:
        st = StatsC()
        status = load_library().gmg_solve(self.handle, _ptr(b), _ptr(x), tol, max_iter, fixed_iterations,
                                          C.byref(st))
        self.last_status = status
        if raise_on_error:
            _check(status, "gmg_solve")
        return st

    # ---- level operations on slot-layout device vectors
    def level_apply(self, level, x, y):
        _check(load_library().gmg_level_apply(self.handle, level, _ptr(x), _ptr(y)), "gmg_level_apply")

    def level_residual_restrict(self, level, u, g, gc):
        _check(load_library().gmg_level_residual_restrict(self.handle, level, _ptr(u), _ptr(g), _ptr(gc)),
               "gmg_level_residual_restrict")

    def level_prolongate(self, level, uc, u, u2):
        _check(load_library().gmg_level_prolongate(self.handle, level, _ptr(uc), _ptr(u), _ptr(u2)),
               "gmg_level_prolongate")

    def level_smooth(self, level, g, u, tmp, from_zero: bool):
        _check(load_library().gmg_level_smooth(self.handle, level, _ptr(g), _ptr(u), _ptr(tmp), int(from_zero)),
               "gmg_level_smooth")

    def level_smooth_noalloc(self, level, g, u, from_zero: bool):
        """gmg_level_smooth with the library's static scratch instead of a caller buffer."""
        _check(load_library().gmg_level_smooth_noalloc(self.handle, level, _ptr(g), _ptr(u), int(from_zero)),
               "gmg_level_smooth_noalloc")

    def level_inv_diag(self, level, out):
        _check(load_library().gmg_level_inv_diag(self.handle, level, _ptr(out)), "gmg_level_inv_diag")

    def coarse_solve(self, g0, u0):
        _check(load_library().gmg_coarse_solve(self.handle, _ptr(g0), _ptr(u0)), "gmg_coarse_solve")

    def solve_async(self, b, x, tol: float = 1e-8, max_iter: int = 1000) -> None:
        """Enqueue a graph-mode solve on the context stream (gmg_solve_async)."""
        _check(load_library().gmg_solve_async(self.handle, _ptr(b), _ptr(x), tol, max_iter), "gmg_solve_async")

    def solve_poll(self, wait: bool = False):
        """(ready, stats, status) of the pending asynchronous solve."""
        ready, st, status = C.c_int(0), StatsC(), C.c_int(0)
        _check(load_library().gmg_solve_poll(self.handle, int(wait), C.byref(ready), C.byref(st), C.byref(status)),
               "gmg_solve_poll")
        return bool(ready.value), st, status.value

    def profile_reset(self, timing: bool = False):
        _check(load_library().gmg_profile_reset(self.handle, int(timing)), "gmg_profile_reset")

    def profile_read(self) -> dict:
        st = KernelStatsC()
        _check(load_library().gmg_profile_read(self.handle, C.byref(st)), "gmg_profile_read")
        return {name: {"launches": int(st.launches[i]), "ms": float(st.ms[i]), "bytes": float(st.bytes[i]),
                       "flops": float(st.flops[i])} for i, name in enumerate(KERNEL_KINDS)}

    def close(self):
        if self.handle:
            load_library().gmg_hier_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(hiers, bs, xs, tol: float = 1e-8, max_iter: int = 1000, n_streams: int = 16):
    """Batched solves (gmg_solve_batch): hiers[i] x_i = b_i for device tensors
    b_i, x_i.  Returns (stats list, status list)."""
    n = len(hiers)
    H = (C.c_void_p * n)(*[h.handle for h in hiers])
    B = (C.c_void_p * n)(*[_ptr(b) for b in bs])
    X = (C.c_void_p * n)(*[_ptr(x) for x in xs])
    st = (StatsC * n)()
    status = (C.c_int * n)()
    rc = load_library().gmg_solve_batch(H, B, X, n, tol, max_iter, n_streams, st, status)
    if rc not in (OK, ENOTCONV, ENAN, EBREAKDOWN):
        _check(rc, "gmg_solve_batch")
    return list(st), list(status)


def build_mesh(workload: Workload) -> Mesh:
    m = Mesh(workload.coarse)
    m.apply_rounds(workload.rounds)
    return m


def build_hierarchy(ctx: Context, coarse: CoarseMesh, rounds, degree: int, coarse_coeff=None,
                    **params) -> "Hierarchy":
    """gmg_build_hierarchy: forest, refinement rounds (each a function of the
    current leaves, as in Mesh.apply_rounds) and hierarchy in one call."""
    lib = load_library()
    cm, mask = _coarse_struct(coarse)
    rounds = list(rounds)
    failure = []

    def refine(user, r, n, level_p, coords_p, flags_p):
        try:
            level = np.ctypeslib.as_array(level_p, shape=(n,)).astype(np.int64)
            coords = np.ctypeslib.as_array(coords_p, shape=(n, 3)).astype(np.int64)
            flags = np.asarray(rounds[r](coarse, level, coords, int(level.max()) if n else 0), dtype=bool)
            np.ctypeslib.as_array(flags_p, shape=(n,))[:] = flags.astype(np.uint8)
            return 0
        except Exception as e:  # an exception must not cross the C frames
            failure.append(e)
            return 1

    cb = REFINE_FN(refine)
    p, keep = _make_params(**params)
    coeff = None if coarse_coeff is None else np.ascontiguousarray(np.asarray(coarse_coeff, dtype=np.float64))
    h = C.c_void_p()
    status = lib.gmg_build_hierarchy(ctx.handle, C.byref(cm), len(rounds), cb, None, degree, _ptr(coeff),
                                     C.byref(p), C.byref(h))
    if failure:
        raise failure[0]
    _check(status, "gmg_build_hierarchy")
    H = Hierarchy.__new__(Hierarchy)
    H._attach(ctx, h, p.vcycle_prec, keep)
    return H
