"""Shared test helpers: build the same workload on both sides and map vectors."""
import dataclasses
import functools

import numpy as np

from oracle import fem, gmg as ogmg
from oracle.mesh import build_forest
from paper_1904_03317_gb300 import gmg as G
from paper_1904_03317_gb300 import inputs


def small_workloads():
    """Workloads the oracle finishes in seconds that still span many groups,
    ghost blocks, hanging nodes and a ragged last block of cells."""
    # anisotropic cells (0.5 x 0.5 x 0.4) keep the general-scale kernels covered
    cm3 = inputs.CoarseMesh(3, (3, 2, 2), (0.0, 0.0, 0.0), (1.5, 1.0, 0.8))
    return {
        "2d_q1_circle": inputs.poisson2d_circle(3, 3),
        "2d_q2_circle": inputs.Workload("2d_q2", inputs.CoarseMesh(2, (4, 3, 1), (0, 0, 0), (1.0, 0.75, 1)), 2,
                                        [inputs.round_uniform()] * 2 + [inputs.round_sphere_surface((0.5, 0.4), 0.27)] * 2,
                                        None, "sine", 3),
        "3d_q2_sphere": inputs.poisson3d_sphere(1, 2),
        "3d_q1_sphere": inputs.poisson3d_sphere(2, 2, degree=1),
        # leaf patches (4x4x4 cells), groups and single cells side by side
        "3d_q2_patches": inputs.Workload("3d_q2_patches",
                                         inputs.CoarseMesh(3, (3, 2, 2), (0.0, 0.0, 0.0), (1.5, 1.0, 1.0)), 2,
                                         [inputs.round_uniform()] * 2
                                         + [inputs.round_sphere_surface((0.3, 0.3, 0.3), 0.12)],
                                         None, "sine", 4),
        "3d_q2_checker": inputs.Workload("3d_q2_checker", cm3, 2,
                                         [inputs.round_uniform(), inputs.round_uniform(),
                                          inputs.round_sphere_surface((0.7, 0.5, 0.4), 0.3)],
                                         np.array([1.0, 100.0, 3.0, 1.0, 50.0, 1.0, 7.0, 1.0, 1.0, 100.0, 2.0, 1.0]),
                                         "random", 4, seed=7),
        # the Fichera corner (Sec. 4.3): a brick without one octant, Dirichlet
        # on the re-entrant faces, coefficient jumps of 100 inside the domain;
        # here with the Chebyshev smoother of degree 4 that the step-by-step
        # parity tests use (the paper's own solver settings for it are tested
        # on their own)
        "3d_q2_fichera": dataclasses.replace(inputs.fichera(3, 1), cheb_degree=4, smoother="chebyshev",
                                             coarse_solver="cholesky"),
    }


@functools.lru_cache(maxsize=None)
def oracle_hierarchy(name: str, cheb: int = None):
    w = small_workloads()[name]
    f = build_forest(w.coarse, w.rounds)
    d = fem.Discretization(f, w.degree, w.coeff)
    return ogmg.build_hierarchy(d, cheb or w.cheb_degree)


def workload_rhs(O, w):
    """The workload's right-hand side on the oracle's unknowns."""
    if w.rhs == "sine":
        return O.disc.rhs_sine()
    if w.rhs == "one":
        return O.disc.rhs_one()
    return inputs.random_rhs(w.seed, O.disc.n)


def level_maps(H, O, level):
    """For level `level`: slot -> oracle index arrays (S∪I), slot classes."""
    keys = H.export(G.EXPORT_LEVEL_KEYS, level)
    cls = H.export(G.EXPORT_LEVEL_CLASS, level)
    lev = O.levels[level]
    used = (cls == 1) | (cls == 2)
    idx = np.full(len(keys), -1, dtype=np.int64)
    idx[used] = fem.lookup(lev.keys, keys[used])
    assert np.all(idx[used] >= 0)
    return idx, cls


def to_slots(vec_oracle, idx, n_slots):
    out = np.zeros(n_slots)
    m = idx >= 0
    out[m] = vec_oracle[idx[m]]
    return out


def from_slots(vec_slots, idx, n):
    out = np.zeros(n)
    m = idx >= 0
    out[idx[m]] = vec_slots[m]
    return out
