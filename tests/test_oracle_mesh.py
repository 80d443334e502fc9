"""Pins of the oracle's forest and closure (CPU only).

The closure must give a leaf set in which any two leaves whose closures touch
differ by at most one level (Sec. 3.5, one-irregular meshes of Sec. 1), and it
must be the minimal such refinement of the requested one.  Both are checked by
brute force on small meshes, independently of the oracle's own algorithm.
"""
import itertools

import numpy as np
import pytest

from oracle.mesh import Forest, build_forest
from paper_1904_03317_gb300 import inputs


def _touch(cm, a, b):
    """Do the closed boxes of leaves a=(l, c) and b touch?  (exact rational test)"""
    (la, ca), (lb, cb) = a, b
    L = max(la, lb)
    for d in range(cm.dim):
        a0, a1 = ca[d] << (L - la), (ca[d] + 1) << (L - la)
        b0, b1 = cb[d] << (L - lb), (cb[d] + 1) << (L - lb)
        if a1 < b0 or b1 < a0:
            return False
    return True


def _brute_balanced(f):
    lv = f.leaves()
    for a, b in itertools.combinations(lv, 2):
        if abs(a[0] - b[0]) > 1 and _touch(f.cm, a, b):
            return False
    return True


def _covering(f, level, c):
    return all(0 <= c[d] < (f.n0[d] << level) for d in range(f.dim))


def _small_cases():
    cm2 = inputs.CoarseMesh(2, (2, 3, 1), (0, 0, 0), (1.0, 1.5, 1))
    cm3 = inputs.CoarseMesh(3, (2, 2, 2), (0, 0, 0), (1, 1, 1))
    # a tiny circle inside one cell, away from the boundary: each round refines
    # one or a few finest cells, which forces a cascade of closure refinements
    corner2 = [inputs.round_sphere_surface((0.4301, 0.6701), 0.003, finest_only=True)] * 5
    corner3 = [inputs.round_sphere_surface((0.4301, 0.3701, 0.5501), 0.003, finest_only=True)] * 4
    return [(cm2, corner2), (cm3, corner3),
            (cm2, [inputs.round_uniform(), inputs.round_sphere_surface((0.5, 0.7), 0.3)] * 2)]


@pytest.mark.parametrize("case", range(3))
def test_closure_balanced_by_brute_force(case):
    cm, rounds = _small_cases()[case]
    f = build_forest(cm, rounds)
    assert f.num_levels() >= 4
    assert _brute_balanced(f)


@pytest.mark.parametrize("case", range(3))
def test_closure_minimal(case):
    """No refinement that closure added can be undone without breaking balance.

    The balanced refinements containing the requested one are closed under
    intersection, so a refinement from which no single closure-added cell
    can be removed is the unique minimum.
    """
    cm, rounds = _small_cases()[case]
    f = Forest(cm)
    requested = set()
    for fn in rounds:
        level, coords = f.leaf_arrays()
        flags = fn(cm, level, coords, int(level.max()))
        for l, c, fl in zip(level.tolist(), coords.tolist(), flags):
            if fl:
                requested.add((l, tuple(c)))
        f.refine(flags)
    for l in range(f.num_levels() - 1):
        for c in list(f.refined[l]):
            if (l, c) in requested:
                continue
            kids = [tuple(2 * c[d] + b[d] if d < f.dim else 0 for d in range(3))
                    for b in itertools.product(*[(0, 1) if d < f.dim else (0,) for d in range(3)])]
            if any(k in f.refined[l + 1] for k in kids):
                continue
            # undo this one refinement and check that balance breaks
            f.refined[l].discard(c)
            for k in kids:
                f.cells[l + 1].discard(k)
            assert not _brute_balanced(f), f"refinement of {(l, c)} was not forced"
            f.refined[l].add(c)
            for k in kids:
                f.cells[l + 1].add(k)


def test_closure_idempotent():
    cm, rounds = _small_cases()[1]
    f = build_forest(cm, rounds)
    before = [set(s) for s in f.cells]
    f.close()
    assert [set(s) for s in f.cells] == before
    f.refine(np.zeros(len(f.leaves()), dtype=bool))
    assert [set(s) for s in f.cells] == before


def test_complete_layer():
    """A complete layer of level l-1 cells surrounds the level-l cells (Sec. 2.3):
    every in-domain lattice neighbour of a refined cell exists."""
    w = inputs.poisson2d_circle(2, 3)
    f = build_forest(w.coarse, w.rounds)
    for l in range(1, f.num_levels()):
        for c in f.refined[l]:
            for o in f.neighbour_offsets():
                n = tuple(c[d] + o[d] for d in range(3))
                if _covering(f, l, n):
                    assert f.exists(l, n)


def test_leaves_tile_the_domain():
    cm, rounds = _small_cases()[0]
    f = build_forest(cm, rounds)
    L = f.num_levels() - 1
    area = sum(4.0 ** (L - l) for l, _ in f.leaves())
    assert area == cm.n0[0] * cm.n0[1] * 4.0 ** L
