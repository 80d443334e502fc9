"""Oracle of the partition-efficiency model (test infrastructure only).

The model of the paper's parallel-complexity section: every cell of every
level of the hierarchy costs one unit of work.  Leaves are split into n_p
contiguous pieces of the space-filling-curve order (depth-first over the
forest, children in z-order), processor p taking leaves [p N / n_p, (p+1) N /
n_p) (integer division).  A refined cell belongs to the owner of its first
child, recursively (the "first-child rule").  With N_l the cells of level l
and N_{l,p} those owned by p:

    W_opt  = (sum_l N_l) / n_p          (perfect balance)
    W_sync = sum_l ceil(N_l / n_p)      (balance within each level)
    W      = sum_l max_p N_{l,p}        (the partition at hand)
    E      = W_opt / W

The coarse solve counts as level 0 with one unit per coarse cell, as in the
paper's worked example.  Plain Python over the oracle's forest; shares no
code with the library.
"""
from __future__ import annotations

import math
from typing import Dict, List, Tuple

from oracle.mesh import Forest


def _dfs_leaves(f: Forest) -> List[Tuple[int, Tuple[int, int, int]]]:
    """Leaves in depth-first order: the domain's coarse cells in lexicographic
    (z, y, x) order, children in z-order (x bit first, then y, then z)."""
    out = []

    def visit(level, c):
        if c in f.refined[level]:
            for b in range(1 << f.dim):
                ch = tuple(2 * c[d] + ((b >> d) & 1) if d < f.dim else 0 for d in range(3))
                visit(level + 1, ch)
        else:
            out.append((level, c))

    for z in range(f.n0[2]):
        for y in range(f.n0[1]):
            for x in range(f.n0[0]):
                if f.exists(0, (x, y, z)):  # coarse cells of the domain only
                    visit(0, (x, y, z))
    return out


def owners(f: Forest, n_parts: int) -> List[Dict[Tuple[int, int, int], int]]:
    """Owner of every cell of every level under the first-child rule."""
    leaves = _dfs_leaves(f)
    n = len(leaves)
    own: List[Dict[Tuple[int, int, int], int]] = [dict() for _ in range(f.num_levels())]
    for i, (l, c) in enumerate(leaves):
        own[l][c] = i * n_parts // n
    for l in range(f.num_levels() - 2, -1, -1):
        for c in f.refined[l]:
            first = tuple(2 * c[d] if d < f.dim else 0 for d in range(3))
            own[l][c] = own[l + 1][first]
    return own


def model(f: Forest, n_parts: int) -> Dict[str, object]:
    own = owners(f, n_parts)
    n_l = [len(f.cells[l]) for l in range(f.num_levels())]
    w_l = []
    for l in range(f.num_levels()):
        counts = [0] * n_parts
        for c in f.cells[l]:
            counts[own[l][c]] += 1
        w_l.append(max(counts))
    w_opt = sum(n_l) / n_parts
    w_sync = sum(math.ceil(x / n_parts) for x in n_l)
    w = sum(w_l)
    return {"n_cells": n_l, "w_level": w_l, "w_opt": w_opt, "w_sync": w_sync, "w": w, "efficiency": w_opt / w}
