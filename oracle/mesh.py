"""Oracle forest on a Cartesian brick (test infrastructure only).

A cell is named by its level l and integer lattice coordinates c (3 entries,
unused dimensions 0); the level-l lattice has n0[d] * 2^l cells along
dimension d.  The children of (l, c) are (l+1, 2c + b) for b in {0,1}^dim
(isotropic refinement into 2^d children, Sec. 2.2).

Closure (Sec. 3.5, and the one-irregular rule of Sec. 1): two leaves that
share a degree of freedom -- for continuous elements, any point of their
closures -- differ by at most one level.  The oracle restores it by a plain
fixed-point iteration: while some refined cell has a lattice neighbour at its
own level (inside the domain) that does not exist, refine the leaf that
covers that neighbour.  Every refinement it makes is forced, so the result is
the unique minimal balanced refinement.
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Set, Tuple

import numpy as np

Cell = Tuple[int, int, int]


class Forest:
    def __init__(self, coarse):
        self.cm = coarse
        self.dim = coarse.dim
        self.n0 = [int(coarse.n0[d]) if d < self.dim else 1 for d in range(3)]
        # the domain is the union of the present coarse cells (all of the brick
        # unless the coarse mesh lists some as absent)
        self.present = None if getattr(coarse, "present", None) is None else \
            [bool(v) for v in coarse.present]
        coarse_cells = set(c for c in itertools.product(range(self.n0[0]), range(self.n0[1]), range(self.n0[2]))
                           if self.coarse_present(c))
        # cells[l]: coordinates (x, y, z) of every existing cell of level l
        self.cells: List[Set[Cell]] = [coarse_cells]
        # refined[l]: existing cells of level l that have children
        self.refined: List[Set[Cell]] = [set()]

    # ---------------------------------------------------------------- queries
    def extent(self, level: int) -> List[int]:
        return [self.n0[d] << level if d < self.dim else 1 for d in range(3)]

    def coarse_present(self, c: Cell) -> bool:
        return self.present is None or self.present[c[0] + self.n0[0] * (c[1] + self.n0[1] * c[2])]

    def inside(self, level: int, c: Cell) -> bool:
        """Whether lattice cell c of level l lies in the domain: inside the
        brick and in a present coarse cell."""
        ext = self.extent(level)
        if not all(0 <= c[d] < ext[d] for d in range(3)):
            return False
        return self.coarse_present(tuple(c[d] >> level if d < self.dim else 0 for d in range(3)))

    def exists(self, level: int, c: Cell) -> bool:
        return level < len(self.cells) and c in self.cells[level]

    def is_leaf(self, level: int, c: Cell) -> bool:
        return self.exists(level, c) and c not in self.refined[level]

    def num_levels(self) -> int:
        return len(self.cells)

    def leaves(self) -> List[Tuple[int, Cell]]:
        out = []
        for l in range(len(self.cells)):
            for c in sorted(self.cells[l] - self.refined[l]):
                out.append((l, c))
        return out

    def leaf_arrays(self):
        lv = self.leaves()
        level = np.array([l for l, _ in lv], dtype=np.int64)
        coords = np.array([c for _, c in lv], dtype=np.int64).reshape(-1, 3)
        return level, coords

    def neighbour_offsets(self):
        rng = [(-1, 0, 1) if d < self.dim else (0,) for d in range(3)]
        return [o for o in itertools.product(*rng) if any(o)]

    # ------------------------------------------------------------- mutations
    def _refine_cell(self, level: int, c: Cell) -> None:
        assert self.is_leaf(level, c)
        if level + 1 == len(self.cells):
            self.cells.append(set())
            self.refined.append(set())
        self.refined[level].add(c)
        rng = [(0, 1) if d < self.dim else (0,) for d in range(3)]
        for b in itertools.product(*rng):
            self.cells[level + 1].add(tuple(2 * c[d] + b[d] for d in range(3)))

    def _covering_leaf(self, level: int, c: Cell) -> Tuple[int, Cell]:
        """The leaf that contains the (non-existing) lattice cell (level, c)."""
        l, cc = level, c
        while not self.exists(l, cc):
            l, cc = l - 1, tuple(x >> 1 if d < self.dim else 0 for d, x in enumerate(cc))
        assert self.is_leaf(l, cc)
        return l, cc

    def close(self) -> None:
        offsets = self.neighbour_offsets()
        changed = True
        while changed:
            changed = False
            for l in range(1, len(self.cells)):
                for c in list(self.refined[l]):
                    for o in offsets:
                        n = tuple(c[d] + o[d] for d in range(3))
                        if self.inside(l, n) and not self.exists(l, n):
                            lc, cc = self._covering_leaf(l, n)
                            self._refine_cell(lc, cc)
                            changed = True

    def refine(self, flags) -> None:
        """Refine the flagged leaves (flags follow ``leaves()`` order), then close."""
        lv = self.leaves()
        flags = np.asarray(flags, dtype=bool)
        assert len(flags) == len(lv)
        for (l, c), f in zip(lv, flags):
            if f:
                self._refine_cell(l, c)
        self.close()

    def apply_rounds(self, rounds) -> None:
        for fn in rounds:
            level, coords = self.leaf_arrays()
            self.refine(fn(self.cm, level, coords, int(level.max())))

    # ------------------------------------------------------------ invariants
    def is_balanced(self) -> bool:
        """True iff any two leaves whose closures touch differ by at most one level."""
        for l in range(1, len(self.cells)):
            for c in self.refined[l]:
                for o in self.neighbour_offsets():
                    n = tuple(c[d] + o[d] for d in range(3))
                    if self.inside(l, n) and not self.exists(l, n):
                        return False
        return True


def build_forest(coarse, rounds) -> Forest:
    f = Forest(coarse)
    f.apply_rounds(rounds)
    return f
