"""Oracle finite-element layer (test infrastructure only).

Continuous Q_k Lagrange elements on axis-aligned boxes (Sec. 2.1).  The paper
only says the shape functions come from "interpolation points"; the reading
used here is Gauss-Lobatto points, which are equidistant for k <= 2 -- the
degrees this oracle supports -- so every node of every level sits on one
integer lattice and node identity is exact integer equality.

Node key: the node's coordinates on the node lattice of the finest level Lf
(spacing h_Lf / k), packed as (z << 42) | (y << 21) | x.  Sorting by key is
lexicographic (z, y, x) order, the canonical order of unknowns.

Everything is assembled explicitly:

* the element matrix  a_K * sum_q w_q grad phi_i . grad phi_j |J|  by
  Gauss-Legendre quadrature with (k+1)^d points (exact on boxes);
* the leaf-mesh operator A = C^T A_full C with the hanging-node constraint
  matrix C (Sec. 1, "elimination of hanging nodes");
* per level l the matrix of the level-l cells on the level's non-Dirichlet
  nodes, split into S (strictly on level l) and I (on the refinement edge,
  Sec. 2.3, Fig. 1);
* the prolongation P_{l-1} as the embedding V_{l-1} -> V_l (Sec. 2.2) and
  the restriction R = P^T.
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Tuple

import numpy as np
import scipy.sparse as sp

KEY_BITS = 21
_KMASK = (1 << KEY_BITS) - 1


# ----------------------------------------------------------------- 1-D basis
def gauss_lobatto_points(k: int) -> np.ndarray:
    """k+1 Gauss-Lobatto points on [0, 1]: the two ends plus the roots of P_k'."""
    if k == 1:
        return np.array([0.0, 1.0])
    dP = np.polynomial.legendre.Legendre.basis(k).deriv()
    inner = np.sort(np.real(dP.roots()))
    return np.concatenate([[0.0], 0.5 * (inner + 1.0), [1.0]])


def lagrange_values(nodes: np.ndarray, x) -> np.ndarray:
    """phi_j(x_q) for the Lagrange basis on ``nodes``; shape (len(x), len(nodes))."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    out = np.ones((len(x), n))
    for j in range(n):
        for m in range(n):
            if m != j:
                out[:, j] *= (x - nodes[m]) / (nodes[j] - nodes[m])
    return out


def lagrange_derivatives(nodes: np.ndarray, x) -> np.ndarray:
    """phi_j'(x_q) by the product rule; shape (len(x), len(nodes))."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    out = np.zeros((len(x), n))
    for j in range(n):
        for i in range(n):
            if i == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[i]))
            for m in range(n):
                if m != j and m != i:
                    term *= (x - nodes[m]) / (nodes[j] - nodes[m])
            out[:, j] += term
    return out


def gauss_legendre(n: int) -> Tuple[np.ndarray, np.ndarray]:
    """n-point Gauss-Legendre rule on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def local_index_tuples(dim: int, k: int) -> np.ndarray:
    """Local node multi-indices (ix, iy, iz) of a cell, x fastest; shape (nloc, 3)."""
    rng = [range(k + 1) if d < dim else range(1) for d in range(3)]
    return np.array([(ix, iy, iz) for iz in rng[2] for iy in rng[1] for ix in rng[0]],
                    dtype=np.int64)


def _tensor_points(dim: int, n: int):
    return list(itertools.product(range(n), repeat=dim))


def element_stiffness(dim: int, k: int, h) -> np.ndarray:
    """int_K grad phi_i . grad phi_j on a box with sides h (coefficient 1).

    Plain definition: phi_i(x) = prod_e l_{i_e}((x_e - x0_e) / h_e), integrated
    with the tensor Gauss-Legendre rule of k+1 points per direction, which is
    exact for these polynomial integrands on a box.
    """
    nodes = gauss_lobatto_points(k)
    xq, wq = gauss_legendre(k + 1)
    V = lagrange_values(nodes, xq)  # (q, j)
    Dv = lagrange_derivatives(nodes, xq)
    loc = local_index_tuples(dim, k)
    nloc = len(loc)
    A = np.zeros((nloc, nloc))
    jac = float(np.prod(h[:dim]))
    for q in _tensor_points(dim, len(xq)):
        w = float(np.prod([wq[q[e]] for e in range(dim)])) * jac
        grads = np.zeros((nloc, dim))
        for e in range(dim):
            g = Dv[q[e], loc[:, e]] / h[e]
            for f in range(dim):
                if f != e:
                    g = g * V[q[f], loc[:, f]]
            grads[:, e] = g
        A += w * grads @ grads.T
    return A


def sine_rhs_function(dim: int):
    """f = d pi^2 prod sin(pi x_i): then u = prod sin(pi x_i) solves -lap u = f."""

    def f(x):  # x: (..., dim)
        return dim * np.pi ** 2 * np.prod(np.sin(np.pi * x[..., :dim]), axis=-1)

    return f


def sine_solution(dim: int):
    def u(x):
        return np.prod(np.sin(np.pi * np.asarray(x)[..., :dim]), axis=-1)

    return u


# --------------------------------------------------------------- node keys
def pack_keys(q: np.ndarray) -> np.ndarray:
    """Pack node-lattice coordinates (..., 3) into int64 keys."""
    q = np.asarray(q, dtype=np.int64)
    return (q[..., 2] << (2 * KEY_BITS)) | (q[..., 1] << KEY_BITS) | q[..., 0]


def unpack_keys(keys) -> np.ndarray:
    keys = np.asarray(keys, dtype=np.int64)
    return np.stack([keys & _KMASK, (keys >> KEY_BITS) & _KMASK, keys >> (2 * KEY_BITS)], axis=-1)


def lookup(sorted_keys: np.ndarray, query: np.ndarray) -> np.ndarray:
    """Index of each query key in ``sorted_keys``, -1 where absent."""
    query = np.asarray(query, dtype=np.int64)
    if len(sorted_keys) == 0:
        return np.full(query.shape, -1, dtype=np.int64)
    pos = np.searchsorted(sorted_keys, query)
    pos_c = np.minimum(pos, len(sorted_keys) - 1)
    return np.where(sorted_keys[pos_c] == query, pos_c, -1)


class Discretization:
    """All oracle matrices for one forest, degree and coefficient field."""

    def __init__(self, forest, k: int, coarse_coeff=None):
        assert k in (1, 2), "the oracle supports Q1 and Q2 (equidistant Gauss-Lobatto points)"
        assert forest.is_balanced()
        self.forest = forest
        self.k = k
        self.dim = forest.dim
        self.L = forest.num_levels() - 1  # finest level that has cells
        self.n0 = forest.n0
        cm = forest.cm
        self.lo = np.array([cm.lo[d] if d < self.dim else 0.0 for d in range(3)])
        self.hi = np.array([cm.hi[d] if d < self.dim else 1.0 for d in range(3)])
        ncoarse = self.n0[0] * self.n0[1] * self.n0[2]
        self.coarse_coeff = (np.ones(ncoarse) if coarse_coeff is None
                             else np.asarray(coarse_coeff, dtype=np.float64))
        self.loc = local_index_tuples(self.dim, k)
        self.nloc = len(self.loc)
        self._ref_stiff: Dict[int, np.ndarray] = {}
        self._build_active()

    # ------------------------------------------------------------ geometry
    def cell_h(self, level: int) -> np.ndarray:
        return (self.hi - self.lo) / (np.array(self.n0, dtype=np.float64) * (1 << level))

    def stiffness(self, level: int) -> np.ndarray:
        if level not in self._ref_stiff:
            self._ref_stiff[level] = element_stiffness(self.dim, self.k, self.cell_h(level))
        return self._ref_stiff[level]

    def coefficients(self, level: int, coords: np.ndarray) -> np.ndarray:
        """a_K per cell, inherited from the coarse cell that contains K."""
        cc = np.asarray(coords, dtype=np.int64) >> level
        return self.coarse_coeff[cc[:, 0] + self.n0[0] * (cc[:, 1] + self.n0[1] * cc[:, 2])]

    def node_scale(self, level: int) -> int:
        return 1 << (self.L - level)

    def cell_node_keys(self, level: int, coords: np.ndarray) -> np.ndarray:
        """Keys of the nodes of the given level-l cells; shape (ncells, nloc)."""
        coords = np.asarray(coords, dtype=np.int64).reshape(-1, 3)
        q = (coords[:, None, :] * self.k + self.loc[None, :, :]) * self.node_scale(level)
        q[:, :, self.dim:] = 0
        return pack_keys(q)

    def node_extent(self) -> np.ndarray:
        """Largest node-lattice coordinate per dimension (the far boundary)."""
        return np.array([self.n0[d] * self.k * (1 << self.L) if d < self.dim else 0
                         for d in range(3)], dtype=np.int64)

    def is_dirichlet(self, keys) -> np.ndarray:
        """Nodes on the boundary of the domain (the union of the present
        coarse cells): some coarse cell whose closure contains the node lies
        outside the brick or is absent."""
        q = unpack_keys(keys)
        s0 = self.k << self.L  # node-lattice units per coarse cell
        f = self.forest
        sides = []
        for d in range(3):
            if d >= self.dim:
                sides.append([np.zeros(q.shape[:-1], dtype=np.int64)])
                continue
            up = q[..., d] // s0
            low = np.where(q[..., d] % s0 == 0, up - 1, up)
            sides.append([low, up])
        on = np.zeros(q.shape[:-1], dtype=bool)
        for cz in sides[2]:
            for cy in sides[1]:
                for cx in sides[0]:
                    c = (cx, cy, cz)
                    inb = np.ones(q.shape[:-1], dtype=bool)
                    for d in range(self.dim):
                        inb &= (c[d] >= 0) & (c[d] < self.n0[d])
                    ok = inb.copy()
                    if f.present is not None:
                        pres = np.asarray(f.present, dtype=bool)
                        idx = np.where(inb, np.clip(cx, 0, self.n0[0] - 1) + self.n0[0] * (
                            np.clip(cy, 0, self.n0[1] - 1) + self.n0[1] * np.clip(cz, 0, self.n0[2] - 1)), 0)
                        ok &= pres[idx]
                    on |= ~ok
        return on

    def node_positions(self, keys) -> np.ndarray:
        q = unpack_keys(keys).astype(np.float64)
        return self.lo + q * (self.cell_h(self.L) / self.k)

    def cells_touching(self, level: int, key: int):
        """Level-l lattice cells (inside the domain) whose closure contains the node."""
        q = unpack_keys(key)
        s = self.node_scale(level) * self.k  # node-lattice units per level-l cell
        cand = []
        for d in range(3):
            if d >= self.dim:
                cand.append([0])
                continue
            c = int(q[d]) // s
            cand.append([c - 1, c] if int(q[d]) % s == 0 else [c])
        return [c for c in itertools.product(*cand) if self.forest.inside(level, c)]

    def is_node_of(self, level: int, c, key: int) -> bool:
        q = unpack_keys(key)
        s = self.node_scale(level)
        for d in range(self.dim):
            r = int(q[d]) - c[d] * self.k * s
            if r < 0 or r > self.k * s or r % s != 0:
                return False
        return True

    def basis_at(self, level: int, c, key: int) -> List[Tuple[int, float]]:
        """(node key, phi_j^K(x)) for the nonzero shape functions of cell K at node x."""
        q = unpack_keys(key)
        s = self.node_scale(level)
        nodes = gauss_lobatto_points(self.k)
        vals = []
        for d in range(3):
            if d < self.dim:
                t = (int(q[d]) - c[d] * self.k * s) / (self.k * s)
                vals.append(lagrange_values(nodes, [t])[0])
            else:
                vals.append(np.ones(1))
        keys = self.cell_node_keys(level, np.array([c]))[0]
        out = []
        for j in range(self.nloc):
            w = 1.0
            for d in range(self.dim):
                w *= vals[d][self.loc[j, d]]
            if abs(w) > 1e-14:
                out.append((int(keys[j]), w))
        return out

    # --------------------------------------------------------- assembly
    def _assemble(self, groups, index_keys: np.ndarray) -> sp.csr_matrix:
        """Sum of a_K * stiffness over the given cells, on the nodes ``index_keys``.

        ``groups`` is a list of (level, coords array); nodes not in
        ``index_keys`` (Dirichlet nodes) are dropped.
        """
        n = len(index_keys)
        rows, cols, vals = [], [], []
        for level, coords in groups:
            if len(coords) == 0:
                continue
            ids = lookup(index_keys, self.cell_node_keys(level, coords))
            Ke = self.stiffness(level)
            a = self.coefficients(level, coords)
            r = np.broadcast_to(ids[:, :, None], (len(coords), self.nloc, self.nloc))
            c = np.broadcast_to(ids[:, None, :], (len(coords), self.nloc, self.nloc))
            v = a[:, None, None] * Ke[None, :, :]
            m = (r >= 0) & (c >= 0)
            rows.append(r[m]); cols.append(c[m]); vals.append(v[m])
        if not rows:
            return sp.csr_matrix((n, n))
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(n, n))

    # --------------------------------------------------------- leaf mesh
    def _build_active(self) -> None:
        f = self.forest
        self.leaves = f.leaves()
        self.leaf_groups = []
        for l in range(self.L + 1):
            cs = np.array(sorted(f.cells[l] - f.refined[l]), dtype=np.int64).reshape(-1, 3)
            self.leaf_groups.append((l, cs))
        # every node of every leaf, with the coarsest level of a leaf that has it as a node
        all_k, all_l = [], []
        for l, cs in self.leaf_groups:
            if len(cs):
                kk = self.cell_node_keys(l, cs).ravel()
                all_k.append(kk); all_l.append(np.full(len(kk), l))
        all_k = np.concatenate(all_k); all_l = np.concatenate(all_l)
        order = np.lexsort((all_l, all_k))
        all_k, all_l = all_k[order], all_l[order]
        first = np.concatenate([[True], all_k[1:] != all_k[:-1]])
        self.all_keys = all_k[first]
        lmin = all_l[first]
        # Hanging node (Sec. 1): lies in the closure of a coarser leaf without being
        # one of its nodes.  Under the 2:1 closure that leaf is one level coarser
        # than the coarsest leaf having the node.  Constraint row = that leaf's
        # shape functions evaluated at the node.
        self.hanging: Dict[int, List[Tuple[int, float]]] = {}
        for key, lm in zip(self.all_keys.tolist(), lmin.tolist()):
            if lm == 0:
                continue
            for c in self.cells_touching(lm - 1, key):
                if f.is_leaf(lm - 1, c) and not self.is_node_of(lm - 1, c, key):
                    self.hanging[key] = self.basis_at(lm - 1, c, key)
        for key, row in self.hanging.items():
            for m, _ in row:
                assert m not in self.hanging, "constraint chain"
        dir_mask = self.is_dirichlet(self.all_keys)
        hang_mask = np.isin(self.all_keys, np.array(list(self.hanging), dtype=np.int64))
        unk = ~dir_mask & ~hang_mask
        self.unknown_keys = self.all_keys[unk]
        self.home_level = lmin[unk]  # coarsest leaf level containing the unknown
        self.n = len(self.unknown_keys)
        # constraint matrix C: values on all leaf nodes <- unknowns
        nall = len(self.all_keys)
        rows = list(np.nonzero(unk)[0]); cols = list(range(self.n)); vals = [1.0] * self.n
        for key, row in self.hanging.items():
            r = int(lookup(self.all_keys, np.array([key]))[0])
            for m, w in row:
                cm = int(lookup(self.unknown_keys, np.array([m]))[0])
                if cm >= 0:  # Dirichlet masters carry the value 0
                    rows.append(r); cols.append(cm); vals.append(w)
        self.C = sp.csr_matrix((vals, (rows, cols)), shape=(nall, self.n))
        self.A_full = self._assemble(self.leaf_groups, self.all_keys)
        self.A = (self.C.T @ self.A_full @ self.C).tocsr()

    def rhs_sine(self) -> np.ndarray:
        """b = C^T b_full, b_full_i = sum_K int_K f phi_i with (k+1)^d Gauss-Legendre
        points per cell (the paper does not fix the rule; this is the reading)."""
        return self._rhs(sine_rhs_function(self.dim))

    def rhs_one(self) -> np.ndarray:
        """The same for f = 1 (the Laplace example of Sec. 4.3)."""
        return self._rhs(lambda x: np.ones(len(x)))

    def _rhs(self, f) -> np.ndarray:
        nodes = gauss_lobatto_points(self.k)
        xq, wq = gauss_legendre(self.k + 1)
        V = lagrange_values(nodes, xq)
        bfull = np.zeros(len(self.all_keys))
        for l, cs in self.leaf_groups:
            if len(cs) == 0:
                continue
            h = self.cell_h(l)
            blo = self.lo[None, :] + cs * h[None, :]
            ids = lookup(self.all_keys, self.cell_node_keys(l, cs))
            be = np.zeros((len(cs), self.nloc))
            for q in _tensor_points(self.dim, len(xq)):
                x = blo.copy()
                for e in range(self.dim):
                    x[:, e] += h[e] * xq[q[e]]
                w = float(np.prod([wq[q[e]] for e in range(self.dim)])) * float(np.prod(h[: self.dim]))
                phi = np.ones(self.nloc)
                for e in range(self.dim):
                    phi = phi * V[q[e], self.loc[:, e]]
                be += w * f(x)[:, None] * phi[None, :]
            np.add.at(bfull, ids.ravel(), be.ravel())
        return self.C.T @ bfull

    def l2_error(self, u: np.ndarray, exact) -> float:
        """|| u_h - u ||_L2 over the leaves with (k+2)^d Gauss points per cell."""
        nodes = gauss_lobatto_points(self.k)
        xq, wq = gauss_legendre(self.k + 2)
        V = lagrange_values(nodes, xq)
        full = self.C @ u
        err2 = 0.0
        for l, cs in self.leaf_groups:
            if len(cs) == 0:
                continue
            h = self.cell_h(l)
            blo = self.lo[None, :] + cs * h[None, :]
            vals = full[lookup(self.all_keys, self.cell_node_keys(l, cs))]
            for q in _tensor_points(self.dim, len(xq)):
                x = blo.copy()
                for e in range(self.dim):
                    x[:, e] += h[e] * xq[q[e]]
                w = float(np.prod([wq[q[e]] for e in range(self.dim)])) * float(np.prod(h[: self.dim]))
                phi = np.ones(self.nloc)
                for e in range(self.dim):
                    phi = phi * V[q[e], self.loc[:, e]]
                err2 += w * float(np.sum((vals @ phi - exact(x)) ** 2))
        return float(np.sqrt(err2))

    # ------------------------------------------------------------ levels
    def level_space(self, level: int):
        """Level-l space on the cells of level l (Sec. 2.3).

        Returns (keys, is_interface, A_l): the non-Dirichlet nodes of the
        level-l cells sorted canonically, the I flag per node (some level-l
        lattice cell inside the domain whose closure contains the node does
        not exist), and the matrix assembled over the level-l cells only.
        """
        f = self.forest
        cs = np.array(sorted(f.cells[level]), dtype=np.int64).reshape(-1, 3)
        keys = np.unique(self.cell_node_keys(level, cs))
        keys = keys[~self.is_dirichlet(keys)]
        iface = np.array([any(not f.exists(level, c) for c in self.cells_touching(level, int(key)))
                          for key in keys], dtype=bool)
        A = self._assemble([(level, cs)], keys)
        return keys, iface, A

    def prolongation(self, level: int, keys_fine, keys_coarse) -> sp.csr_matrix:
        """P_{l-1}: level l-1 nodes -> level l nodes, the embedding v -> v (Sec. 2.2).

        Row of fine node x: phi_j^{K'}(x) over the nodes of the parent K' of a
        level-l cell containing x.  Every such cell gives the same row
        (continuity of the coarse function); this is asserted.
        """
        f = self.forest
        keys_fine = np.asarray(keys_fine, dtype=np.int64)
        keys_coarse = np.asarray(keys_coarse, dtype=np.int64)
        cs = np.array(sorted(f.cells[level]), dtype=np.int64).reshape(-1, 3)
        parents = cs >> 1
        parents[:, self.dim:] = 0
        fine_keys = self.cell_node_keys(level, cs)            # (ncell, nloc)
        coarse_keys = self.cell_node_keys(level - 1, parents)  # (ncell, nloc)
        # phi_j^{K'} at the child's nodes: the child's node sits at parent-local
        # coordinate (child bit * k + i) / (2k) along each direction.
        nodes = gauss_lobatto_points(self.k)
        E = lagrange_values(nodes, np.arange(2 * self.k + 1) / (2.0 * self.k))  # (2k+1, k+1)
        bits = cs & 1
        W = np.ones((len(cs), self.nloc, self.nloc))
        for d in range(self.dim):
            r = bits[:, d][:, None] * self.k + self.loc[None, :, d]   # (ncell, nloc) fine pos
            W *= E[r[:, :, None], self.loc[None, None, :, d]]
        rows = lookup(keys_fine, fine_keys)[:, :, None].repeat(self.nloc, axis=2)
        cols = lookup(keys_coarse, coarse_keys)[:, None, :].repeat(self.nloc, axis=1)
        cdir = self.is_dirichlet(coarse_keys)[:, None, :].repeat(self.nloc, axis=1)
        keep = (rows >= 0) & (np.abs(W) > 1e-14) & ~cdir
        assert np.all(cols[keep] >= 0)
        r, c, w = rows[keep], cols[keep], W[keep]
        # a fine node shared by several cells appears several times: keep one copy
        # and check that all copies agree
        pair = r.astype(np.int64) * (len(keys_coarse) + 1) + c
        order = np.argsort(pair, kind="stable")
        pair, r, c, w = pair[order], r[order], c[order], w[order]
        first = np.concatenate([[True], pair[1:] != pair[:-1]])
        grp = np.cumsum(first) - 1
        assert np.all(np.abs(w - w[first][grp]) < 1e-13)
        # every fine node must get the same set of columns from every cell: the
        # number of copies of each (row, col) pair equals the number of cells
        # containing the row's node
        copies = np.bincount(grp)
        cells_per_row = np.bincount(lookup(keys_fine, fine_keys).ravel()[
            lookup(keys_fine, fine_keys).ravel() >= 0], minlength=len(keys_fine))
        assert np.all(copies == cells_per_row[r[first]])
        return sp.csr_matrix((w[first], (r[first], c[first])),
                             shape=(len(keys_fine), len(keys_coarse)))
