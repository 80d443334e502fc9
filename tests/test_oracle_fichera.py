"""The oracle on the Fichera corner of Sec. 4.3, Omega = [-1, 1]^3 minus
[0, 1]^3 with epsilon = 100 where min(x, y, z) <= -1/2 (else 1), u = 0 on the
whole boundary, f = 1, Q2: pinned against closed forms of the domain and of
the textbook 1-D Q2 element matrices, and against a dense direct solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem, gmg as O
from oracle.mesh import build_forest
from paper_1904_03317_gb300 import inputs

# 1-D Q2 element matrices on [0, 1] (textbook): stiffness and mass
K1 = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / 3.0
M1 = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) / 30.0


def _disc(adaptive, glob=0):
    w = inputs.fichera(adaptive, glob)
    f = build_forest(w.coarse, w.rounds)
    return w, f, fem.Discretization(f, w.degree, w.coeff)


def test_domain_and_boundary_in_closed_form():
    """Nodes on the boundary are those on the brick's faces and those on the
    three re-entrant faces (all coordinates >= 0 with the smallest 0); the
    hole holds no node; the leaves tile a volume of 7."""
    w, f, d = _disc(2)
    keys = np.unique(d.all_keys)
    p = d.node_positions(keys)
    on_brick = np.any(np.abs(np.abs(p) - 1.0) < 1e-12, axis=1)
    on_reentrant = np.all(p >= -1e-12, axis=1) & (np.abs(p.min(axis=1)) < 1e-12)
    assert np.array_equal(d.is_dirichlet(keys), on_brick | on_reentrant)
    assert not np.any(np.all(p > 1e-12, axis=1))  # nothing strictly inside the hole
    lv, co = f.leaf_arrays()
    blo, bhi = w.coarse.boxes(lv, co)
    assert abs(np.prod(bhi - blo, axis=1).sum() - 7.0) < 1e-12
    assert f.is_balanced()
    # the unknowns of the 56 coarse cells: the 7^3 interior lattice nodes of
    # the brick minus the 4^3 in [0, 1)^3
    H0 = O.build_hierarchy(_disc(0)[2], 1)
    assert len(H0.levels[0].keys) == 7 ** 3 - 4 ** 3 == H0.disc.n


def _node_index(d, keys, pos):
    k = d.node_positions(keys)
    i = np.nonzero(np.all(np.abs(k - np.asarray(pos)) < 1e-12, axis=1))[0]
    assert len(i) == 1
    return int(i[0])


def test_coarse_matrix_entries_from_the_element_matrices():
    """A_0 on the 56 coarse cells (side h = 1/2): the diagonal at a vertex
    node is sum_cells a_c h 3 K1[0,0] M1[0,0]^2, an edge entry between a
    vertex and its neighbouring mid-edge node along x is sum_cells a_c h
    (K1[0,1] M1[0,0]^2 + 2 M1[0,1] K1[0,0] M1[0,0]), each sum over the cells
    holding both nodes with their coefficients from min(centre) < -1/2."""
    H = O.build_hierarchy(_disc(0)[2], 1)
    lev = H.levels[0]
    A = lev.A.toarray()
    d = H.disc
    h = 0.5
    vertex = h * 3 * K1[0, 0] * M1[0, 0] ** 2
    edge = h * (K1[0, 1] * M1[0, 0] ** 2 + 2 * M1[0, 1] * K1[0, 0] * M1[0, 0])
    # (-1/2, -1/2, -1/2): 8 cells, 7 of them with an index-0 coordinate (a = 100)
    i = _node_index(d, lev.keys, (-0.5, -0.5, -0.5))
    assert abs(A[i, i] - (7 * 100 + 1) * vertex) < 1e-12 * A[i, i]
    # (0, 0, -1/2) below the re-entrant corner: 4 cells with z in [-1, -1/2]
    # (a = 100), 4 with z in [-1/2, 0] (a = 1); none of them in the hole
    j = _node_index(d, lev.keys, (0.0, 0.0, -0.5))
    assert abs(A[j, j] - (4 * 100 + 4 * 1) * vertex) < 1e-12 * A[j, j]
    # (-1/2, -1/2, -1/2) -- (-1/4, -1/2, -1/2): the 4 cells with x in [-1/2, 0]
    # around the x edge, 3 of them with a = 100
    m = _node_index(d, lev.keys, (-0.25, -0.5, -0.5))
    assert abs(A[i, m] - (3 * 100 + 1) * edge) < 1e-12 * abs(A[i, m])
    # a node next to the hole couples to no node of the hole's faces: those
    # are Dirichlet and not unknowns
    assert np.allclose(A, A.T, rtol=0, atol=1e-13 * np.abs(A).max())


def test_leaf_operator_symmetric_positive_definite():
    w, f, d = _disc(3)
    A = d.A
    assert abs(A - A.T).max() <= 1e-13 * abs(A).max()
    lam = spla.eigsh(A, k=1, which="SA", return_eigenvectors=False)[0]
    assert lam > 0


def test_mf_setting_matches_a_dense_direct_solve():
    """The paper's "MF" setting (one undamped Jacobi step, unpreconditioned CG
    coarse solver) as the preconditioner of CG to 1e-10 gives the direct
    solution of the adaptive Fichera problem with f = 1, within the
    tolerance times the condition number."""
    w, f, d = _disc(3)
    H = O.build_hierarchy(d, w.cheb_degree)
    H.smoother = w.smoother
    O.setup_coarse(H, w.coarse_solver)
    b = d.rhs_one()
    res = O.solve(H, b, w.tol)
    assert res.converged
    x = np.linalg.solve(d.A.toarray(), b)
    ev = np.linalg.eigvalsh(d.A.toarray())
    kappa = ev[-1] / ev[0]
    assert np.linalg.norm(res.x - x) <= 10 * kappa * w.tol * np.linalg.norm(x)
    assert np.linalg.norm(b - d.A @ res.x) <= w.tol * np.linalg.norm(b) * (1 + 1e-9)
    # f = 1 > 0 and a maximum principle: the discrete solution is positive
    # at the unknowns far from the boundary and its integral is positive
    assert x.max() > 0 and b @ x > 0


def test_rhs_one_integrates_the_basis():
    """b = C^T int phi_i: summed over the unknowns and the Dirichlet nodes
    the nodal integrals of the basis give the domain's volume; the unknowns'
    share is the integral of the interpolant of the indicator of the
    interior nodes, below 7."""
    w, f, d = _disc(1)
    b = d.rhs_one()
    assert 0 < b.sum() < 7.0 and np.all(np.isfinite(b))
