"""Pins of the oracle's smoother, eigenvalue estimate, V-cycle and CG (CPU only)."""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, gmg
from oracle.mesh import build_forest
from paper_1904_03317_gb300 import inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_facts.json")))


def test_chebyshev_error_polynomial_closed_form():
    """On A = diag(lambda) with D = I, m Chebyshev updates from x0 multiply each
    error component by T_m((theta - lambda)/delta) / T_m(theta/delta)."""
    rng = np.random.default_rng(1)
    lam = np.linspace(0.02, 1.3, 40)
    A = sp.diags(lam)
    xstar = rng.standard_normal(40)
    b = A @ xstar
    x0 = rng.standard_normal(40)
    lam_max = 1.1
    theta, delta, _ = gmg.chebyshev_coefficients(lam_max, *GOLDEN["cheb_eig_range"]["value"])
    for m in (1, 2, 4, 5):
        x = gmg.chebyshev(A, np.ones(40), x0, b, lam_max, m)
        Tm = np.zeros(m + 1); Tm[m] = 1.0
        factor = (np.polynomial.chebyshev.chebval((theta - lam) / delta, Tm)
                  / np.polynomial.chebyshev.chebval(theta / delta, Tm))
        np.testing.assert_allclose(x - xstar, factor * (x0 - xstar), rtol=1e-10, atol=1e-12)
    # from zero: same polynomial
    x = gmg.chebyshev(A, np.ones(40), np.zeros(40), b, lam_max, 3, x0_is_zero=True)
    T3 = np.array([0, 0, 0, 1.0])
    factor = (np.polynomial.chebyshev.chebval((theta - lam) / delta, T3)
              / np.polynomial.chebyshev.chebval(theta / delta, T3))
    np.testing.assert_allclose(x - xstar, factor * (-xstar), rtol=1e-10, atol=1e-12)


def test_eigen_start_vector_is_papers_pattern():
    v = gmg.eigen_start_vector(30)
    pat = GOLDEN["eig_start_pattern"]["value"]
    np.testing.assert_array_equal(v[:12], pat)
    np.testing.assert_array_equal(v[12:24], pat)
    assert abs(v[:24].sum()) == 0.0


def test_lanczos_exact_for_few_distinct_eigenvalues():
    """With fewer distinct eigenvalues than CG steps the Krylov space is exhausted
    and the largest Ritz value is the largest eigenvalue."""
    lam = np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 7.0, 8.0])
    est = gmg.estimate_lambda_max(sp.diags(lam), np.ones(8), gmg.eigen_start_vector(8), 10)
    assert est == pytest.approx(8.0, rel=1e-10)


def _hier(dim, k, g, rounds, cheb=4, coeff=None, eig_iters=10):
    if dim == 2:
        cm = inputs.CoarseMesh(2, (4, 4, 1), (0, 0, 0), (1, 1, 1))
        rr = [inputs.round_uniform()] * g + [inputs.round_sphere_surface((0.5, 0.5), 0.3)] * rounds
    else:
        cm = inputs.CoarseMesh(3, (2, 2, 2), (0, 0, 0), (1, 1, 1))
        rr = [inputs.round_uniform()] * g + [inputs.round_sphere_surface((0.5, 0.5, 0.5), 0.25)] * rounds
    c = inputs.checkerboard_coefficients(cm) if coeff == "checker" else None
    d = fem.Discretization(build_forest(cm, rr), k, c)
    return gmg.build_hierarchy(d, cheb, eig_iters=eig_iters)


def test_lanczos_estimate_bounds_on_level_matrices():
    H = _hier(2, 2, 1, 2)
    for lev in H.levels[1:]:
        Ad = lev.A_S.toarray()
        Dm = np.diag(np.sqrt(lev.dinv))
        lmax = np.linalg.eigvalsh(Dm @ Ad @ Dm)[-1]
        assert lev.lam <= lmax * (1 + 1e-12)
        assert lev.lam >= 0.85 * lmax


@pytest.mark.parametrize("dim,k,coeff", [(2, 1, None), (2, 2, "checker"), (3, 2, None)])
def test_vcycle_symmetric_positive(dim, k, coeff):
    H = _hier(dim, k, 1, 2, coeff=coeff)
    n = H.disc.n
    rng = np.random.default_rng(2)
    r1, r2 = rng.standard_normal(n), rng.standard_normal(n)
    z1, z2 = gmg.vcycle(H, r1), gmg.vcycle(H, r2)
    assert abs(r2 @ z1 - r1 @ z2) <= 1e-12 * abs(r1 @ z1)
    assert r1 @ z1 > 0 and r2 @ z2 > 0


def test_vcycle_is_exact_solve_without_refinement():
    cm = inputs.CoarseMesh(2, (5, 3, 1), (0, 0, 0), (1.0, 0.6, 1))
    d = fem.Discretization(build_forest(cm, []), 2)
    H = gmg.build_hierarchy(d, 3)
    r = np.random.default_rng(3).standard_normal(d.n)
    np.testing.assert_allclose(d.A @ gmg.vcycle(H, r), r, rtol=1e-12, atol=1e-12)


def test_vcycle_contracts_error():
    """x <- x + B(b - A x) is a contraction: one V-cycle reduces the A-norm error."""
    H = _hier(2, 2, 1, 3)
    A = H.disc.A
    rng = np.random.default_rng(4)
    e = rng.standard_normal(H.disc.n)
    for _ in range(3):
        e_new = e - gmg.vcycle(H, A @ e)
        ratio = np.sqrt((e_new @ (A @ e_new)) / (e @ (A @ e)))
        assert ratio < 0.2
        e = e_new


class _CountingMatrix:
    def __init__(self, M, counter):
        self.M, self.c = M, counter
        self.shape = M.shape

    def __matmul__(self, x):
        self.c[0] += 1
        return self.M @ x


def test_matvec_count_per_level_matches_paper():
    """At Chebyshev degree 5 each level does 8 smoother products and 2 residual
    products with A^S (Sec. 4.1: 12 per level = 8 smoother + 2 residual + 2 transfer)."""
    m = GOLDEN["cheb_degree_superMUC"]["value"]
    H = _hier(2, 1, 1, 2, cheb=m)
    counters = []
    for lev in H.levels[1:]:
        c = [0]
        lev.A_S = _CountingMatrix(lev.A_S, c)
        counters.append(c)
    gmg.vcycle(H, np.ones(H.disc.n))
    want = GOLDEN["smoother_matvecs_per_level_deg5"]["value"] + GOLDEN["residual_matvecs_per_level"]["value"]
    assert [c[0] for c in counters] == [want] * len(counters)


@pytest.mark.parametrize("dim,k,g,rounds", [
    (2, 1, 3, 0), (2, 1, 2, 3), (2, 2, 2, 0), (2, 2, 1, 3), (3, 2, 1, 0), (3, 2, 1, 2),
])
def test_cg_iterations_in_papers_band(dim, k, g, rounds):
    """Chebyshev degree 5, relative tolerance 1e-10: the paper reports 7-11 CG
    iterations for uniform and adaptive meshes in 2D and 3D (Sec. 4.1)."""
    band = GOLDEN["cg_iterations_band"]
    H = _hier(dim, k, g, rounds, cheb=GOLDEN["cheb_degree_superMUC"]["value"])
    b = H.disc.rhs_sine()
    res = gmg.solve(H, b, band["tol"])
    assert res.converged
    assert res.iterations <= band["value"][1]
    assert res.iterations >= 4


def test_iterations_mesh_independent():
    its = []
    for g in (1, 2, 3):
        H = _hier(2, 2, g, 2, cheb=4)
        its.append(gmg.solve(H, H.disc.rhs_sine(), 1e-8).iterations)
    assert max(its) - min(its) <= 1, its


def test_gmg_cg_matches_dense_direct_solve():
    """The literal reading of the 2D circle problem (4x4 quads, 3 adaptive rounds,
    about 100-300 unknowns): GMG-preconditioned CG agrees with a dense solve."""
    w = inputs.poisson2d_circle(0, 3)
    d = fem.Discretization(build_forest(w.coarse, w.rounds), 1)
    assert 100 <= d.n <= 400
    H = gmg.build_hierarchy(d, 2)
    b = d.rhs_sine()
    res = gmg.solve(H, b, 1e-13)
    x = np.linalg.solve(d.A.toarray(), b)
    np.testing.assert_allclose(res.x, x, rtol=1e-11, atol=1e-13 * np.abs(x).max())
