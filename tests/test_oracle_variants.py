"""Oracle solver variants of the paper: the Chebyshev coarse solver with an
a-priori degree (Sec. 4.1), the unpreconditioned CG coarse solver and the
undamped Jacobi smoother (Sec. 4.3), pinned against closed forms."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import gmg as O
from paper_1904_03317_gb300 import inputs
from tests.helpers import workload_rhs, oracle_hierarchy, small_workloads


@pytest.mark.parametrize("kappa", [2.0, 10.0, 100.0, 1e4])
@pytest.mark.parametrize("eps", [1e-3, 1e-6])
def test_chebyshev_degree_is_the_smallest_meeting_the_bound(kappa, eps):
    m = O.chebyshev_degree(kappa, eps)
    q = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    assert 2 * q ** m <= eps < 2 * q ** (m - 1)


def test_chebyshev_meets_its_a_priori_bound_in_the_energy_norm():
    # the 343-unknown coarse matrix of the 3D Q2 workloads, exact spectrum of D^-1 A
    H = oracle_hierarchy("3d_q2_sphere")
    A = H.levels[0].A
    dinv = 1.0 / A.diagonal()
    ev = np.linalg.eigvals(np.diag(dinv) @ A.toarray()).real
    a, b = ev.min(), ev.max()
    m = O.chebyshev_degree(b / a, 1e-3)
    rng = np.random.default_rng(3)
    for _ in range(3):
        g = rng.uniform(-1, 1, A.shape[0])
        xe = np.linalg.solve(A.toarray(), g)
        x = O.chebyshev(A, dinv, np.zeros_like(g), g, 1.0, m, x0_is_zero=True, lo=a, hi=b)
        e = x - xe
        assert np.sqrt(e @ (A @ e)) <= 1e-3 * np.sqrt(xe @ (A @ xe)) * (1 + 1e-9)


def test_ritz_values_lie_inside_the_spectrum():
    H = oracle_hierarchy("3d_q2_sphere")
    A = H.levels[0].A
    dinv = 1.0 / A.diagonal()
    ev = np.linalg.eigvals(np.diag(dinv) @ A.toarray()).real
    lo, hi = O.lanczos_extremes(A, dinv, O.eigen_start_vector(A.shape[0]), 1e-3)
    assert ev.min() - 1e-12 <= lo <= hi <= ev.max() + 1e-12
    # from a start vector with components along every eigenvector, run to
    # convergence, the extreme Ritz values reach the extremes
    b0 = np.random.default_rng(6).uniform(-1, 1, A.shape[0])
    lo, hi = O.lanczos_extremes(A, dinv, b0, 1e-14)
    assert abs(hi - ev.max()) <= 1e-3 * ev.max() and abs(lo - ev.min()) <= 1e-6 * ev.min()


def test_jacobi_closed_forms():
    rng = np.random.default_rng(4)
    d = rng.uniform(1, 5, 30)
    A = sp.diags(d).tocsr()
    g = rng.uniform(-1, 1, 30)
    # a diagonal system is solved by one step
    np.testing.assert_allclose(O.jacobi(A, 1 / d, None, g, 1, x0_is_zero=True), g / d, rtol=1e-15)
    # two steps on a general matrix: x2 = x1 + D^-1 (g - A x1), x1 = D^-1 g
    H = oracle_hierarchy("2d_q1_circle")
    B = H.levels[2].A_S
    di = H.levels[2].dinv
    h = rng.uniform(-1, 1, B.shape[0])
    x1 = di * h
    np.testing.assert_allclose(O.jacobi(B, di, None, h, 2, x0_is_zero=True), x1 + di * (h - B @ x1), rtol=1e-14)


def test_plain_cg_exact_after_distinct_eigenvalues():
    A = sp.diags(np.repeat([1.0, 3.0, 7.0], 10)).tocsr()
    b = np.random.default_rng(5).uniform(-1, 1, 30)
    x = O.cg_plain(A, b, 1e-14)
    np.testing.assert_allclose(A @ x, b, atol=1e-12)


@pytest.mark.parametrize("variant", [("chebyshev", "cholesky", 4), ("chebyshev", "chebyshev", 4),
                                     ("chebyshev", "cg", 4), ("jacobi", "cg", 1)])
@pytest.mark.parametrize("name", ["2d_q1_circle", "3d_q2_sphere"])
def test_solver_variants_converge(variant, name):
    smoother, coarse, degree = variant
    H = oracle_hierarchy(name)
    saved = (H.smoother, H.coarse, H.cheb_degree)
    try:
        H.smoother, H.cheb_degree = smoother, degree
        O.setup_coarse(H, coarse)
        w = small_workloads()[name]
        b = workload_rhs(H, w)
        res = O.solve(H, b, 1e-8)
        assert res.converged
        assert res.iterations <= (12 if smoother == "chebyshev" else 40)
        assert np.linalg.norm(b - H.disc.A @ res.x) <= 2e-8 * np.linalg.norm(b)
    finally:
        H.smoother, H.cheb_degree = saved[0], saved[2]
        O.setup_coarse(H, saved[1])
