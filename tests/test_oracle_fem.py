"""Pins of the oracle's finite-element layer against closed forms (CPU only)."""
import itertools

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem
from oracle.mesh import build_forest
from oracle.gmg import build_hierarchy
from paper_1904_03317_gb300 import inputs

# textbook 1-D matrices on the unit interval
K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
M1 = np.array([[2.0, 1.0], [1.0, 2.0]]) / 6.0
K2 = np.array([[7.0, -8.0, 1.0], [-8.0, 16.0, -8.0], [1.0, -8.0, 7.0]]) / 3.0
M2 = np.array([[4.0, 2.0, -1.0], [2.0, 16.0, 2.0], [-1.0, 2.0, 4.0]]) / 30.0


def _kron_sum(dim, K, M, h):
    """sum_i (x-fastest Kronecker product with K/h_i in direction i, M h_j elsewhere)."""
    out = 0.0
    for i in range(dim):
        mats = [K / h[e] if e == i else M * h[e] for e in range(dim)]
        term = mats[0]
        for e in range(1, dim):
            term = np.kron(mats[e], term)  # later directions vary slower
        out = out + term
    return out


@pytest.mark.parametrize("dim,k", [(1, 1), (1, 2), (2, 1), (2, 2), (3, 1), (3, 2)])
def test_element_stiffness_is_kronecker_sum_of_textbook_1d(dim, k):
    h = np.array([0.3, 0.7, 1.1])[:dim]
    K, M = (K1, M1) if k == 1 else (K2, M2)
    A = fem.element_stiffness(dim, k, np.concatenate([h, [1.0] * (3 - dim)]))
    np.testing.assert_allclose(A, _kron_sum(dim, K, M, h), rtol=1e-13, atol=1e-14)


def _uniform(dim, k, g, n0=4):
    cm = inputs.CoarseMesh(dim, (n0, n0, n0 if dim == 3 else 1), (0, 0, 0), (1, 1, 1))
    f = build_forest(cm, [inputs.round_uniform()] * g)
    return fem.Discretization(f, k)


def _row_stencil(d, key):
    i = int(fem.lookup(d.unknown_keys, np.array([key]))[0])
    row = d.A.getrow(i)
    q0 = fem.unpack_keys(key)
    out = {}
    for j, v in zip(row.indices, row.data):
        q = fem.unpack_keys(d.unknown_keys[j])
        out[tuple(int(x) for x in (q - q0) // d.node_scale(d.L))] = v
    return out


def test_q1_2d_nine_point_stencil():
    """Bilinear Laplacian on a uniform grid: 8/3 at the centre, -1/3 at the 8 neighbours."""
    d = _uniform(2, 1, 2)
    key = int(fem.pack_keys(np.array([8, 8, 0])))
    st = _row_stencil(d, key)
    assert st.pop((0, 0, 0)) == pytest.approx(8.0 / 3.0, rel=1e-14)
    assert len(st) == 8
    for v in st.values():
        assert v == pytest.approx(-1.0 / 3.0, rel=1e-14)


def test_q1_3d_27_point_stencil():
    """Trilinear Laplacian, spacing h: 8h/3 centre, 0 faces, -h/6 edges, -h/12 corners."""
    d = _uniform(3, 1, 1)
    h = 1.0 / 8.0
    key = int(fem.pack_keys(np.array([4, 4, 4])))
    st = _row_stencil(d, key)
    for off in itertools.product((-1, 0, 1), repeat=3):
        n = sum(abs(o) for o in off)
        want = {0: 8 * h / 3, 1: 0.0, 2: -h / 6, 3: -h / 12}[n]
        assert st.get(off, 0.0) == pytest.approx(want, rel=1e-13, abs=1e-15)


def _adaptive(dim, k, coeff=None, g=1, rounds=2):
    if dim == 2:
        cm = inputs.CoarseMesh(2, (4, 4, 1), (0, 0, 0), (1, 1, 1))
        rr = [inputs.round_uniform()] * g + [inputs.round_sphere_surface((0.5, 0.5), 0.3)] * rounds
    else:
        cm = inputs.CoarseMesh(3, (2, 2, 2), (0, 0, 0), (1, 1, 1))
        rr = [inputs.round_uniform()] * g + [inputs.round_sphere_surface((0.5, 0.5, 0.5), 0.3)] * rounds
    f = build_forest(cm, rr)
    c = None
    if coeff == "checker":
        c = inputs.checkerboard_coefficients(cm, 1.0, 100.0)
    return fem.Discretization(f, k, c)


def _bubble(x):
    return np.prod(x * (1.0 - x), axis=-1)


def _bubble_energy_box(lo, hi, dim):
    """int_box |grad prod x_i(1-x_i)|^2 from 1-D antiderivatives."""
    def F_sq(a, b):  # int (x(1-x))^2 = x^3/3 - x^4/2 + x^5/5
        P = lambda x: x ** 3 / 3 - x ** 4 / 2 + x ** 5 / 5
        return P(b) - P(a)

    def F_dsq(a, b):  # int (1-2x)^2 = x - 2x^2 + 4x^3/3
        P = lambda x: x - 2 * x ** 2 + 4 * x ** 3 / 3
        return P(b) - P(a)

    tot = 0.0
    for j in range(dim):
        t = F_dsq(lo[j], hi[j])
        for i in range(dim):
            if i != j:
                t *= F_sq(lo[i], hi[i])
        tot += t
    return tot


@pytest.mark.parametrize("dim", [2, 3])
def test_q2_bubble_energy_with_hanging_nodes_and_jumps(dim):
    """u = prod x_i(1-x_i) lies in Q2 and vanishes on the boundary, so its nodal
    interpolant on the adaptive mesh is exact and u^T A u must equal
    sum over coarse cells of a_c int_c |grad u|^2.  Pins element matrices,
    coefficients, assembly and the hanging-node elimination C together."""
    d = _adaptive(dim, 2, coeff="checker")
    assert len(d.hanging) > 0
    u = _bubble(d.node_positions(d.unknown_keys)[:, :dim])
    # the constrained interpolant reproduces u at every leaf node
    full = d.C @ u
    np.testing.assert_allclose(full, _bubble(d.node_positions(d.all_keys)[:, :dim]), atol=1e-14)
    cm = d.forest.cm
    want = 0.0
    for idx, a in enumerate(d.coarse_coeff):
        c = [idx % cm.n0[0], (idx // cm.n0[0]) % cm.n0[1], idx // (cm.n0[0] * cm.n0[1])]
        lo = [c[e] / cm.n0[e] for e in range(dim)]
        hi = [(c[e] + 1) / cm.n0[e] for e in range(dim)]
        want += a * _bubble_energy_box(lo, hi, dim)
    assert float(u @ (d.A @ u)) == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("dim,k,expected", [
    (2, 1, {0.5}),
    (3, 1, {0.5, 0.25}),
    (2, 2, {0.375, 0.75, -0.125}),
])
def test_hanging_weights_closed_form(dim, k, expected):
    d = _adaptive(dim, k)
    ws = set()
    for row in d.hanging.values():
        for _, w in row:
            ws.add(round(w, 12))
    assert ws == {round(x, 12) for x in expected}


def test_q2_3d_face_hanging_weights_are_products():
    d = _adaptive(3, 2)
    e = [0.375, 0.75, -0.125]
    allowed = {round(x, 12) for x in e} | {round(a * b, 12) for a in e for b in e}
    got = {round(w, 12) for row in d.hanging.values() for _, w in row}
    assert got <= allowed and len(got) > 3
    for row in d.hanging.values():
        assert sum(w for _, w in row) == pytest.approx(1.0, abs=1e-13) or len(row) < 3


@pytest.mark.parametrize("dim,k,g", [(2, 1, 2), (2, 2, 1), (3, 1, 1)])
def test_manufactured_convergence_rate(dim, k, g):
    """L2 error of the Galerkin solution for u = prod sin(pi x_i) drops by about
    2^(k+1) per uniform refinement."""
    errs = []
    for gg in (g, g + 1):
        d = _uniform(dim, k, gg)
        x = spla.spsolve(d.A.tocsc(), d.rhs_sine())
        errs.append(d.l2_error(x, fem.sine_solution(dim)))
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - (k + 1)) < 0.25, (errs, rate)


def test_adaptive_solution_matches_manufactured():
    d = _adaptive(2, 2, g=1, rounds=2)
    x = spla.spsolve(d.A.tocsc(), d.rhs_sine())
    assert d.l2_error(x, fem.sine_solution(2)) < 2e-3


def test_matrices_symmetric():
    d = _adaptive(3, 2, coeff="checker")
    assert abs(d.A - d.A.T).max() < 1e-13 * abs(d.A).max()
    for l in range(d.L + 1):
        keys, iface, A = d.level_space(l)
        assert abs(A - A.T).max() < 1e-13 * abs(A).max()


def test_uniform_mesh_has_no_interface():
    d = _uniform(2, 2, 2)
    for l in range(d.L + 1):
        keys, iface, A = d.level_space(l)
        assert not iface.any()


def _corner_refined(dim, n0x, k):
    """Coarse cells n0x x 1 (x 1) on [0, n0x] x [0, 1] (x [0, 1]): the cell at
    the origin refined, then its child at the origin refined again."""
    cm = inputs.CoarseMesh(dim, (n0x, 1, 1), (0, 0, 0), (n0x, 1, 1))

    def at_origin(level):
        return lambda cm_, lv, co, maxl: (lv == level) & np.all(co == 0, axis=1)

    f = build_forest(cm, [at_origin(0), at_origin(1)])
    assert [len(c) for c in f.cells] == [n0x, 2 ** dim, 2 ** dim]
    return fem.Discretization(f, k)


def _level_nodes(d, level):
    keys, iface, _ = d.level_space(level)
    pos = d.node_positions(keys)[:, :d.dim]
    fr = lambda p: tuple(float(v) for v in p)
    return {fr(p) for p in pos}, {fr(p) for p in pos[iface]}


@pytest.mark.parametrize("k", [1, 2])
def test_interface_nodes_listed_by_hand_2d(k):
    """Sec. 2.3's I set on a hand-built 2D mesh: coarse cells [0,1]x[0,1] and
    [1,2]x[0,1]; the first refined once and its child at the origin once more.
    Level 1 (h = 1/2) has its four cells in [0,1]^2: a level-1 node is I iff a
    level-1 lattice cell touching it is missing, which happens only on x = 1,
    next to the unrefined coarse cell.  Level 2 (h = 1/4) has its four cells
    in [0,1/2]^2: its I nodes are those on x = 1/2 or y = 1/2.  The domain's
    boundary (x in {0, 2}, y in {0, 1}) is Dirichlet and holds no level node."""
    d = _corner_refined(2, 2, k)
    grid = lambda hi, step: [step * i for i in range(1, int(round(hi / step)) + 1)]
    h1, h2 = 0.5 / k, 0.25 / k  # node spacing on levels 1 and 2
    nodes1, iface1 = _level_nodes(d, 1)
    assert nodes1 == {(x, y) for x in grid(1.0, h1) for y in grid(1.0, h1) if y < 1.0}
    assert iface1 == {(1.0, y) for y in grid(1.0, h1) if y < 1.0}
    nodes2, iface2 = _level_nodes(d, 2)
    assert nodes2 == {(x, y) for x in grid(0.5, h2) for y in grid(0.5, h2)}
    assert iface2 == {(x, y) for (x, y) in nodes2 if x == 0.5 or y == 0.5}
    assert len(iface2) == (3 if k == 1 else 7)
    # level 0: Q1 has no interior vertex (every vertex has y in {0, 1}); Q2
    # has the two cell centres and the midpoint of the shared edge; no level-0
    # cell is missing
    nodes0, iface0 = _level_nodes(d, 0)
    want0 = set() if k == 1 else {(0.5, 0.5), (1.0, 0.5), (1.5, 0.5)}
    assert nodes0 == want0 and not iface0


def test_interface_nodes_listed_by_hand_3d():
    """The same construction on the unit cube (Q1): level 2's cells fill
    [0,1/2]^3, and its I nodes are the seven non-Dirichlet nodes with a
    coordinate equal to 1/2; level 1's one interior node is not I."""
    d = _corner_refined(3, 1, 1)
    nodes1, iface1 = _level_nodes(d, 1)
    assert nodes1 == {(0.5, 0.5, 0.5)} and not iface1
    nodes2, iface2 = _level_nodes(d, 2)
    q = (0.25, 0.5)
    assert nodes2 == {(x, y, z) for x in q for y in q for z in q}
    assert iface2 == nodes2 - {(0.25, 0.25, 0.25)}


def test_adaptive_mesh_has_interface():
    d = _adaptive(2, 1)
    assert any(d.level_space(l)[1].any() for l in range(1, d.L + 1))


def test_prolongation_q1_hat_functions():
    """P e_y is the coarse hat function of node y sampled at the fine nodes (embedding)."""
    d = _adaptive(2, 1)
    for l in range(1, d.L + 1):
        kf = d.level_space(l)[0]
        kc = d.level_space(l - 1)[0]
        P = d.prolongation(l, kf, kc).toarray()
        H = d.cell_h(l - 1)[:2]
        xf = d.node_positions(kf)[:, :2]
        xc = d.node_positions(kc)[:, :2]
        for j in range(0, len(kc), max(1, len(kc) // 15)):
            hat = np.prod(np.maximum(0.0, 1.0 - np.abs(xf - xc[j]) / H), axis=1)
            np.testing.assert_allclose(P[:, j], hat, atol=1e-14)


@pytest.mark.parametrize("dim", [2, 3])
def test_prolongation_q2_polynomial_exact(dim):
    d = _adaptive(dim, 2)
    for l in range(1, d.L + 1):
        kf = d.level_space(l)[0]
        kc = d.level_space(l - 1)[0]
        P = d.prolongation(l, kf, kc)
        uc = _bubble(d.node_positions(kc)[:, :dim])
        uf = _bubble(d.node_positions(kf)[:, :dim])
        np.testing.assert_allclose(P @ uc, uf, atol=1e-14)


def test_restriction_lands_on_s_nodes_and_homes_unique():
    """R = P^T maps level l into V_{l-1}^S (complete layer, Sec. 2.3); every unknown
    has exactly one home level and is an S node there (asserted in the build)."""
    d = _adaptive(2, 2, g=1, rounds=3)
    H = build_hierarchy(d, 2)
    for l in range(1, len(H.levels)):
        P = H.levels[l].P.tocoo()
        cols = np.unique(P.col[P.data != 0])
        assert not H.levels[l - 1].iface[cols].any()
    assert len(H.home_index) == d.n
