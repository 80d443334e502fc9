"""C-ABI library on the CPU: it loads, exports every declared symbol, builds
hierarchies on a host-only context identical to the oracle's, and rejects
invalid input with GMG_EINVAL.  No compute call runs here (no GPU)."""
import os
import re

import numpy as np
import pytest

from oracle import fem
from oracle.mesh import build_forest
from paper_1904_03317_gb300 import gmg as G
from paper_1904_03317_gb300 import inputs
from tests.helpers import small_workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1904_03317_gb300 import build
    build.build()
    yield


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gmg_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = G.load_library()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(G.EXPORTED) == names


def test_build_info_reports_sm103a():
    import ctypes as C
    a, v = C.c_int(), C.c_int()
    assert G.load_library().gmg_build_info(C.byref(a), C.byref(v)) == 0
    assert a.value == 1 and v.value == 2


def test_leaf_cells_partitioned_into_patches_groups_and_single_cells():
    """Every leaf cell is in exactly one patch, group or single-cell list,
    and the parity workloads exercise all three forms of the leaf operator
    (Q2 3D with cubic and with stretched cells, Q1 3D, Q1 2D)."""
    seen = {}
    for name, w in small_workloads().items():
        m = G.build_mesh(w)
        i = G.Hierarchy(G.Context(-1), m, w.degree, w.coeff).info
        nch = 2 ** w.coarse.dim
        assert i.leaf_patches * nch * nch + i.leaf_groups * nch + i.leaf_single_cells == i.n_leaves
        seen[name] = (i.leaf_patches, i.leaf_groups, i.leaf_single_cells)
    for name in ("3d_q2_patches", "3d_q2_checker", "3d_q1_sphere", "2d_q1_circle"):
        assert min(seen[name]) > 0, (name, seen[name])
    # a ragged last block of the Q2 3D patch kernel (3 patches per block)
    assert seen["3d_q2_patches"][0] % 3 != 0


def test_smoother_tiles_of_the_parity_workloads():
    """The 3D parity workloads exercise both brick forms of the smoother:
    full bricks (eight uniform groups of one coefficient) and partial bricks
    (four to seven), and every group is in at most one brick."""
    for name, w in small_workloads().items():
        m = G.build_mesh(w)
        i = G.Hierarchy(G.Context(-1), m, w.degree, w.coeff).info
        full = sum(i.bricks[l] for l in range(i.n_levels))
        partial = sum(i.bricks_partial[l] for l in range(i.n_levels))
        for l in range(1, i.n_levels):
            assert 8 * i.bricks[l] + 4 * i.bricks_partial[l] <= i.groups[l]
        if w.coarse.dim == 3:
            assert full > 0 and partial > 0, name
        else:
            assert full == 0 and partial == 0, name


@pytest.mark.parametrize("name", list(small_workloads()))
def test_host_hierarchy_matches_oracle(name):
    w = small_workloads()[name]
    m = G.build_mesh(w)
    H = G.Hierarchy(G.Context(-1), m, w.degree, w.coeff)
    f = build_forest(w.coarse, w.rounds)
    lv, co = m.leaves()
    assert set((l, tuple(c)) for l, c in f.leaves()) == set(
        (int(l), tuple(int(x) for x in c)) for l, c in zip(lv, co))
    d = fem.Discretization(f, w.degree, w.coeff)
    np.testing.assert_array_equal(H.export(G.EXPORT_UNKNOWN_KEYS), d.unknown_keys)
    np.testing.assert_array_equal(H.export(G.EXPORT_HOME_LEVEL), d.home_level)
    hang = H.export(G.EXPORT_HANGING)
    got = sorted((int(r["key"]), int(r["master"]), round(float(r["w"]), 12)) for r in hang)
    want = sorted((k, m_, round(w_, 12)) for k, row in d.hanging.items() for m_, w_ in row
                  if not d.is_dirichlet(m_))
    assert got == want
    for l in range(d.L + 1):
        keys, iface, _ = d.level_space(l)
        lk = H.export(G.EXPORT_LEVEL_KEYS, l)
        lc = H.export(G.EXPORT_LEVEL_CLASS, l)
        np.testing.assert_array_equal(np.sort(lk[lc == 1]), keys[~iface])
        np.testing.assert_array_equal(np.sort(lk[lc == 2]), keys[iface])
    info = H.info
    assert info.n_unknowns == d.n and info.n_levels == d.L + 1
    assert sum(info.n_home[l] for l in range(info.n_levels)) == d.n


def test_leaves_are_in_morton_order_within_coarse_cells():
    cm = inputs.CoarseMesh(2, (2, 1, 1), (0, 0, 0), (2, 1, 1))
    m = G.Mesh(cm)
    m.refine(np.ones(2, dtype=np.uint8))
    lv, co = m.leaves()
    # coarse cell 0 first; children in z-order (x fastest, then y)
    assert [tuple(c[:2]) for c in co[:4]] == [(0, 0), (1, 0), (0, 1), (1, 1)]
    assert [tuple(c[:2]) for c in co[4:]] == [(2, 0), (3, 0), (2, 1), (3, 1)]


def test_invalid_arguments_are_rejected():
    with pytest.raises(G.GmgError) as e:
        G.Mesh(inputs.CoarseMesh(4, (1, 1, 1), (0, 0, 0), (1, 1, 1)))
    assert e.value.status == G.EINVAL
    with pytest.raises(G.GmgError) as e:
        G.Mesh(inputs.CoarseMesh(2, (2, 2, 1), (0, 0, 0), (0.0, 1.0, 1.0)))
    assert e.value.status == G.EINVAL
    m = G.Mesh(inputs.CoarseMesh(2, (2, 2, 1), (0, 0, 0), (1, 1, 1)))
    with pytest.raises(G.GmgError) as e:
        m.refine(np.ones(3, dtype=np.uint8))  # wrong length
    assert e.value.status == G.EINVAL
    ctx = G.Context(-1)
    with pytest.raises(G.GmgError) as e:
        G.Hierarchy(ctx, m, 3)
    assert e.value.status == G.EINVAL
    with pytest.raises(G.GmgError) as e:
        G.Hierarchy(ctx, m, 1, coarse_coeff=[1.0, -1.0, 1.0, 1.0])
    assert e.value.status == G.EINVAL
    H = G.Hierarchy(ctx, m, 1)
    # device calls on a host-only hierarchy fail cleanly
    x = np.zeros(max(1, H.n))
    with pytest.raises(G.GmgError) as e:
        H.apply(x, x.copy())
    assert e.value.status == G.EINVAL


def test_closure_after_deep_refinement_matches_oracle():
    cm = inputs.CoarseMesh(3, (2, 2, 2), (0, 0, 0), (1, 1, 1))
    rounds = [inputs.round_sphere_surface((0.4301, 0.3701, 0.5501), 0.003)] * 5
    m = G.Mesh(cm)
    m.apply_rounds(rounds)
    f = build_forest(cm, rounds)
    lv, co = m.leaves()
    assert set((l, tuple(c)) for l, c in f.leaves()) == set(
        (int(l), tuple(int(x) for x in c)) for l, c in zip(lv, co))


@pytest.mark.parametrize("name", ["3d_q2_sphere", "2d_q2_circle", "3d_q2_checker"])
def test_chebyshev_coarse_setup_matches_oracle(name):
    """Degree and eigenvalue range of the Chebyshev coarse solver (Sec. 4.1)
    from the host builder equal the oracle's."""
    from oracle import gmg as ogmg
    from tests.helpers import oracle_hierarchy
    w = small_workloads()[name]
    H = G.Hierarchy(G.Context(-1), G.build_mesh(w), w.degree, w.coeff, coarse_solver=G.COARSE_CHEBYSHEV)
    O = oracle_hierarchy(name)
    try:
        ogmg.setup_coarse(O, "chebyshev")
        assert H.info.coarse_degree == O.coarse_degree
        np.testing.assert_allclose(list(H.info.coarse_range), O.coarse_range, rtol=1e-9)
    finally:
        ogmg.setup_coarse(O, "cholesky")


def test_invalid_solver_variants_rejected():
    w = small_workloads()["2d_q1_circle"]
    m = G.build_mesh(w)
    for kw in (dict(smoother=7), dict(coarse_solver=3), dict(coarse_tol=0.0), dict(coarse_tol=1.5)):
        with pytest.raises(Exception):
            G.Hierarchy(G.Context(-1), m, w.degree, **kw)


@pytest.mark.parametrize("depth", [6, 20])
def test_leaf_order_is_depth_first_z_order(depth):
    """The library lists leaves in the canonical order (coarse cells in
    lexicographic order, then depth-first with children in z-order), both
    when tree, Morton index and level fit one 64-bit sort key and at the
    deepest allowed level (3D, level 20), where they do not."""
    from oracle import partition
    cm = inputs.CoarseMesh(3, (2, 1, 1), (0.0, 0.0, 0.0), (2.0, 1.0, 1.0))
    rounds = [inputs.round_sphere_surface((0.3001, 0.4001, 0.5001), 1e-7)] * depth
    f = build_forest(cm, rounds)
    m = G.Mesh(cm)
    m.apply_rounds(rounds)
    lv, co = m.leaves()
    assert int(lv.max()) == depth
    got = [(int(l), tuple(int(x) for x in c)) for l, c in zip(lv, co)]
    assert got == [(l, tuple(c)) for l, c in partition._dfs_leaves(f)]


@pytest.mark.parametrize("name", ["2d_q2_circle", "3d_q2_checker", "3d_q1_sphere"])
def test_build_hierarchy_in_one_call_equals_stepwise(name):
    """gmg_build_hierarchy (forest, rounds through the flag callback, then the
    hierarchy) gives the hierarchy of gmg_mesh_create + gmg_mesh_refine per
    round + gmg_hier_build."""
    w = small_workloads()[name]
    ctx = G.Context(-1)
    a = G.Hierarchy(ctx, G.build_mesh(w), w.degree, w.coeff, cheb_degree=w.cheb_degree)
    b = G.build_hierarchy(ctx, w.coarse, w.rounds, w.degree, w.coeff, cheb_degree=w.cheb_degree)
    assert a.n == b.n and a.info.n_levels == b.info.n_levels
    for what in (G.EXPORT_UNKNOWN_KEYS, G.EXPORT_HOME_LEVEL, G.EXPORT_HOME_SLOT):
        np.testing.assert_array_equal(a.export(what), b.export(what))
    np.testing.assert_array_equal(a.export(G.EXPORT_HANGING), b.export(G.EXPORT_HANGING))
    for l in range(a.info.n_levels):
        np.testing.assert_array_equal(a.export(G.EXPORT_LEVEL_KEYS, l), b.export(G.EXPORT_LEVEL_KEYS, l))
        np.testing.assert_array_equal(a.export(G.EXPORT_LEVEL_CLASS, l), b.export(G.EXPORT_LEVEL_CLASS, l))


def test_build_hierarchy_errors():
    w = small_workloads()["2d_q1_circle"]
    ctx = G.Context(-1)
    # no rounds: the coarse mesh alone
    h = G.build_hierarchy(ctx, w.coarse, [], w.degree)
    assert h.info.n_levels == 1 and h.n == (4 - 1) * (4 - 1)

    def stop(cm, level, coords, finest):
        raise KeyError("flag function failed")

    with pytest.raises(KeyError):
        G.build_hierarchy(ctx, w.coarse, [inputs.round_uniform(), stop], w.degree)
    import ctypes as C
    lib = G.load_library()
    cm = G.CoarseMeshC()
    cm.dim, cm.n0[0], cm.n0[1], cm.n0[2] = 2, 2, 2, 1
    for d in range(3):
        cm.lo[d], cm.hi[d] = 0.0, 1.0
    out = C.c_void_p()
    halt = G.REFINE_FN(lambda user, r, n, lv, co, fl: 1)
    assert lib.gmg_build_hierarchy(ctx.handle, C.byref(cm), 1, halt, None, 1, None, None, C.byref(out)) == G.EINVAL
    assert not out.value
    assert lib.gmg_build_hierarchy(ctx.handle, C.byref(cm), 1, G.REFINE_FN(), None, 1, None, None,
                                   C.byref(out)) == G.EINVAL
    assert lib.gmg_build_hierarchy(ctx.handle, C.byref(cm), -1, halt, None, 1, None, None, C.byref(out)) == G.EINVAL


def test_brick_min_members_is_the_partial_brick_threshold():
    """gmg_params.brick_min_members (the smoother's tile shape): lowering it
    forms more partial bricks, 8 forms none (a position with all eight
    groups smoothable is a full brick); every group stays in at most one
    brick; values outside [2, 8] other than 0 are rejected."""
    w = small_workloads()["3d_q2_checker"]
    m = G.build_mesh(w)
    counts = {}
    for t in (2, 3, 4, 8):
        i = G.Hierarchy(G.Context(-1), m, w.degree, w.coeff, brick_min_members=t).info
        counts[t] = sum(i.bricks_partial[l] for l in range(i.n_levels))
        assert all(8 * i.bricks[l] + t * i.bricks_partial[l] <= i.groups[l] for l in range(1, i.n_levels))
    assert counts[2] >= counts[3] >= counts[4] >= counts[8] == 0 and counts[2] > counts[4]
    for bad in (1, 9, -1):
        with pytest.raises(G.GmgError):
            G.Hierarchy(G.Context(-1), m, w.degree, w.coeff, brick_min_members=bad)
