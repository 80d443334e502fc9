"""Batched solves (gmg_solve_batch): each problem's result in the batch equals
its result alone and, for the problems the oracle can solve, the oracle's; a
failing problem does not disturb the others."""
import numpy as np
import pytest

from oracle import gmg as ogmg
from paper_1904_03317_gb300 import gmg as G
from paper_1904_03317_gb300 import inputs
from tests.helpers import oracle_hierarchy, small_workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_03317_gb300 import build
    build.build()
    return T


def _problems():
    ws = list(small_workloads().values())
    ws += [w for w in inputs.batched_problems(24) if w.coarse.dim == 2 or w.degree == 1][:6]
    return ws


def _setup(torch, prec):
    ctx = G.Context(0)
    out = []
    for w in _problems():
        m = G.build_mesh(w)
        H = G.Hierarchy(ctx, m, w.degree, w.coeff, cheb_degree=w.cheb_degree, vcycle_prec=prec)
        b = torch.empty(H.n, dtype=torch.float64, device="cuda")
        H.assemble_rhs(b, "random", w.seed + 11)
        out.append((H, m, b))
    return ctx, out


@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_batch_equals_alone(torch, prec):
    ctx, probs = _setup(torch, prec)
    alone = []
    for H, m, b in probs:
        x = torch.zeros_like(b)
        st = H.solve(b, x, tol=1e-8)
        alone.append((st.iterations, x.clone()))
    xs = [torch.full_like(b, 3.0) for _, _, b in probs]
    stats, status = G.solve_batch([H for H, _, _ in probs], [b for _, _, b in probs], xs, tol=1e-8, n_streams=4)
    tol = 1e-11 if prec == G.PREC_FP64 else 1e-5
    for (its, xa), st, rc, xb in zip(alone, stats, status, xs):
        assert rc == G.OK and st.converged
        assert abs(st.iterations - its) <= (0 if prec == G.PREC_FP64 else 1)
        if st.iterations == its:
            assert float(torch.linalg.vector_norm(xb - xa) / torch.linalg.vector_norm(xa)) <= tol
    # the problems of the parity set against the FP64 oracle
    if prec == G.PREC_FP64:
        for name, (st, rc, xb) in zip(small_workloads(), zip(stats, status, xs)):
            w = small_workloads()[name]
            O = oracle_hierarchy(name)
            ref = ogmg.solve(O, inputs.random_rhs(w.seed + 11, O.disc.n), 1e-8)
            assert abs(ref.iterations - st.iterations) <= 1
            if ref.iterations == st.iterations:
                xh = xb.cpu().numpy()
                assert np.abs(xh - ref.x).max() <= 1e-10 * np.abs(ref.x).max(), name
    # a second batch reuses the graphs and gives the same answers
    xs2 = [torch.zeros_like(b) for _, _, b in probs]
    stats2, status2 = G.solve_batch([H for H, _, _ in probs], [b for _, _, b in probs], xs2, tol=1e-8, n_streams=3)
    assert all(rc == G.OK for rc in status2)
    assert [s.iterations for s in stats2] == [s.iterations for s in stats] or prec == G.PREC_FP32


def test_batch_isolates_a_failing_problem(torch):
    ctx, probs = _setup(torch, G.PREC_FP64)
    bs = [b.clone() for _, _, b in probs]
    bs[2][5] = float("nan")
    xs = [torch.zeros_like(b) for b in bs]
    stats, status = G.solve_batch([H for H, _, _ in probs], bs, xs, tol=1e-8, max_iter=2, n_streams=2)
    assert status[2] == G.ENAN
    for i, (rc, st) in enumerate(zip(status, stats)):
        if i != 2:
            assert rc in (G.OK, G.ENOTCONV) and st.iterations == 2 or (rc == G.OK and st.converged)


def test_deterministic_batch_equals_alone_bitwise(torch):
    """In deterministic mode a problem's result in the batch has the same bits
    as the problem solved alone (FP32 V-cycle)."""
    ctx = G.Context(0)
    probs = []
    for w in _problems():
        H = G.Hierarchy(ctx, G.build_mesh(w), w.degree, w.coeff, cheb_degree=w.cheb_degree,
                        vcycle_prec=G.PREC_FP32, deterministic=True)
        b = torch.empty(H.n, dtype=torch.float64, device="cuda")
        H.assemble_rhs(b, "random", w.seed + 11)
        probs.append((H, b))
    alone = []
    for H, b in probs:
        x = torch.zeros_like(b)
        H.solve(b, x, tol=1e-8)
        alone.append(x.clone())
    xs = [torch.full_like(b, 3.0) for _, b in probs]
    stats, status = G.solve_batch([H for H, _ in probs], [b for _, b in probs], xs, tol=1e-8, n_streams=4)
    torch.cuda.synchronize()
    for xa, xb, rc in zip(alone, xs, status):
        assert rc == G.OK and torch.equal(xa, xb)


def test_tile_shape_does_not_change_the_solve(torch):
    """The smoother's partial-brick threshold (2, the default 4, full bricks
    only) moves groups between the brick and the single-group kernels; with
    FP64 V-cycles each setting matches the oracle's solve at its iteration
    count."""
    name = "3d_q2_checker"
    w = small_workloads()[name]
    O = oracle_hierarchy(name)
    b = inputs.random_rhs(w.seed + 5, O.disc.n)
    ref = ogmg.solve(O, b, 1e-10)
    ctx = G.Context(0)
    m = G.build_mesh(w)
    seen = set()
    for t in (2, 4, 8):
        H = G.Hierarchy(ctx, m, w.degree, w.coeff, cheb_degree=w.cheb_degree, vcycle_prec=G.PREC_FP64,
                        brick_min_members=t, fixed_lambda=[lev.lam for lev in O.levels])
        seen.add(tuple(int(v) for v in H.info.bricks_partial[:H.info.n_levels]))
        x = torch.zeros(H.n, dtype=torch.float64, device="cuda")
        st = H.solve(torch.tensor(b, device="cuda"), x, tol=1e-10)
        assert st.converged and abs(st.iterations - ref.iterations) <= 1
        if st.iterations == ref.iterations:
            xh = x.cpu().numpy()
            assert np.abs(xh - ref.x).max() <= 1e-10 * np.abs(ref.x).max(), t
        H.close()
    assert len(seen) > 1  # the thresholds really give different partitions


def test_autotuner_picks_a_tile_per_3d_class(torch):
    from paper_1904_03317_gb300 import batch
    pool = list(inputs.batched_problems(48, n_max=6e4))
    ws = [w for w in pool if w.coarse.dim == 3][:3] + [w for w in pool if w.coarse.dim == 2][:2]
    meshes = [G.build_mesh(w) for w in ws]
    ctx = G.Context(0)
    tun = batch.tune_tiles(torch, ctx, ws, meshes, reps=1, candidates=(2, 8))
    want = {batch.problem_class(3, w.degree, m.num_leaves()) for w, m in zip(ws, meshes) if w.coarse.dim == 3}
    assert want and set(tun.tile) == want
    for c, v in tun.tile.items():
        assert v in (2, 8) and set(tun.tile_ms[c]) == {2, 8} and all(t > 0 for t in tun.tile_ms[c].values())
    assert len(tun.record()["tile_brick_min_members"]) == len(want)
