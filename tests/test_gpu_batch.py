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
