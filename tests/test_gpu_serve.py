"""Request loop (continuous batching): every request is served, each result
in the mix equals the same request solved alone and agrees with the CPU
oracle, identical meshes reuse a cached hierarchy, and the memory budget
bounds the hierarchies in flight."""
import numpy as np
import pytest

from oracle import gmg as ogmg
from paper_1904_03317_gb300 import gmg as G
from paper_1904_03317_gb300 import inputs, serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_03317_gb300 import build
    build.build()
    return T


def _alone(torch, ctx, w):
    h = G.Hierarchy(ctx, G.build_mesh(w), w.degree, w.coeff, cheb_degree=w.cheb_degree, vcycle_prec=G.PREC_FP64)
    b = torch.empty(h.n, dtype=torch.float64, device="cuda")
    h.assemble_rhs(b, "random", w.seed)
    x = torch.zeros_like(b)
    st = h.solve(b, x, tol=1e-8)
    h.close()
    return st, x


def test_result_in_the_mix_equals_alone_and_oracle(torch):
    """FP64 V-cycles: a request's result in the mix is the result alone (to
    the rounding of the leaf operator's atomics) and, for the small requests,
    the oracle's FP64 solution (1e-10 at the same iteration count, +-1
    iteration otherwise)."""
    arrivals, ws = inputs.serving_requests(10, n_min=1e4, n_max=1.5e5, rate=200.0)
    srv = serve.Server(torch, setup_workers=4, max_live=8, vcycle_prec=G.PREC_FP64, keep_x=True)
    res = srv.run(arrivals, ws)
    assert all(r.status == G.OK and r.converged for r in res)
    assert all(r.ready >= r.setup_done >= r.hier_start >= r.meshed >= r.admitted >= r.arrival - 1e-9 for r in res)
    ctx = G.Context(0)
    oracle_checked = 0
    for r, w in zip(res, ws):
        st, x = _alone(torch, ctx, w)
        assert st.iterations == r.iterations and x.numel() == r.n
        assert float(torch.linalg.vector_norm(x - r.x) / torch.linalg.vector_norm(x)) <= 1e-11
        if r.n <= 40000:
            O = ogmg.setup(w)
            ref = ogmg.solve(O, inputs.random_rhs(w.seed, O.disc.n), 1e-8)
            xr = r.x.cpu().numpy()
            err = np.abs(xr - ref.x).max() / np.abs(ref.x).max()
            assert abs(ref.iterations - r.iterations) <= 1
            if ref.iterations == r.iterations:
                assert err <= 1e-10, err
            oracle_checked += 1
    assert oracle_checked >= 2


def test_identical_meshes_reuse_a_cached_hierarchy(torch):
    """Requests that repeat an earlier request's mesh (with their own
    right-hand sides) after it has finished take its hierarchy from the cache
    and give the same results as when solved alone."""
    _, base = inputs.serving_requests(2, n_min=1e4, n_max=4e4, rate=1.0)
    import dataclasses
    ws = [base[0], base[1], dataclasses.replace(base[0], seed=base[0].seed + 1),
          dataclasses.replace(base[1], seed=base[1].seed + 7)]
    arrivals = np.array([0.0, 0.0, 1.5, 1.5])
    srv = serve.Server(torch, setup_workers=2, max_live=4, vcycle_prec=G.PREC_FP64, keep_x=True)
    res = srv.run(arrivals, ws)
    assert all(r.status == G.OK and r.converged for r in res)
    assert [r.cache_hit for r in res] == [False, False, True, True] and srv.cache_hits == 2
    ctx = G.Context(0)
    for r, w in zip(res, ws):
        st, x = _alone(torch, ctx, w)
        assert st.iterations == r.iterations
        assert float(torch.linalg.vector_norm(x - r.x) / torch.linalg.vector_norm(x)) <= 1e-11


def test_memory_budget_serialises_hierarchies(torch):
    """A budget that holds one measured hierarchy but not two: after the first
    measurement every hierarchy is built only when the previous result has
    freed its memory."""
    arrivals, ws = inputs.serving_requests(5, n_min=1e4, n_max=5e4, rate=1e6)
    probe = serve.Server(torch, setup_workers=1, max_live=2, cache=False)
    probe.run(arrivals[:1], ws[:1])
    per_leaf = probe.bytes_per_leaf
    leaves = min(G.build_mesh(w).num_leaves() for w in ws)
    srv = serve.Server(torch, mem_budget=1.5 * per_leaf * leaves, setup_workers=4, max_live=8, cache=False)
    srv.bytes_per_leaf, srv._measured = per_leaf, True
    res = srv.run(arrivals, ws)
    assert all(r.status == G.OK for r in res)
    spans = sorted((r.hier_start, r.ready) for r in res)
    for (a0, e0), (a1, e1) in zip(spans, spans[1:]):
        assert a1 >= e0 - 1e-6


def test_deterministic_mix_equals_alone_bitwise(torch):
    """Deterministic mode: every request's result in the mix (FP32 V-cycles,
    overlapping on the device) has the same bits as the request solved
    alone."""
    arrivals, ws = inputs.serving_requests(6, n_min=1e4, n_max=6e4, rate=500.0)
    srv = serve.Server(torch, setup_workers=3, max_live=6, keep_x=True, deterministic=True)
    res = srv.run(arrivals, ws)
    ctx = G.Context(0)
    for r, w in zip(res, ws):
        assert r.status == G.OK and r.converged
        h = G.Hierarchy(ctx, G.build_mesh(w), w.degree, w.coeff, cheb_degree=w.cheb_degree,
                        vcycle_prec=G.PREC_FP32, deterministic=True)
        b = torch.empty(h.n, dtype=torch.float64, device="cuda")
        h.assemble_rhs(b, "random", w.seed)
        x = torch.zeros_like(b)
        st = h.solve(b, x, tol=1e-8)
        h.close()
        assert st.iterations == r.iterations and torch.equal(x, r.x)
