"""Request loop (continuous batching): each request's result in the mix equals
its result when solved alone, and every request is served."""
import numpy as np
import pytest

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


def test_result_alone_equals_result_in_the_mix(torch):
    arrivals, ws = inputs.serving_requests(10, n_min=1e4, n_max=1.5e5, rate=200.0)
    srv = serve.Server(torch, setup_workers=4, max_live=8, vcycle_prec=G.PREC_FP64, keep_x=True)
    res = srv.run(arrivals, ws)
    assert all(r.status == G.OK and r.converged for r in res)
    assert all(r.ready >= r.setup_done >= r.admitted >= r.arrival - 1e-9 for r in res)
    ctx = G.Context(0)
    for r, w in zip(res, ws):
        h = G.Hierarchy(ctx, G.build_mesh(w), w.degree, w.coeff, cheb_degree=w.cheb_degree,
                        vcycle_prec=G.PREC_FP64)
        b = torch.tensor(inputs.random_rhs(w.seed, h.n), dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        st = h.solve(b, x, tol=1e-8)
        assert st.iterations == r.iterations and h.n == r.n
        assert float(torch.linalg.vector_norm(x - r.x) / torch.linalg.vector_norm(x)) <= 1e-11
        h.close()


def test_memory_budget_serialises_admissions(torch):
    arrivals, ws = inputs.serving_requests(6, n_min=1e4, n_max=5e4, rate=1e6)
    # a budget below any two requests' estimates: one request in the system at a
    # time (a request larger than the budget is admitted alone)
    smallest = serve.BYTES_PER_UNKNOWN * 8 * min(serve.Server._leaves_estimate(w) for w in ws)
    srv = serve.Server(torch, mem_budget=1.5 * smallest, setup_workers=4, max_live=8)
    res = srv.run(arrivals, ws)
    assert all(r.status == G.OK for r in res)
    spans = sorted((r.admitted, r.ready) for r in res)
    for (a0, e0), (a1, e1) in zip(spans, spans[1:]):
        assert a1 >= e0 - 1e-6  # the next admission waits for the previous result
