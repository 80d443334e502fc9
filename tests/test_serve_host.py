"""Request loop logic on the CPU: the scheduling of `serve.Server.run`
(admission in arrival order, setup slots, stream slots, memory budget,
release of finished requests) with the setup and the device solve replaced
by fakes, so that no GPU is involved.  The GPU tests run the real loop."""
import threading
import time

import numpy as np

from paper_1904_03317_gb300 import gmg as G
from paper_1904_03317_gb300 import inputs, serve


class _FakeStream:
    cuda_stream = 0


class _FakeTorch:
    class cuda:
        Stream = staticmethod(lambda device=0: _FakeStream())


class _Info:
    device_bytes = 1000


class _FakeHier:
    """A solve that becomes ready `solve_s` seconds after it was enqueued."""

    def __init__(self, n, solve_s, log, rid):
        self.n, self.info, self.solve_s, self.log, self.rid = n, _Info(), solve_s, log, rid
        self.t_ready = None

    def solve_async(self, b, x, tol):
        self.t_ready = time.perf_counter() + self.solve_s
        self.log.append(("enqueue", self.rid, time.perf_counter()))

    def solve_poll(self, wait):
        ready = time.perf_counter() >= self.t_ready
        st = G.StatsC()
        st.iterations, st.converged = 7, 1
        return ready, st, G.OK

    def close(self):
        self.log.append(("close", self.rid, time.perf_counter()))


class _FakeServer(serve.Server):
    def __init__(self, setup_s=0.01, solve_s=0.02, **kw):
        super().__init__(_FakeTorch, mem_budget=kw.pop("mem_budget", 1e30), **kw)
        self.setup_s, self.solve_s = setup_s, solve_s
        self.log = []
        self.live_setups = 0
        self.max_live_setups = 0
        self.lock = threading.Lock()

    def _setup(self, req_id, w, stream, t0):
        with self.lock:
            self.live_setups += 1
            self.max_live_setups = max(self.max_live_setups, self.live_setups)
        time.sleep(self.setup_s)
        with self.lock:
            self.live_setups -= 1
        h = _FakeHier(1000 + req_id, self.solve_s, self.log, req_id)
        return None, None, h, None, None, time.perf_counter() - t0


def _requests(n, rate):
    return inputs.serving_requests(n, n_min=1e4, n_max=5e4, rate=rate)


def test_every_request_served_once_after_its_arrival():
    arrivals, ws = _requests(12, rate=400.0)
    srv = _FakeServer(setup_workers=3, max_live=4)
    res = srv.run(arrivals, ws)
    assert [r.rid for r in res] == list(range(12))
    for r, a in zip(res, arrivals):
        assert r.status == G.OK and r.converged and r.iterations == 7 and r.n == 1000 + r.rid
        assert a - 1e-9 <= r.admitted <= r.setup_done <= r.ready
    closes = [e[1] for e in srv.log if e[0] == "close"]
    assert sorted(closes) == list(range(12))  # every hierarchy released exactly once
    assert srv.max_live_setups <= 3


def test_admission_in_arrival_order():
    arrivals, ws = _requests(10, rate=2000.0)
    srv = _FakeServer(setup_workers=2, max_live=3, setup_s=0.005, solve_s=0.01)
    res = srv.run(arrivals, ws)
    order = np.argsort(arrivals, kind="stable")
    admitted = [res[i].admitted for i in order]
    assert all(a <= b + 1e-9 for a, b in zip(admitted, admitted[1:]))


def test_stream_slots_bound_requests_in_the_system():
    arrivals, ws = _requests(10, rate=1e6)  # all at once
    srv = _FakeServer(setup_workers=4, max_live=2, setup_s=0.002, solve_s=0.03)
    res = srv.run(arrivals, ws)
    spans = sorted((r.admitted, r.ready) for r in res)
    for t, _ in spans:
        in_system = sum(1 for a, e in spans if a <= t + 1e-9 and e > t + 1e-9)
        assert in_system <= 2


def test_memory_budget_serialises_admissions():
    arrivals, ws = _requests(6, rate=1e6)
    smallest = serve.BYTES_PER_UNKNOWN * 8 * min(serve.Server._leaves_estimate(w) for w in ws)
    srv = _FakeServer(setup_workers=4, max_live=8, mem_budget=1.5 * smallest, setup_s=0.002, solve_s=0.01)
    res = srv.run(arrivals, ws)
    spans = sorted((r.admitted, r.ready) for r in res)
    for (a0, e0), (a1, e1) in zip(spans, spans[1:]):
        assert a1 >= e0 - 1e-6
