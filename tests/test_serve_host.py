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
    def __init__(self, device_bytes):
        self.device_bytes = device_bytes


class _FakeHier:
    """A solve that becomes ready `solve_s` seconds after it was enqueued."""

    def __init__(self, n, device_bytes, solve_s, log, key):
        self.n, self.info, self.solve_s, self.log, self.key = n, _Info(device_bytes), solve_s, log, key
        self.t_ready = None

    def solve_async(self, b, x, tol):
        self.t_ready = time.perf_counter() + self.solve_s
        self.log.append(("enqueue", self.key, time.perf_counter()))

    def solve_poll(self, wait):
        ready = time.perf_counter() >= self.t_ready
        st = G.StatsC()
        st.iterations, st.converged = 7, 1
        return ready, st, G.OK

    def close(self):
        self.log.append(("close", self.key, time.perf_counter()))


def _rid(w):
    return int(w.name.split("_")[0][len("request"):])


class _FakeServer(serve.Server):
    """The real scheduling with the setup phases replaced: request i has
    1000 + i leaves and its hierarchy `bytes_per_leaf` device bytes per leaf;
    requests with the same name have the same mesh."""

    def __init__(self, setup_s=0.01, solve_s=0.02, bytes_per_leaf=100.0, **kw):
        super().__init__(_FakeTorch, mem_budget=kw.pop("mem_budget", 1e30), **kw)
        self.setup_s, self.solve_s, self.bpl = setup_s, solve_s, bytes_per_leaf
        self.log = []
        self.live_setups = 0
        self.max_live_setups = 0
        self.builds = 0
        self.lock = threading.Lock()

    def _busy(self, dt):
        with self.lock:
            self.live_setups += 1
            self.max_live_setups = max(self.max_live_setups, self.live_setups)
        time.sleep(dt)
        with self.lock:
            self.live_setups -= 1

    def _mesh(self, w, t0):
        self._busy(self.setup_s / 2)
        return None, 1000 + _rid(w), w.name.encode(), time.perf_counter() - t0

    def _hierarchy(self, w, m, stream, t0):
        self._busy(self.setup_s / 2)
        with self.lock:
            self.builds += 1
        leaves = 1000 + _rid(w)
        return None, _FakeHier(leaves, self.bpl * leaves - 16.0 * leaves, self.solve_s, self.log, w.name), \
            time.perf_counter() - t0

    def _vectors(self, w, h, stream):
        return None, None


def _requests(n, rate):
    return inputs.serving_requests(n, n_min=1e4, n_max=5e4, rate=rate)


def test_every_request_served_once_after_its_arrival():
    arrivals, ws = _requests(12, rate=400.0)
    srv = _FakeServer(setup_workers=3, max_live=4)
    res = srv.run(arrivals, ws)
    assert [r.rid for r in res] == list(range(12))
    for r, a in zip(res, arrivals):
        assert r.status == G.OK and r.converged and r.iterations == 7 and r.n == 1000 + r.rid
        assert a - 1e-9 <= r.admitted <= r.meshed <= r.hier_start <= r.setup_done <= r.ready
    closes = [e[1] for e in srv.log if e[0] == "close"]
    assert sorted(closes) == sorted(w.name for w in ws)  # every hierarchy released exactly once
    assert srv.max_live_setups <= 3 and srv.builds == 12 and srv.cache_hits == 0


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


def test_memory_budget_serialises_hierarchies():
    """A budget below any two hierarchies: once the first hierarchy has been
    measured, the next one is built only after the previous result (and its
    cached hierarchy, evicted to make room) has freed the memory."""
    arrivals, ws = _requests(6, rate=1e6)
    srv = _FakeServer(setup_workers=4, max_live=8, mem_budget=1.5 * 100.0 * 1000, setup_s=0.002, solve_s=0.01)
    srv.bytes_per_leaf = 100.0  # the initial prediction equals the measured size here
    res = srv.run(arrivals, ws)
    assert all(r.status == G.OK for r in res)
    spans = sorted((r.hier_start, r.ready) for r in res)
    for (a0, e0), (a1, e1) in zip(spans, spans[1:]):
        assert a1 >= e0 - 1e-6


def test_prediction_learns_from_measured_hierarchies():
    """The first hierarchies are admitted with the initial bytes-per-leaf
    guess; after a measurement the prediction is the measured ratio (with
    margin), so a budget that fits two measured hierarchies runs two at once."""
    arrivals, ws = _requests(8, rate=1e6)
    srv = _FakeServer(setup_workers=4, max_live=8, bytes_per_leaf=300.0, mem_budget=2.2 * 300.0 * 1010,
                      setup_s=0.004, solve_s=0.03)
    res = srv.run(arrivals, ws)
    assert all(r.status == G.OK for r in res)
    assert abs(srv.bytes_per_leaf - 1.05 * 300.0) < 1e-9
    spans = sorted((r.hier_start, r.ready) for r in res)
    most = max(sum(1 for a, e in spans if a <= t + 1e-9 and e > t + 1e-9) for t, _ in spans)
    assert most == 2


def test_identical_meshes_reuse_the_cached_hierarchy():
    """Requests whose meshes are identical (same key) after the first one has
    finished take its idle hierarchy from the cache: no second build, and the
    hierarchy is released once at the end."""
    arrivals, ws = _requests(3, rate=1e6)
    ws = [ws[0]] * 3
    arrivals = np.array([0.0, 0.2, 0.4])
    srv = _FakeServer(setup_workers=2, max_live=4, setup_s=0.004, solve_s=0.01)
    res = srv.run(arrivals, ws)
    assert all(r.status == G.OK for r in res)
    assert srv.builds == 1 and srv.cache_hits == 2
    assert [r.cache_hit for r in res] == [False, True, True]
    assert sum(1 for e in srv.log if e[0] == "close") == 1
