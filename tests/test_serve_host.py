"""Host-side scheduling of the serving layer, without a GPU.

The device hooks of Server are replaced by fakes that sleep and record how
many requests run at once; failures are injected on the host (a request that
raises, a worker that dies), never on a GPU.
"""
import threading
import time

import numpy as np
import pytest

from paper_1906_01211_gb300.serve import Server, estimate_bytes, percentile, request_stream
from paper_1906_01211_gb300.synth import make_waters


class FakeServer(Server):
    def __init__(self, *a, work_s=0.02, **kw):
        self.work_s = work_s
        self.lock = threading.Lock()
        self.now_running = 0
        self.max_running = 0
        self.order = []
        super().__init__(*a, **kw)

    def _create_stream(self):
        return None

    def _bind_thread(self):
        pass

    def _execute(self, slot, req, res):
        if req.system.alpha.min() <= 0:
            raise ValueError("alpha must be > 0 for every site")
        if req.key == "kill-worker":
            raise SystemExit("injected worker death")
        with self.lock:
            self.now_running += 1
            self.max_running = max(self.max_running, self.now_running)
            self.order.append(req.rid)
        time.sleep(self.work_s)
        with self.lock:
            self.now_running -= 1
        res.energy = float(req.system.n)


def small(nw=8, seed=0, periodic=True):
    return make_waters(nw, 10.0 if periodic else 8.0, seed, periodic=periodic)


def test_all_requests_complete_and_overlap():
    srv = FakeServer(n_slots=4, mem_budget_bytes=1 << 40)
    ids = [srv.submit(small(seed=k)) for k in range(16)]
    res = [srv.result(i, timeout=10) for i in ids]
    assert all(r.ok for r in res)
    assert srv.max_running > 1  # requests ran concurrently
    assert srv.stats()["done"] == 16
    srv.close()


def test_memory_budget_limits_concurrency():
    sysm = small()
    est = estimate_bytes(sysm, "mixed")
    srv = FakeServer(n_slots=4, mem_budget_bytes=2 * est + est // 2)
    ids = [srv.submit(small(seed=k)) for k in range(10)]
    assert all(srv.result(i, timeout=10).ok for i in ids)
    assert srv.max_running == 2
    srv.close()


def test_oversize_request_is_refused_and_others_run():
    sysm = small()
    est = estimate_bytes(sysm, "mixed")
    srv = FakeServer(n_slots=2, mem_budget_bytes=est)
    big = srv.submit(make_waters(200, 20.0, 1))
    ok = srv.submit(sysm)
    r = srv.result(big, timeout=5)
    assert not r.ok and "memory budget" in r.error
    assert srv.result(ok, timeout=5).ok
    srv.close()


def test_cancel_queued_request():
    srv = FakeServer(n_slots=1, mem_budget_bytes=1 << 40, work_s=0.2)
    first = srv.submit(small(seed=1))
    time.sleep(0.05)
    queued = srv.submit(small(seed=2))
    assert srv.cancel(queued)
    assert not srv.cancel(first)  # already running
    assert srv.result(queued, timeout=5).error == "cancelled"
    assert srv.result(first, timeout=5).ok
    srv.close()


def test_bad_request_fails_alone():
    bad = small(seed=3)
    bad.alpha = bad.alpha.copy()
    bad.alpha[0] = 0.0
    srv = FakeServer(n_slots=2, mem_budget_bytes=1 << 40)
    ids = [srv.submit(small(seed=4)), srv.submit(bad), srv.submit(small(seed=5))]
    res = [srv.result(i, timeout=5) for i in ids]
    assert res[0].ok and res[2].ok
    assert not res[1].ok and "alpha" in res[1].error
    srv.close()


def test_dead_worker_is_reported_and_others_continue():
    srv = FakeServer(n_slots=2, mem_budget_bytes=1 << 40)
    killer = srv.submit(small(seed=6), key="kill-worker")
    r = srv.result(killer, timeout=5)
    assert not r.ok and "worker died" in r.error
    time.sleep(0.05)
    assert list(srv.health().values()).count(False) == 1
    ids = [srv.submit(small(seed=7 + k)) for k in range(4)]
    assert all(srv.result(i, timeout=10).ok for i in ids)
    srv.close()


def test_request_stream_is_seeded_and_mixed():
    a = request_stream(40, seed=4)
    b = request_stream(40, seed=4)
    assert [s.n for s in a] == [s.n for s in b]
    assert np.array_equal(a[5].xyz, b[5].xyz)
    sizes = np.array([s.n // 3 for s in a])
    assert sizes.min() >= 64 and sizes.max() <= 4096
    kinds = [s.box is None for s in a]
    assert 0 < sum(kinds) < len(kinds)


def test_percentile():
    xs = list(range(1, 101))
    assert percentile(xs, 50) == 50 and percentile(xs, 99) == 99 and percentile(xs, 100) == 100
    with pytest.raises(TypeError):
        percentile(None, 50)
