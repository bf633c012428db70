"""Host logic of the serving loop (admission, slots, memory budget, latency
statistics) with a fake executor: CPU only."""
import threading
import time

import pytest

from paper_2601_20758_gb300 import serve


class FakeExecutor:
    def __init__(self, service_s=0.02):
        self.service_s = service_s
        self.lock = threading.Lock()
        self.running = 0
        self.max_running = 0
        self.order = []

    def workspace(self, req):
        g = int(req.dims[0]) * int(req.dims[1]) * int(req.dims[2])
        return 20 * g

    def run(self, req, slot):
        with self.lock:
            self.running += 1
            self.max_running = max(self.max_running, self.running)
            self.order.append(req.rid)
        time.sleep(self.service_s)
        with self.lock:
            self.running -= 1
        return {"slot": slot}


def _reqs(n, dims=(16, 16, 16), gap=0.0):
    return [serve.Request(rid=i, lo=(0, 0, 0), hi=(1, 1, 1), dims=dims, arrival=i * gap)
            for i in range(n)]


def test_slots_bound_concurrency_and_admission_is_fifo():
    ex = FakeExecutor(0.02)
    srv = serve.Server(ex, slots=3, mem_budget=1 << 40)
    try:
        st = srv.replay(_reqs(12))
    finally:
        srv.close()
    assert st["done"] == 12 and st["errors"] == 0
    assert ex.max_running <= 3 and srv.max_concurrent == 3
    adm = [r.admitted for r in sorted(srv.completed, key=lambda r: r.rid)]
    assert adm == sorted(adm)                    # admitted in arrival order
    assert st["p99_ms"] >= st["p50_ms"] >= 20.0 * 0.9


def test_memory_budget_limits_admission_and_rejects_oversize():
    small = serve.Request(rid=0, lo=(0, 0, 0), hi=(1, 1, 1), dims=(32, 32, 32))
    ex = FakeExecutor(0.02)
    need = ex.workspace(small)
    srv = serve.Server(ex, slots=8, mem_budget=2 * need + need // 2)
    try:
        reqs = [serve.Request(rid=i, lo=(0, 0, 0), hi=(1, 1, 1), dims=(32, 32, 32)) for i in range(6)]
        huge = serve.Request(rid=99, lo=(0, 0, 0), hi=(1, 1, 1), dims=(512, 512, 512))
        st = srv.replay(reqs + [huge])
    finally:
        srv.close()
    assert st["done"] == 6 and st["rejected"] == 1
    assert ex.max_running <= 2                   # two fit in the budget, never three
    assert srv.max_bytes <= 2 * need + need // 2


def test_navigation_stream_is_seeded_and_in_the_unit_cube():
    a = serve.navigation_requests(200, rate=200.0, centre=(0.3, 0.4, 0.5), seed=5)
    b = serve.navigation_requests(200, rate=200.0, centre=(0.3, 0.4, 0.5), seed=5)
    assert [(r.lo, r.hi, r.dims, r.arrival) for r in a] == [(r.lo, r.hi, r.dims, r.arrival) for r in b]
    for r in a:
        e = r.hi[0] - r.lo[0]
        assert 1e-3 * 0.999 <= e <= 1.0 + 1e-12
        assert all(0.0 - 1e-12 <= v <= 1.0 + 1e-12 for v in r.lo + r.hi)
        assert r.dims[0] in (64, 96, 128, 192, 256)
    gaps = [y.arrival - x.arrival for x, y in zip(a, a[1:])]
    assert sum(gaps) / len(gaps) == pytest.approx(1 / 200.0, rel=0.25)
    assert not any(r.want_points for r in a)      # view changes recompute the grid only
    c = serve.navigation_requests(200, rate=200.0, centre=(0.3, 0.4, 0.5), seed=5, select_every=10)
    assert [r.want_points for r in c] == [i % 10 == 0 for i in range(200)]
    assert [(r.lo, r.dims) for r in c] == [(r.lo, r.dims) for r in a]


def test_percentile_nearest_rank():
    assert serve.percentile([5, 1, 4, 2, 3], 50) == 3
    assert serve.percentile([5, 1, 4, 2, 3], 99) == 5
    assert serve.percentile([], 50) is None


def test_workers_are_fixed_per_slot():
    """Each slot is served by one long-lived worker thread (no thread per request)."""
    seen = {}

    class Ex(FakeExecutor):
        def run(self, req, slot):
            seen.setdefault(slot, set()).add(threading.get_ident())
            return super().run(req, slot)

    ex = Ex(0.005)
    srv = serve.Server(ex, slots=2, mem_budget=1 << 40)
    try:
        st = srv.replay(_reqs(20))
    finally:
        srv.close()
    assert st["done"] == 20
    assert all(len(v) == 1 for v in seen.values()) and len(seen) == 2


def test_a_request_whose_workspace_query_fails_errors_alone():
    class Ex(FakeExecutor):
        def workspace(self, req):
            if req.rid == 3:
                raise ValueError("bad ROI")
            return super().workspace(req)

    ex = Ex(0.002)
    srv = serve.Server(ex, slots=2, mem_budget=1 << 40)
    try:
        st = srv.replay(_reqs(6))
    finally:
        srv.close()
    assert st["done"] == 5 and st["errors"] == 1


def test_bf16_share_is_seeded_and_leaves_the_walk_alone():
    a = serve.navigation_requests(400, rate=200.0, centre=(0.5, 0.5, 0.5), seed=9)
    b = serve.navigation_requests(400, rate=200.0, centre=(0.5, 0.5, 0.5), seed=9, bf16_share=0.3)
    assert [(r.lo, r.dims, r.arrival) for r in a] == [(r.lo, r.dims, r.arrival) for r in b]
    share = sum(r.prec == "bf16" for r in b) / len(b)
    assert 0.24 < share < 0.36 and all(r.prec == "fp32" for r in a)


def test_supersede_drops_waiting_views_of_the_same_client_only():
    """Recompute trigger: with one slot busy, requests of client 0 arriving while
    it runs replace each other in the queue (only the newest is computed); a
    request of client 1 waiting at the same time is kept."""
    ex = FakeExecutor(0.05)
    srv = serve.Server(ex, slots=1, mem_budget=1 << 40, supersede=True)
    try:
        reqs = [serve.Request(rid=i, lo=(0, 0, 0), hi=(1, 1, 1), dims=(8, 8, 8), arrival=0.002 * i,
                              client=0) for i in range(6)]
        reqs.append(serve.Request(rid=100, lo=(0, 0, 0), hi=(1, 1, 1), dims=(8, 8, 8), arrival=0.003,
                                  client=1))
        st = srv.replay(reqs)
    finally:
        srv.close()
    by = {r.rid: r.status for r in srv.completed}
    assert by[0] == "done"                      # admitted at once
    assert by[5] == "done" and by[100] == "done"
    assert all(by[i] == "superseded" for i in range(1, 5))
    assert st["superseded"] == 4 and st["done"] == 3
    assert ex.order == [0, 100, 5] or ex.order == [0, 5, 100]
    # without the trigger every request is computed, in arrival order
    ex2 = FakeExecutor(0.01)
    srv2 = serve.Server(ex2, slots=1, mem_budget=1 << 40)
    try:
        st2 = srv2.replay([serve.Request(rid=i, lo=(0, 0, 0), hi=(1, 1, 1), dims=(8, 8, 8),
                                         arrival=0.001 * i) for i in range(5)])
    finally:
        srv2.close()
    assert st2["done"] == 5 and st2["superseded"] == 0 and ex2.order == list(range(5))
