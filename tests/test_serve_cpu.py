"""Host logic of the serving loop, driven by a fake executor on the CPU: every request resolves,
the HBM budget and the slot count are never exceeded, idle designs are evicted least recently
used first, a design runs one request at a time, and failures stay with their request."""
import threading
import time

import numpy as np
import pytest

from paper_2002_07627_gb300.serve import DesignSpec, ImfServer
from paper_2002_07627_gb300 import synth


class FakeExecutor:
    def __init__(self, sizes, duration=0.002, fail_on=None):
        self.sizes = sizes
        self.duration = duration
        self.fail_on = fail_on or set()
        self.lock = threading.Lock()
        self.resident = {}
        self.running = set()
        self.max_bytes = 0
        self.max_running = 0
        self.created = []
        self.destroyed = []
        self.calls = 0

    def footprint(self, spec):
        return self.sizes[spec.fixture]        # the fixture slot carries the fake design id

    def create(self, design_id, spec):
        with self.lock:
            self.resident[design_id] = self.footprint(spec)
            self.max_bytes = max(self.max_bytes, sum(self.resident.values()))
            self.created.append(design_id)
        return {"id": design_id}

    def destroy(self, st):
        with self.lock:
            self.resident.pop(st["id"])
            self.destroyed.append(st["id"])

    def launch(self, st, rho, slot):
        with self.lock:
            self.calls += 1
            assert st["id"] not in {r[0] for r in self.running}, "two requests of one design in flight"
            self.running.add((st["id"], slot))
            self.max_running = max(self.max_running, len(self.running))
        if float(rho.ravel()[0]) in self.fail_on:
            with self.lock:
                self.running.discard((st["id"], slot))
            raise RuntimeError("injected launch failure")
        return (st["id"], slot, time.perf_counter() + self.duration, rho)

    def done(self, tok):
        return time.perf_counter() >= tok[2]

    def result(self, tok):
        with self.lock:
            self.running.discard((tok[0], tok[1]))
        return tok[0], float(tok[3].sum())


def _spec(i):
    tool = synth.planar_tool(n_orient=2)
    return DesignSpec((1, 4, 4), [tool], fixture=i)


def test_all_requests_resolve_within_budget_and_slots():
    sizes = {i: 30 for i in range(6)}
    ex = FakeExecutor(sizes)
    srv = ImfServer(ex, hbm_budget=100, slots=3)
    for i in range(6):
        srv.register(i, _spec(i))
    futs = []
    rng = np.random.default_rng(0)
    for k in range(120):
        d = int(rng.integers(0, 6))
        futs.append((d, k, srv.submit(d, np.full((1, 4, 4), k, np.float32))))
    for d, k, f in futs:
        did, s = f.result(timeout=30)
        assert did == d and s == 16 * k
    srv.close()
    assert ex.max_bytes <= 100
    assert ex.max_running <= 3
    assert srv.stats.completed == 120 and srv.stats.failed == 0
    assert srv.stats.evictions > 0          # 6 x 30 bytes cannot all be resident under 100
    assert len(srv.stats.latencies) == 120


def test_lru_eviction_order():
    sizes = {0: 40, 1: 40, 2: 40}
    ex = FakeExecutor(sizes, duration=0.0)
    srv = ImfServer(ex, hbm_budget=80, slots=1)
    for i in range(3):
        srv.register(i, _spec(i))
    for d in (0, 1, 0):
        srv.submit(d, np.zeros((1, 4, 4), np.float32)).result(timeout=10)
    srv.submit(2, np.zeros((1, 4, 4), np.float32)).result(timeout=10)
    srv.close()
    assert ex.destroyed[0] == 1              # design 1 was used least recently


def test_failures_stay_with_their_request():
    ex = FakeExecutor({0: 10, 1: 10}, fail_on={7.0})
    srv = ImfServer(ex, hbm_budget=100, slots=2)
    srv.register(0, _spec(0))
    srv.register(1, _spec(1))
    ok = srv.submit(0, np.full((1, 4, 4), 1, np.float32))
    bad = srv.submit(1, np.full((1, 4, 4), 7, np.float32))
    ok2 = srv.submit(1, np.full((1, 4, 4), 2, np.float32))
    assert ok.result(timeout=10)[1] == 16
    with pytest.raises(RuntimeError, match="injected"):
        bad.result(timeout=10)
    assert ok2.result(timeout=10)[1] == 32
    unknown = srv.submit(9, np.zeros((1, 4, 4), np.float32))
    with pytest.raises(KeyError):
        unknown.result(timeout=1)
    srv.close()
    assert srv.stats.failed == 1


def test_design_above_budget_is_rejected_not_hung():
    ex = FakeExecutor({0: 500})
    srv = ImfServer(ex, hbm_budget=100, slots=2)
    srv.register(0, _spec(0))
    with pytest.raises(MemoryError):
        srv.submit(0, np.zeros((1, 4, 4), np.float32)).result(timeout=10)
    srv.close()


def test_requests_of_one_design_run_in_order():
    ex = FakeExecutor({0: 10}, duration=0.001)
    srv = ImfServer(ex, hbm_budget=100, slots=4)
    srv.register(0, _spec(0))
    futs = [srv.submit(0, np.full((1, 4, 4), k, np.float32)) for k in range(20)]
    done = [f.result(timeout=10)[1] for f in futs]
    srv.close()
    assert done == [16 * k for k in range(20)]
    assert ex.max_running == 1


class FakeCtxExecutor(FakeExecutor):
    """A fake executor that can add contexts to a resident design (each a further concurrent
    request of that design), costing `ctx_size` bytes each."""

    def __init__(self, sizes, ctx_size, duration=0.003):
        super().__init__(sizes, duration)
        self.ctx_size = ctx_size
        self.ctxs = {}
        self.max_ctx_running = 0

    def context_footprint(self, spec):
        return self.ctx_size

    def create(self, design_id, spec):
        st = super().create(design_id, spec)
        self.ctxs[design_id] = 1
        return st

    def add_context(self, st):
        with self.lock:
            self.ctxs[st["id"]] += 1
            self.resident[st["id"]] += self.ctx_size
            self.max_bytes = max(self.max_bytes, sum(self.resident.values()))

    def destroy(self, st):
        super().destroy(st)
        self.ctxs.pop(st["id"], None)

    def launch(self, st, rho, slot, ctx=0):
        with self.lock:
            self.calls += 1
            key = (st["id"], ctx)
            assert key not in {(r[0], r[2]) for r in self.running}, "one context runs one request"
            assert ctx < self.ctxs[st["id"]]
            self.running.add((st["id"], slot, ctx))
            self.max_running = max(self.max_running, len(self.running))
            per = sum(1 for r in self.running if r[0] == st["id"])
            self.max_ctx_running = max(self.max_ctx_running, per)
        return (st["id"], slot, time.perf_counter() + self.duration, rho, ctx)

    def result(self, tok):
        with self.lock:
            self.running.discard((tok[0], tok[1], tok[4]))
        return tok[0], float(tok[3].sum())


def test_several_requests_of_one_design_run_on_their_own_contexts():
    """With an executor that can add contexts, up to max_inflight requests of one design run at
    once (each on its own context), the budget counts every context, every result is right, and
    a context that does not fit the budget is not added (the request waits instead)."""
    ex = FakeCtxExecutor({0: 30, 1: 30}, ctx_size=10)
    srv = ImfServer(ex, hbm_budget=100, slots=4, max_inflight=3)
    srv.register(0, _spec(0))
    srv.register(1, _spec(1))
    futs = [(k, srv.submit(k % 2, np.full((1, 4, 4), k, np.float32))) for k in range(40)]
    for k, f in futs:
        did, s = f.result(timeout=30)
        assert did == k % 2 and s == 16 * k
    srv.close()
    assert ex.max_ctx_running >= 2 and ex.max_ctx_running <= 3
    assert ex.max_bytes <= 100
    assert srv.stats.max_contexts <= 3
    # a budget with no room for a second context keeps one request per design in flight
    ex = FakeCtxExecutor({0: 95}, ctx_size=10)
    srv = ImfServer(ex, hbm_budget=100, slots=4, max_inflight=3)
    srv.register(0, _spec(0))
    futs = [srv.submit(0, np.full((1, 4, 4), k, np.float32)) for k in range(8)]
    assert [f.result(timeout=30)[1] for f in futs] == [16 * k for k in range(8)]
    srv.close()
    assert ex.max_ctx_running == 1 and ex.max_bytes <= 100


class FakePrioExecutor(FakeExecutor):
    """A fake executor whose first two of four slots are high-priority streams; it records the
    slot priority each design's launches got."""

    def __init__(self, sizes, duration=0.01):
        super().__init__(sizes, duration)
        self.prio_of = {}

    def slot_priority(self, slot):
        return 1 if slot < 2 else 0

    def launch(self, st, rho, slot):
        with self.lock:
            self.prio_of.setdefault(st["id"], set()).add(self.slot_priority(slot))
        return super().launch(st, rho, slot)


def test_small_requests_take_high_priority_slots():
    """With an executor that reports stream priorities, requests of designs no larger than the
    median registered design go to high-priority slots and larger ones to low-priority slots
    whenever a slot of the wanted kind is free; every result is still right."""
    ex = FakePrioExecutor({i: 10 for i in range(4)})
    srv = ImfServer(ex, hbm_budget=1000, slots=4)
    tool = synth.planar_tool(n_orient=2)
    shapes = {0: (1, 4, 4), 1: (1, 4, 4), 2: (1, 12, 12), 3: (1, 12, 12)}
    for i, sh in shapes.items():
        srv.register(i, DesignSpec(sh, [tool], fixture=i))
    assert srv.small_units == 4 * 4 * 2
    # one wave of four requests, one per design, queued while the server loop waits on its lock,
    # so that one admission pass places all four into the four free slots
    from concurrent.futures import Future
    from paper_2002_07627_gb300.serve import _Req
    futs = []
    with srv._lock:
        for i in range(4):
            f = Future()
            srv.pending.append(_Req(i, np.full(shapes[i], i + 1, np.float32), time.perf_counter(), f))
            futs.append((i, f))
        srv._wake.notify()
    for i, f in futs:
        did, s = f.result(timeout=30)
        assert did == i and s == (i + 1) * np.prod(shapes[i])
    srv.close()
    assert ex.prio_of[0] == {1} and ex.prio_of[1] == {1}
    assert ex.prio_of[2] == {0} and ex.prio_of[3] == {0}
