"""The serving scheduler on the host, against a simulated engine (no GPU):
admission by footprint never over-commits the budget, slots are never
over-subscribed and a plan never runs two solves at once, admission is first
come first served, requests too big for the budget and malformed meshes are
refused without disturbing the others, and continuous batching overlaps
requests.  Failures are injected on the host."""
import threading
import time
from types import SimpleNamespace

import numpy as np
import pytest

from paper_0908_0673_gb300 import bem, inputs as I
from paper_0908_0673_gb300.serve import EngineError, Request, Server, summarize, synthetic_stream


class FakeEngine:
    """Set-up takes SETUP s per element, each right-hand side SOLVE s per
    element; a plan's real footprint is 0.8 of the estimate."""
    SETUP, SOLVE = 4e-6, 2e-6

    def __init__(self, max_slots=4, budget=10**9):
        self.max_slots = max_slots
        self._budget = budget
        self.lock = threading.Lock()
        self.live = self.max_live = 0
        self.slots = {}
        self.max_used = 0
        self.building = self.max_building = 0

    def estimate(self, req):
        return 1000 * req.mesh.n_nodes

    def budget(self):
        return self._budget

    def build(self, req):
        if np.any(req.mesh.elems < 0) or np.any(req.mesh.elems >= req.mesh.n_nodes):
            raise EngineError(bem.BEM_EINVAL, "element references a missing node")
        with self.lock:
            self.building += 1
            self.max_building = max(self.max_building, self.building)
            self.live += int(0.8 * self.estimate(req))
            self.max_live = max(self.max_live, self.live)
        time.sleep(self.SETUP * req.mesh.n_elems)
        with self.lock:
            self.building -= 1
        return SimpleNamespace(req=req, busy=False)

    def submit(self, h, r):
        assert not h.busy, "a plan runs one solve at a time"
        free = [s for s in range(self.max_slots) if s not in self.slots]
        assert free, "slot over-subscribed"
        h.busy = True
        self.slots[free[0]] = (h, time.perf_counter() + self.SOLVE * h.req.mesh.n_elems)
        self.max_used = max(self.max_used, len(self.slots))
        return free[0]

    def progress(self):
        return sum(1 for _, t in self.slots.values() if time.perf_counter() < t)

    def poll(self, slot):
        h, t = self.slots[slot]
        return (True, (3, 1e-11, bem.BEM_OK)) if time.perf_counter() >= t else (False, None)

    def release(self, slot):
        h, _ = self.slots.pop(slot)
        h.busy = False

    def fetch(self, h):
        return [np.zeros(h.req.mesh.n_nodes)] * len(h.req.rhs)

    def peak(self, h):
        return int(0.8 * self.estimate(h.req))

    def destroy(self, h):
        with self.lock:
            self.live -= int(0.8 * self.estimate(h.req))


def _stream(n, seed=0, gap=0.002):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        m = I.geodesic(int(rng.integers(2, 7)), I.TRI6)
        out.append(Request(i, i * gap, m, bem.BEM_LAPLACE, 0.0, [None] * int(rng.integers(1, 4))))
    return out


def test_budget_slots_and_order():
    reqs = _stream(24)
    budget = 3 * 1000 * max(r.mesh.n_nodes for r in reqs)       # about three plans at once
    eng = FakeEngine(max_slots=4, budget=budget)
    srv = Server(eng, setup_threads=2)
    res = srv.run(reqs)
    assert all(r.status == "ok" for r in res)
    assert srv.max_reserved <= budget and eng.max_live <= budget
    assert eng.max_used <= 4 and eng.max_building <= 2
    adm = [r.admitted_s for r in sorted(res, key=lambda r: r.arrival_s)]
    assert adm == sorted(adm)                                  # first come, first served
    for r in res:
        assert r.arrival_s <= r.admitted_s <= r.ready_s <= r.done_s
        assert len(r.iters) == r.n_rhs
    s = summarize(res)
    assert s["served"] == 24 and s["latency_ms"]["p50"] <= s["latency_ms"]["p99"]


def test_continuous_batching_overlaps():
    reqs = [Request(i, 0.0, I.geodesic(6, I.TRI6), bem.BEM_LAPLACE, 0.0, [None] * 2) for i in range(8)]
    serial = sum(FakeEngine.SETUP * r.mesh.n_elems + FakeEngine.SOLVE * r.mesh.n_elems * 2 for r in reqs)
    eng = FakeEngine(max_slots=4)
    res = Server(eng, setup_threads=4).run(reqs)
    span = max(r.done_s for r in res)
    assert eng.max_used >= 3 and span < 0.7 * serial


def test_refusals_do_not_disturb_others():
    reqs = _stream(6)
    big = I.geodesic(20, I.TRI6)                               # estimate above the whole budget
    bad = I.geodesic(3, I.TRI6)
    bad.elems = bad.elems.copy()
    bad.elems[5, 2] = bad.n_nodes + 7                          # malformed: a missing node
    reqs += [Request(6, 0.001, big, bem.BEM_LAPLACE, 0.0, [None]),
             Request(7, 0.002, bad, bem.BEM_LAPLACE, 0.0, [None])]
    budget = 1000 * 2000
    eng = FakeEngine(budget=budget)
    res = {r.rid: r for r in Server(eng).run(reqs)}
    assert res[6].status == "refused" and "budget" in res[6].error
    assert res[7].status == "error" and "missing node" in res[7].error
    assert all(res[i].status == "ok" for i in range(6))
    assert eng.live == 0                                       # every plan freed


def test_synthetic_stream_shape():
    reqs = synthetic_stream(12, elems=(500, 3000), seed=3)
    t = [r.arrival_s for r in reqs]
    assert t == sorted(t) and t[0] > 0
    for r in reqs:
        assert 1 <= len(r.rhs) <= 8
        assert 300 <= r.mesh.n_elems <= 4000
        assert all(np.shape(c) == r.mesh.elems.shape for c in r.rhs)
        if r.green == bem.BEM_HELMHOLTZ:
            assert 1.0 <= r.k <= 4.0 and np.iscomplexobj(r.rhs[0])
    again = synthetic_stream(12, elems=(500, 3000), seed=3)
    assert [r.mesh.n_elems for r in again] == [r.mesh.n_elems for r in reqs]
