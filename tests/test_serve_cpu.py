"""Scheduling policy of the continuous-batching server, on CPU with a fake
backend: device-memory admission, slots, arrival order, rejection of requests
that can never fit, cancellation (pending, preparing, active), failures of a
request's creation, latency bookkeeping, joins between batch calls without a
rebuild, and host work (creation, read-back) overlapping batch calls on worker
threads."""
import dataclasses
import threading
import time

import numpy as np
import pytest

from paper_0901_1053_gb300.serve import Server, latency_stats


@dataclasses.dataclass
class W:
    cells: int
    steps: int
    bad: bool = False


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class FakeBackend:
    """A slot table: each batch call costs 1 ms of fake time per step and
    member; joins and leaves are recorded."""

    def __init__(self, clock, fail_create=()):
        self.clock = clock
        self.live = set()
        self.members = []
        self.fail_create = set(fail_create)
        self.rounds = []       # members per batch call
        self.joins = []        # (call index, members after the join)
        self.leaves = 0

    def bytes_needed(self, w):
        if w.bad:
            raise ValueError("malformed geometry")
        return w.cells

    def prepare(self, w):
        if id(w) in self.fail_create:
            raise RuntimeError("out of memory")
        h = {"w": w, "step": 0, "limit": None}
        self.live.add(id(h))
        return h

    def join(self, h, limit):
        assert h not in self.members
        h["limit"] = limit
        self.members.append(h)
        self.joins.append((len(self.rounds), len(self.members)))

    def advance(self, n):
        self.rounds.append(len(self.members))
        for h in self.members:
            h["step"] = min(h["limit"], h["step"] + n)
        self.clock.t += 1e-3 * n * len(self.members)

    def throttle(self, max_pending):
        return 0.0

    def step_of(self, h):
        return h["step"]

    def leave(self, h):
        self.members.remove(h)
        self.leaves += 1

    def finish(self, h):
        return np.full(3, float(h["w"].cells)), 0.0, 1e-3

    def release(self, h):
        self.live.discard(id(h))


def make(budget=100, slots=4, round_steps=10):
    clk = FakeClock()
    be = FakeBackend(clk)
    return Server(be, hbm_budget=budget, max_slots=slots, round_steps=round_steps, workers=0, clock=clk,
                  sleep=clk.sleep), be, clk


def run(srv):
    while not srv.idle():
        srv.round()


def test_budget_and_slots_bound_the_active_set():
    srv, be, clk = make(budget=100, slots=3)
    for rid, cells in enumerate([40, 40, 30, 10, 10]):
        srv.submit(rid, W(cells, 25))
    srv.round()
    assert sorted(srv.active) == [0, 1]          # 40 + 40 + 30 > 100: request 2 waits ...
    assert [p[0] for p in srv.pending] == [2, 3, 4]   # ... and nobody overtakes it
    run(srv)
    assert all(r.status == "ok" for r in srv.results.values())
    assert max(be.rounds) <= 3
    assert not be.live and not be.members and srv.used == 0


def test_request_larger_than_the_budget_is_rejected_at_once():
    srv, be, clk = make(budget=100)
    srv.submit(0, W(101, 5))
    srv.submit(1, W(50, 5))
    assert srv.results[0].status == "rejected"
    run(srv)
    assert srv.results[1].status == "ok"


def test_cancel_pending_and_active():
    srv, be, clk = make(budget=100, slots=1)
    srv.submit(0, W(10, 100))
    srv.submit(1, W(10, 100))
    srv.round()                 # 0 active, 1 pending
    srv.cancel(0)
    srv.cancel(1)
    srv.round()
    srv.round()
    assert srv.results[0].status == "cancelled" and srv.results[1].status == "cancelled"
    assert srv.idle() and not be.live and srv.used == 0 and not be.members


def test_malformed_and_failed_creation_are_reported():
    srv, be, clk = make()
    good = W(10, 5)
    failing = W(10, 5)
    be.fail_create.add(id(failing))
    srv.submit(0, W(10, 5, bad=True))
    srv.submit(1, failing)
    srv.submit(2, good)
    run(srv)
    assert srv.results[0].status == "error" and "malformed" in srv.results[0].error
    assert srv.results[1].status == "error" and "memory" in srv.results[1].error
    assert srv.results[2].status == "ok"
    assert srv.used == 0


def test_members_join_and_leave_between_calls():
    """Short requests leave after the call that finishes them while a long one
    keeps running; newcomers join the running batch (no rebuild: the backend
    sees single joins and leaves)."""
    srv, be, clk = make(budget=1000, slots=4, round_steps=10)
    srv.submit(0, W(10, 100))
    srv.round()
    for rid in range(1, 4):
        srv.submit(rid, W(10, 15))
    run(srv)
    assert all(srv.results[r].status == "ok" for r in range(4))
    assert be.leaves == 4 and len(be.joins) == 4
    assert be.joins[0] == (0, 1) and all(c >= 1 for c, _ in be.joins[1:])  # joined while 0 ran
    # request 0 ran alone again once the short ones (2 calls each) had left
    assert be.rounds[:3] == [1, 4, 4] and be.rounds[-1] == 1


def test_stream_latencies_and_continuous_admission():
    srv, be, clk = make(budget=1000, slots=8, round_steps=10)

    @dataclasses.dataclass
    class Req:
        rid: int
        arrival: float

    reqs = [Req(i, 0.005 * i) for i in range(20)]
    res = srv.run_stream(reqs, lambda r: W(50, 30))
    st = latency_stats(res)
    assert st["ok"] == 20 and st["p99_s"] >= st["p50_s"] > 0
    assert all(r.t_done >= r.t_arrival for r in res.values())
    # requests that arrived while others ran joined running batches
    assert max(be.rounds) > 1 and srv.max_active > 1


class SlowBackend(FakeBackend):
    """Real time: creation and read-back take 20 ms each on the calling thread;
    a batch call takes 5 ms. Records which threads did what and when."""

    def __init__(self):
        super().__init__(clock=None)
        self.events = []
        self.lock = threading.Lock()

    def _log(self, what):
        with self.lock:
            self.events.append((what, threading.get_ident(), time.perf_counter()))

    def prepare(self, w):
        self._log("prepare0")
        time.sleep(0.02)
        h = super().prepare(w)
        self._log("prepare1")
        return h

    def advance(self, n):
        self._log("advance0")
        self.rounds.append(len(self.members))
        for h in self.members:
            h["step"] = min(h["limit"], h["step"] + n)
        time.sleep(0.005)
        self._log("advance1")

    def finish(self, h):
        time.sleep(0.02)
        self._log("finish")
        return super().finish(h)


def test_host_work_overlaps_batch_calls_on_worker_threads():
    be = SlowBackend()
    srv = Server(be, hbm_budget=1000, max_slots=8, round_steps=10, workers=2)

    @dataclasses.dataclass
    class Req:
        rid: int
        arrival: float

    reqs = [Req(i, 0.01 * i) for i in range(12)]
    res = srv.run_stream(reqs, lambda r: W(10, 60))
    srv.close()
    assert all(r.status == "ok" for r in res.values()) and len(res) == 12
    assert not be.live and srv.used == 0
    main = threading.get_ident()
    prep = [(t, tid) for what, tid, t in be.events if what.startswith("prepare")]
    assert all(tid != main for _, tid in prep)                      # creation off the scheduling thread
    assert all(tid != main for what, tid, _ in be.events if what == "finish")
    # some batch call ran while a creation was in progress
    spans = {}
    for what, tid, t in be.events:
        if what.startswith("prepare"):
            spans.setdefault(tid, []).append((what, t))
    opened = []
    for tid, ev in spans.items():
        for (a, t0), (b, t1) in zip(ev[::2], ev[1::2]):
            opened.append((t0, t1))
    calls = [t for what, _, t in be.events if what == "advance0"]
    assert any(t0 < c < t1 for c in calls for t0, t1 in opened)


def test_cancel_while_preparing():
    be = SlowBackend()
    srv = Server(be, hbm_budget=1000, max_slots=2, round_steps=10, workers=1)
    srv.submit(0, W(10, 1000))
    srv.round()                 # preparation started on the worker
    assert srv.preparing
    srv.cancel(0)
    t_end = time.perf_counter() + 5
    while not srv.idle() and time.perf_counter() < t_end:
        srv.round(wait_timeout=0.05)
    srv.close()
    assert srv.results[0].status == "cancelled"
    assert not be.live and not be.members and srv.used == 0
