"""Scheduling policy of the continuous-batching server, on CPU with a fake
backend and a fake clock: device-memory admission, slots, arrival order,
rejection of requests that can never fit, cancellation, failures of a
request's creation, and latency bookkeeping."""
import dataclasses

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
    """Each step of a round costs 1 ms of fake time per active solve."""

    def __init__(self, clock, fail_create=()):
        self.clock = clock
        self.live = set()
        self.fail_create = set(fail_create)
        self.rounds = []

    def bytes_needed(self, w):
        if w.bad:
            raise ValueError("malformed geometry")
        return w.cells

    def create(self, w):
        if id(w) in self.fail_create:
            raise RuntimeError("out of memory")
        h = {"w": w, "step": 0}
        self.live.add(id(h))
        return h

    def advance(self, hs, limits, n):
        self.rounds.append(len(hs))
        for h, lim in zip(hs, limits):
            h["step"] = min(lim, h["step"] + n)
        self.clock.t += 1e-3 * n * len(hs)

    def step_of(self, h):
        return h["step"]

    def finish(self, h):
        return np.full(3, float(h["w"].cells)), 0.0, 1e-3

    def release(self, h):
        self.live.discard(id(h))


def make(budget=100, slots=4, round_steps=10):
    clk = FakeClock()
    be = FakeBackend(clk)
    return Server(be, hbm_budget=budget, max_slots=slots, round_steps=round_steps, clock=clk,
                  sleep=clk.sleep), be, clk


def test_budget_and_slots_bound_the_active_set():
    srv, be, clk = make(budget=100, slots=3)
    for rid, cells in enumerate([40, 40, 30, 10, 10]):
        srv.submit(rid, W(cells, 25))
    srv.round()
    assert sorted(srv.active) == [0, 1]          # 40 + 40 + 30 > 100: request 2 waits ...
    assert [p[0] for p in srv.pending] == [2, 3, 4]   # ... and nobody overtakes it
    while not srv.idle():
        srv.round()
    assert all(r.status == "ok" for r in srv.results.values())
    assert max(be.rounds) <= 3
    assert not be.live


def test_request_larger_than_the_budget_is_rejected_at_once():
    srv, be, clk = make(budget=100)
    srv.submit(0, W(101, 5))
    srv.submit(1, W(50, 5))
    assert srv.results[0].status == "rejected"
    while not srv.idle():
        srv.round()
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
    assert srv.idle() and not be.live and srv.used == 0


def test_malformed_and_failed_creation_are_reported():
    srv, be, clk = make()
    good = W(10, 5)
    failing = W(10, 5)
    be.fail_create.add(id(failing))
    srv.submit(0, W(10, 5, bad=True))
    srv.submit(1, failing)
    srv.submit(2, good)
    while not srv.idle():
        srv.round()
    assert srv.results[0].status == "error" and "malformed" in srv.results[0].error
    assert srv.results[1].status == "error" and "memory" in srv.results[1].error
    assert srv.results[2].status == "ok"
    assert srv.used == 0


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
    # requests that arrived while others ran joined running rounds
    assert max(be.rounds) > 1 and srv.max_active > 1
