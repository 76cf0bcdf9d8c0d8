"""Continuous-batching server for wakefield solves.

Requests (grid, geometry, bunch) arrive over time. The scheduler keeps every
admitted solve's fields and wake accumulators resident on the GPU and admits
new requests in arrival order whenever a slot and enough of the device-memory
budget are free. All admitted solves advance together, one batch launch per
step, in rounds of ``round_steps`` steps; between rounds finished solves hand
back their wake and free their memory, and newly arrived requests join. A
solve's result does not depend on what it shares the GPU with (batched steps
are bit-identical to solo steps).

The policy lives in ``Server`` and talks to the GPU only through a backend
(``GpuBackend`` here, a fake one in the CPU tests).
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclasses.dataclass
class Result:
    rid: int
    status: str                 # "ok" | "rejected" | "cancelled" | "error"
    wake: Optional[np.ndarray] = None
    s0: float = 0.0
    ds: float = 0.0
    error: Optional[str] = None
    t_arrival: float = 0.0
    t_admit: Optional[float] = None
    t_done: Optional[float] = None
    cell_steps: int = 0

    @property
    def latency(self) -> Optional[float]:
        return None if self.t_done is None else self.t_done - self.t_arrival


class GpuBackend:
    """Solves through the C ABI; active solves advance as one tetm batch."""

    def __init__(self, precision: str = "fp32", tiling=(28, 20, 32), graph: bool = True):
        from . import tetm
        self.tetm = tetm
        self.precision = precision
        self.tiling = tiling
        self.graph = graph
        self.batch = None
        self.members: List = []

    def bytes_needed(self, w) -> int:
        g = self.tetm.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, self.precision)
        return self.tetm.tetm_bytes_needed(g)

    def create(self, w):
        s = self.tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, self.precision, pec=w.pec)
        s.set_bunch(w.sigma, w.charge, w.i0, w.j0)
        s.set_tiling(*self.tiling)
        return s

    def advance(self, handles: List, limits: List[int], nsteps: int) -> None:
        if handles != self.members:
            self._drop_batch()
            self.members = list(handles)
            if handles:
                self.batch = self.tetm.Batch(handles, limits,
                                             graph_steps=nsteps if self.graph else 0)
        if self.batch is not None:
            self.batch.step(nsteps)
            self.batch.sync()

    def step_of(self, h) -> int:
        return int(h.info()["step"])

    def finish(self, h):
        return h.wake()

    def release(self, h) -> None:
        if h in self.members:
            self._drop_batch()
            self.members = []
        h.close()

    def _drop_batch(self):
        if self.batch is not None:
            self.batch.close()
            self.batch = None


class Server:
    def __init__(self, backend, hbm_budget: float = 150e9, max_slots: int = 64,
                 round_steps: int = 64, clock: Callable[[], float] = time.perf_counter,
                 sleep: Callable[[float], None] = time.sleep):
        self.b = backend
        self.budget = float(hbm_budget)
        self.max_slots = int(max_slots)
        self.round_steps = int(round_steps)
        self.clock = clock
        self.sleep = sleep
        self.pending: collections.deque = collections.deque()   # (rid, workload, t_arrival, bytes)
        self.active: Dict[int, dict] = {}
        self.results: Dict[int, Result] = {}
        self.used = 0.0
        self.cancelled = set()
        self.rounds = 0
        self.busy_s = 0.0
        self.max_active = 0

    # ---- requests ------------------------------------------------------------
    def submit(self, rid: int, w, t_arrival: Optional[float] = None) -> None:
        t = self.clock() if t_arrival is None else t_arrival
        try:
            need = float(self.b.bytes_needed(w))
        except Exception as e:  # malformed request
            self.results[rid] = Result(rid, "error", error=str(e), t_arrival=t, t_done=t)
            return
        if need <= 0 or need > self.budget:
            self.results[rid] = Result(rid, "rejected",
                                       error="needs %.3g B of a %.3g B budget" % (need, self.budget),
                                       t_arrival=t, t_done=t)
            return
        self.pending.append((rid, w, t, need))

    def cancel(self, rid: int) -> None:
        self.cancelled.add(rid)

    # ---- scheduling ------------------------------------------------------------
    def _admit(self) -> None:
        kept = collections.deque()
        while self.pending:
            rid, w, t, need = self.pending.popleft()
            if rid in self.cancelled:
                self.results[rid] = Result(rid, "cancelled", t_arrival=t, t_done=self.clock())
                continue
            if len(self.active) >= self.max_slots or self.used + need > self.budget:
                kept.append((rid, w, t, need))
                kept.extend(self.pending)   # keep arrival order: nobody overtakes the head
                self.pending.clear()
                break
            try:
                h = self.b.create(w)
            except Exception as e:
                self.results[rid] = Result(rid, "error", error=str(e), t_arrival=t,
                                           t_done=self.clock())
                continue
            self.used += need
            self.active[rid] = {"h": h, "w": w, "t": t, "need": need, "t_admit": self.clock(),
                                "limit": int(w.steps)}
        self.pending = kept

    def _collect(self) -> None:
        for rid in list(self.active):
            a = self.active[rid]
            done = self.b.step_of(a["h"]) >= a["limit"]
            if not (done or rid in self.cancelled):
                continue
            if done and rid not in self.cancelled:
                wake, s0, ds = self.b.finish(a["h"])
                r = Result(rid, "ok", wake, s0, ds, t_arrival=a["t"], t_admit=a["t_admit"],
                           cell_steps=a["w"].cells * a["limit"])
            else:
                r = Result(rid, "cancelled", t_arrival=a["t"], t_admit=a["t_admit"])
            self.b.release(a["h"])
            r.t_done = self.clock()
            self.results[rid] = r
            self.used -= a["need"]
            del self.active[rid]

    def round(self) -> None:
        self._admit()
        self.max_active = max(self.max_active, len(self.active))
        if self.active:
            t0 = self.clock()
            ids = list(self.active)
            self.b.advance([self.active[i]["h"] for i in ids], [self.active[i]["limit"] for i in ids],
                           self.round_steps)
            self.busy_s += self.clock() - t0
            self.rounds += 1
        self._collect()

    def idle(self) -> bool:
        return not self.pending and not self.active

    def run_stream(self, requests, workload_of, t0: Optional[float] = None) -> Dict[int, Result]:
        """Replay (rid, arrival) requests in real time: each is submitted once
        the clock passes its arrival; runs until every request has a result."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        t0 = self.clock() if t0 is None else t0
        i = 0
        while i < len(reqs) or not self.idle():
            now = self.clock() - t0
            while i < len(reqs) and reqs[i].arrival <= now:
                self.submit(reqs[i].rid, workload_of(reqs[i]), t0 + reqs[i].arrival)
                i += 1
            if self.idle() and i < len(reqs):
                self.sleep(max(0.0, reqs[i].arrival - (self.clock() - t0)))
                continue
            self.round()
        return self.results


def latency_stats(results: Dict[int, Result]) -> dict:
    ok = [r for r in results.values() if r.status == "ok"]
    lat = np.array([r.latency for r in ok]) if ok else np.zeros(0)
    out = {"requests": len(results), "ok": len(ok),
           "rejected": sum(r.status == "rejected" for r in results.values()),
           "cancelled": sum(r.status == "cancelled" for r in results.values()),
           "error": sum(r.status == "error" for r in results.values())}
    if ok:
        t_first = min(r.t_arrival for r in ok)
        t_last = max(r.t_done for r in ok)
        out.update({"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                    "mean_s": float(lat.mean()), "makespan_s": t_last - t_first,
                    "solves_per_s": len(ok) / (t_last - t_first) if t_last > t_first else None,
                    "cell_steps": int(sum(r.cell_steps for r in ok))})
    return out
