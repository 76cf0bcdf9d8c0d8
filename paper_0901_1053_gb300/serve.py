"""Continuous-batching server for wakefield solves.

Requests (grid, geometry, bunch) arrive over time. The scheduler keeps every
admitted solve's fields and wake accumulators resident on the GPU and admits
new requests in arrival order whenever a slot and enough of the device-memory
budget are free. All admitted solves advance together in one batch, a call of
``round_steps`` steps at a time; a request that becomes ready joins at the
next call and a finished one leaves after the call that finished it. A
solve's result does not depend on what it shares the GPU with (batched steps
are bit-identical to solo steps).

Host work overlaps GPU work:
  * building a request's geometry and creating its solve (allocation, upload,
    geometry kernels on a stream of its own), and reading back a finished
    wake and releasing the solve, run on worker threads while the batch runs;
  * the batch is a fixed table of slots (tetm_batch_create_slots): a join or a
    leave is a few stream-ordered copies, never a rebuild of the batch or a
    re-capture of its CUDA graph;
  * the scheduling thread queues at most ``queue_ahead`` calls beyond the one
    the GPU is running, so a newly ready request waits at most that many
    calls and the GPU never waits for the host while work is admitted.

The policy lives in ``Server`` and talks to the GPU only through a backend
(``GpuBackend`` here, a fake one in the CPU tests). With ``workers=0`` the
backend's preparation and read-back run inline on the scheduling thread.
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
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
    """Solves through the C ABI; admitted solves are members of one slot-table
    batch (tetm_batch_create_slots) of ``max_slots`` slots."""

    def __init__(self, precision: str = "fp32", tiling=(56, 28, 32), graph: bool = True,
                 max_slots: int = 64, round_steps: int = 16, pool_bytes: float = 0):
        from . import tetm
        self.tetm = tetm
        self.precision = precision
        self.tiling = tuple(int(t) for t in tiling)
        self.batch = tetm.Batch.slots(max_slots, precision, self.tiling[:2],
                                      graph_steps=round_steps if graph else 0)
        if pool_bytes:
            tetm.tetm_pool_reserve(int(pool_bytes))
        self._tl = threading.local()

    def _stream(self) -> int:
        """A non-blocking stream per host thread: solves created there queue
        their work on it, beside the batch's stream."""
        st = getattr(self._tl, "stream", None)
        if st is None:
            import torch
            st = torch.cuda.Stream()
            self._tl.stream = st
        return int(st.cuda_stream)

    def bytes_needed(self, w) -> int:
        g = self.tetm.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, self.precision)
        return self.tetm.tetm_bytes_needed(g)

    def prepare(self, w):
        w = w.build() if hasattr(w, "build") else w
        s = self.tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, self.precision, pec=w.pec,
                             stream=self._stream())
        s.set_tiling(*self.tiling)
        s.set_bunch(w.sigma, w.charge, w.i0, w.j0)
        return s

    def join(self, h, limit: int) -> None:
        self.batch.add(h, limit)

    def advance(self, nsteps: int) -> None:
        self.batch.step(nsteps)

    def throttle(self, max_pending: int) -> float:
        return self.batch.wait(max_pending)

    def step_of(self, h) -> int:
        return int(h.info()["step"])

    def leave(self, h) -> None:
        self.batch.remove(h)

    def finish(self, h):
        return h.wake()

    def release(self, h) -> None:
        h.close()

    def close(self) -> None:
        if self.batch is not None:
            self.batch.close()
            self.batch = None


class _Inline:
    """Executor stand-in that runs each job at once (workers=0)."""

    def submit(self, fn, *args):
        f = cf.Future()
        try:
            f.set_result(fn(*args))
        except BaseException as e:  # reported through the future, as a pool would
            f.set_exception(e)
        return f

    def shutdown(self, wait=True):
        pass


class Server:
    def __init__(self, backend, hbm_budget: float = 150e9, max_slots: int = 64,
                 round_steps: int = 16, queue_ahead: int = 2, workers: int = 1,
                 clock: Callable[[], float] = time.perf_counter,
                 sleep: Callable[[float], None] = time.sleep):
        self.b = backend
        self.budget = float(hbm_budget)
        self.max_slots = int(max_slots)
        self.round_steps = int(round_steps)
        self.queue_ahead = int(queue_ahead)
        self.clock = clock
        self.sleep = sleep
        self.pool = cf.ThreadPoolExecutor(max_workers=workers) if workers > 0 else _Inline()
        self.pending: collections.deque = collections.deque()   # (rid, workload, t_arrival, bytes)
        self.preparing: List[dict] = []                          # admission order
        self.active: Dict[int, dict] = {}
        self.finishing: List[dict] = []
        self.results: Dict[int, Result] = {}
        self.used = 0.0
        self.cancelled = set()
        self.rounds = 0
        self.busy_s = 0.0          # device time of the batch calls (from the backend)
        self.idle_s = 0.0          # time with no request anywhere, after the first arrival
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
        """Start preparing pending requests, in arrival order, while a slot and
        the budget allow (nobody overtakes the head)."""
        while self.pending:
            rid, w, t, need = self.pending[0]
            if rid in self.cancelled:
                self.pending.popleft()
                self.results[rid] = Result(rid, "cancelled", t_arrival=t, t_done=self.clock())
                continue
            if (len(self.active) + len(self.preparing) >= self.max_slots
                    or self.used + need > self.budget):
                break
            self.pending.popleft()
            self.used += need
            self.preparing.append({"rid": rid, "w": w, "t": t, "need": need, "t_admit": self.clock(),
                                   "limit": int(w.steps), "fut": self.pool.submit(self.b.prepare, w)})

    def _join(self) -> None:
        """Prepared solves join the batch in admission order."""
        while self.preparing and self.preparing[0]["fut"].done():
            p = self.preparing.pop(0)
            rid = p["rid"]
            try:
                h = p["fut"].result()
            except Exception as e:
                self.results[rid] = Result(rid, "error", error=str(e), t_arrival=p["t"],
                                           t_done=self.clock())
                self.used -= p["need"]
                continue
            if rid in self.cancelled:
                self._retire(p, h, finish=False)
                continue
            self.b.join(h, p["limit"])
            p["h"] = h
            self.active[rid] = p

    def _retire(self, a: dict, h, finish: bool) -> None:
        """Hand a solve to a worker: read its wake (finish) and release it."""
        def job():
            try:
                out = self.b.finish(h) if finish else None
            finally:
                self.b.release(h)
            return out, self.clock()
        a["h"] = h
        a["finish"] = finish
        a["fut"] = self.pool.submit(job)
        self.finishing.append(a)

    def _collect(self) -> None:
        """Finished or cancelled members leave the batch."""
        for rid in list(self.active):
            a = self.active[rid]
            done = self.b.step_of(a["h"]) >= a["limit"]
            if not (done or rid in self.cancelled):
                continue
            self.b.leave(a["h"])
            del self.active[rid]
            self._retire(a, a["h"], finish=done and rid not in self.cancelled)

    def _reap(self) -> None:
        """Results of the read-backs that completed; their memory is free."""
        keep = []
        for a in self.finishing:
            if not a["fut"].done():
                keep.append(a)
                continue
            rid = a["rid"]
            try:
                out, t_done = a["fut"].result()
            except Exception as e:
                r = Result(rid, "error", error=str(e), t_arrival=a["t"], t_admit=a["t_admit"],
                           t_done=self.clock())
            else:
                if a["finish"]:
                    wake, s0, ds = out
                    r = Result(rid, "ok", wake, s0, ds, t_arrival=a["t"], t_admit=a["t_admit"],
                               t_done=t_done, cell_steps=a["w"].cells * a["limit"])
                else:
                    r = Result(rid, "cancelled", t_arrival=a["t"], t_admit=a["t_admit"], t_done=t_done)
            self.results[rid] = r
            self.used -= a["need"]
        self.finishing = keep

    def _wait_host(self, timeout: Optional[float]) -> None:
        """Nothing to step: wait for a preparation or a read-back to end."""
        futs = [p["fut"] for p in self.preparing] + [a["fut"] for a in self.finishing]
        if futs:
            cf.wait(futs, timeout=timeout, return_when=cf.FIRST_COMPLETED)

    def round(self, wait_timeout: Optional[float] = None) -> None:
        """Admit, join, queue one batch call of round_steps steps (keeping at
        most queue_ahead calls queued behind the running one), let finished
        members leave, and collect completed read-backs."""
        self._reap()
        self._admit()
        self._join()
        self.max_active = max(self.max_active, len(self.active))
        if self.active:
            self.b.advance(self.round_steps)
            self.rounds += 1
            self.busy_s = self.b.throttle(self.queue_ahead)
            self._collect()
        else:
            self._wait_host(wait_timeout)
        self._reap()

    def drain(self) -> None:
        """Wait for the queued calls and every read-back."""
        self.busy_s = self.b.throttle(0) if hasattr(self.b, "throttle") else self.busy_s
        for a in list(self.finishing):
            cf.wait([a["fut"]])
        self._reap()

    def idle(self) -> bool:
        return not (self.pending or self.preparing or self.active or self.finishing)

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
                t_sleep = self.clock()
                self.sleep(max(0.0, reqs[i].arrival - (t_sleep - t0)))
                if i > 0:
                    self.idle_s += self.clock() - t_sleep
                continue
            nxt = reqs[i].arrival - (self.clock() - t0) if i < len(reqs) else None
            self.round(wait_timeout=None if nxt is None else max(0.0, nxt))
        self.drain()
        return self.results

    def close(self) -> None:
        self.pool.shutdown(wait=True)


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
