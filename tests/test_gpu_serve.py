"""Slot-table batches and the server on the GPU: solves that join a running
batch, leave it early or late, and reuse freed slots advance exactly as alone
(fields and wakes bit for bit); solves created on other streams from a worker
thread join without a host wait; the server's results equal solo results and
the FP32 served wake is within 1e-4 of the FP64 oracle's peak."""
import threading

import numpy as np
import pytest

from oracle import Oracle
from paper_0901_1053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

COMPONENTS = ("ex", "ey", "ez", "hx", "hy", "hz")


@pytest.fixture(scope="module")
def tetm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_1053_gb300 import tetm as t
    return t


def solo(tetm, w, steps, tile, stream=None):
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, w.precision, pec=w.pec, stream=stream)
    s.set_tiling(*tile)
    s.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    s.step(steps)
    return s


def make(tetm, w, tile, stream=None):
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, w.precision, pec=w.pec, stream=stream)
    s.set_tiling(*tile)
    s.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    return s


def same(tetm, got, w, steps, tile):
    ref = solo(tetm, w, steps, tile)
    assert got.info()["step"] == steps
    assert np.array_equal(got.wake()[0], ref.wake()[0])
    for c in COMPONENTS:
        assert np.array_equal(got.get(c), ref.get(c)), c
    ref.close()


@pytest.mark.parametrize("precision,tile", [("fp32", (56, 28, 32)), ("fp32", (28, 20, 16)),
                                            ("fp64", (28, 20, 32))])
def test_slot_batch_join_leave_reuse(tetm, precision, tile):
    import torch
    ws = [wl.make_solve("m%d" % i, n, kind, 4.0, np.random.default_rng(50 + i), precision)
          for i, (n, kind) in enumerate([(40, "pipe"), (24, "collimator"), (32, "cavity"), (48, "pipe")])]
    b = tetm.Batch.slots(3, precision, tile[:2], graph_steps=8)
    side = torch.cuda.Stream()
    a = make(tetm, ws[0], tile)
    assert b.add(a, 70) == 0
    b.step(16)                                   # a alone (one warm launch, one graph, 7 launches)
    made = {}
    th = threading.Thread(target=lambda: made.update(s=make(tetm, ws[1], tile, stream=side.cuda_stream)))
    th.start()
    b.step(8)                                    # a runs while another thread creates b1
    th.join()
    b1 = made["s"]
    assert b.add(b1, 30) == 1
    c = make(tetm, ws[2], tile)
    assert b.add(c, -1) == 2
    with pytest.raises(tetm.TetmError) as e:     # all slots taken
        b.add(make(tetm, ws[3], tile), 10)
    assert e.value.code == tetm.TETM_E_STATE
    b.step(24)                                   # a: 48, b1: 24, c: 24
    b.remove(c)                                  # c leaves early, mid-run
    d = make(tetm, ws[3], tile)
    assert b.add(d, 40) == 2                     # and d takes its slot
    b.step(20)                                   # a: 68, b1: 30 (limit), d: 20
    b.remove(b1)
    b.step(9)                                    # a: 70 (limit), d: 29
    info = b.info()
    assert info["members"] == 2 and info["active"] == 1
    busy = b.wait(0)
    assert busy > 0
    b.sync()
    for s, w, n in ((a, ws[0], 70), (b1, ws[1], 30), (c, ws[2], 24)):
        same(tetm, s, w, n, tile)
    b.remove(d)
    same(tetm, d, ws[3], 29, tile)
    d.step(3)                                    # a member that left steps alone again
    same(tetm, d, ws[3], 32, tile)
    b.close()
    for s in (a, b1, c, d):
        s.close()


def test_served_results_equal_solo_results(tetm):
    from paper_0901_1053_gb300.serve import GpuBackend, Server, latency_stats
    reqs = wl.request_stream(count=10, rate=200.0, seed=77, n_lo=16, n_hi=40)
    tile = (56, 28, 32)
    be = GpuBackend("fp32", tile, max_slots=6, round_steps=16)
    srv = Server(be, hbm_budget=4e9, max_slots=6, round_steps=16, workers=2)
    res = srv.run_stream(reqs, lambda r: r.spec("fp32"))
    srv.close()
    be.close()
    st = latency_stats(res)
    assert st["ok"] == len(reqs)
    assert srv.max_active > 1 and srv.busy_s > 0
    for r in reqs:
        w = r.workload("fp32")
        s = solo(tetm, w, w.steps, tile)
        assert np.array_equal(res[r.rid].wake, s.wake()[0]), r.rid
        s.close()
    # and the FP32 served wake is within 1e-4 of its peak of the FP64 oracle
    r = reqs[0]
    w = r.workload("fp64")
    o = Oracle(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, pec=w.pec)
    o.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    o.step(w.steps)
    ref = o.wake()[0]
    assert np.max(np.abs(res[r.rid].wake - ref)) <= 1e-4 * np.max(np.abs(ref))
