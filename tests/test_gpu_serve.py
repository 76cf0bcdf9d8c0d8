"""The server on the GPU: requests admitted while others run share batch
launches, and every served wake equals the wake of the same request solved
alone (batched steps are bit-identical to solo steps)."""
import numpy as np
import pytest

from oracle import Oracle
from paper_0901_1053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tetm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_1053_gb300 import tetm as t
    return t


def test_served_results_equal_solo_results(tetm):
    from paper_0901_1053_gb300.serve import GpuBackend, Server, latency_stats
    reqs = wl.request_stream(count=10, rate=200.0, seed=77, n_lo=16, n_hi=40)
    srv = Server(GpuBackend("fp32"), hbm_budget=4e9, max_slots=6, round_steps=16)
    res = srv.run_stream(reqs, lambda r: r.workload("fp32"))
    st = latency_stats(res)
    assert st["ok"] == len(reqs)
    assert srv.max_active > 1
    for r in reqs:
        w = r.workload("fp32")
        s = tetm.Solver.from_workload(w)
        s.set_tiling(28, 20, 32)
        s.step(w.steps)
        solo = s.wake()[0]
        s.close()
        assert np.array_equal(res[r.rid].wake, solo), r.rid
    # and the FP32 served wake is within 1e-4 of its peak of the FP64 oracle
    r = reqs[0]
    w = r.workload("fp64")
    o = Oracle(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, pec=w.pec)
    o.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    o.step(w.steps)
    ref = o.wake()[0]
    assert np.max(np.abs(res[r.rid].wake - ref)) <= 1e-4 * np.max(np.abs(ref))
