"""Batches: several uneven solves advancing in one launch per step (optionally
replayed from a CUDA graph) give every member exactly the result it gets
stepped alone, and members retire at their own step limits."""
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


def _mix(precision):
    ws = wl.batch_solves(count=5, seed=123, n_lo=20, n_hi=44, precision=precision)
    ws[1].steps = 37          # uneven limits, one shorter than a graph run
    return ws


@pytest.mark.parametrize("precision,graph_steps,tiling", [("fp32", 8, (28, 20, 16)), ("fp32", 0, (28, 12, 16)),
                                                          ("fp32", 8, (56, 28, 16)), ("fp32", 0, (56, 28, 9)),
                                                          ("fp64", 16, (28, 20, 16)), ("fp64", 4, (28, 8, 16))])
def test_batch_members_equal_solo_runs_bitwise(tetm, precision, graph_steps, tiling):
    """Warp-tiled batches (tile width 28) and, for float32 with the slab
    kernel's 56 x 28 tile, batched slab kernels."""
    ws = _mix(precision)
    solo = []
    for w in ws:
        s = tetm.Solver.from_workload(w)
        s.set_tiling(*tiling)
        s.step(w.steps)
        solo.append((s.wake()[0], s.get("ez"), s.get("hy"), s.get("ex")))
        s.close()
    members = []
    for w in ws:
        s = tetm.Solver.from_workload(w)
        s.set_tiling(*tiling)
        members.append(s)
    b = tetm.Batch(members, [w.steps for w in ws], graph_steps=graph_steps)
    most = max(w.steps for w in ws)
    b.step(most // 3)
    b.step(most - most // 3 + 5)       # past every limit
    b.sync()
    assert b.info()["active"] == 0
    for s, w, ref in zip(members, ws, solo):
        assert s.info()["step"] == w.steps
        got = (s.wake()[0], s.get("ez"), s.get("hy"), s.get("ex"))
        for a, r in zip(got, ref):
            assert np.array_equal(a, r)
    with pytest.raises(tetm.TetmError) as e:
        members[0].step(1)
    assert e.value.code == tetm.TETM_E_STATE
    b.close()
    members[0].step(1)                  # independent again


def test_batch_member_fp64_matches_oracle(tetm):
    ws = _mix("fp64")
    members = [tetm.Solver.from_workload(w) for w in ws]
    b = tetm.Batch(members, [w.steps for w in ws], graph_steps=8)
    b.step(max(w.steps for w in ws))
    b.sync()
    w = ws[2]
    o = Oracle(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, pec=w.pec)
    o.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    o.step(w.steps)
    ref = o.wake()[0]
    got = members[2].wake()[0]
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    b.close()


def test_batch_rejects_mixed_precision(tetm):
    a = tetm.Solver.from_workload(wl.plain_pipe(nz=20, n=8, steps=5, precision="fp64"))
    c = tetm.Solver.from_workload(wl.plain_pipe(nz=20, n=8, steps=5, precision="fp32"))
    with pytest.raises(tetm.TetmError) as e:
        tetm.Batch([a, c])
    assert e.value.code == tetm.TETM_E_ARG
    with pytest.raises(tetm.TetmError):
        tetm.Batch([a, a])


def test_slab_batch_with_many_retired_members_equals_solo_runs(tetm):
    """Float32 slab-kernel batch of twelve solves whose step limits spread
    from 6 to 90: most work items of the later launches belong to members
    that have retired; every member still equals its solo run bit for bit."""
    ws = wl.batch_solves(count=12, seed=77, n_lo=16, n_hi=40, precision="fp32")
    for i, w in enumerate(ws):
        w.steps = 6 + 7 * i
    solo = []
    for w in ws:
        s = tetm.Solver.from_workload(w)
        s.step(w.steps)
        solo.append((s.wake()[0], s.get("ez"), s.get("hx")))
        s.close()
    members = [tetm.Solver.from_workload(w) for w in ws]
    assert members[0].info()["tile_x"] == 56                 # the float32 default: the slab kernel
    b = tetm.Batch(members, [w.steps for w in ws], graph_steps=8)
    b.step(95)
    b.sync()
    for s, w, ref in zip(members, ws, solo):
        assert s.info()["step"] == w.steps
        for a, r in zip((s.wake()[0], s.get("ez"), s.get("hx")), ref):
            assert np.array_equal(a, r)
    b.close()
