"""GPU transverse (dipole) wake of the Cartesian solver (tetm_set_observer,
tetm_transverse_wake; Sec. 5): W_x on the x-edge line (i+1/2, j) and W_y on
the y-edge line (i, j+1/2) of the observer, against the FP64 oracle
(oracle/tetm_oracle.c), whose definition is pinned by the exact discrete
Panofsky-Wenzel relation in tests/test_oracle_pins.py.

Every kernel path is covered: the reference updates (a gather between U5
and U6) and, after a ping-pong step of the block-tiled kernel, the three
warp-tiled sweeps (float64 asynchronous-copy ring, register ring, per-entry
coefficients) or a batch, one gather launch over the observer column. The
wake is gathered once an observer is set. Tolerances as for the
longitudinal wake: 1e-12 of the peak in float64, 1e-4 in float32."""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_0901_1053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32_WAKE = 1e-4


@pytest.fixture(scope="module")
def tetm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_1053_gb300 import tetm as t
    return t


def rel_err(a, b):
    peak = np.max(np.abs(b))
    assert peak > 0
    return float(np.max(np.abs(a - b)) / peak)


def collimator(nx, ny, nz, precision, i0, j0):
    """Staircase collimator on a ragged grid with an off-axis bunch."""
    w = wl.scaled_collimator(max(nx, ny), nz, sigma_cells=2.5, precision=precision)
    w.nx, w.ny = nx, ny
    w.pec = wl.radius_mask(nx, ny, nz, wl.collimator_radius(nz, 0.45 * min(nx, ny),
                                                             0.2 * min(nx, ny), nz // 4, nz // 2))
    w.i0, w.j0 = i0, j0
    w.steps = nz + 25
    return w


def oracle_transverse(w, obs, eps=None, mu=None, static_k=None):
    o = Oracle(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, eps_r=eps, mu_r=mu, pec=w.pec)
    if static_k:
        o.set_bunch_static(w.sigma, w.charge, w.i0, w.j0, static_k)
    else:
        o.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    o.set_observer(*obs)
    o.step(w.steps)
    return o.transverse_wake(), o.wake()[0]


KERNELS = [("reference", None), ("fused", (32, 8, 16)), ("fused", (64, 4, 7)),
           ("fused", (28, 8, 16)), ("fused", (28, 20, 5)), ("fused", (28, 12, 64))]


@pytest.mark.parametrize("kernel,tiling", KERNELS)
@pytest.mark.parametrize("obs", [(22, 15), (27, 16), (28, 20), (21, 18)])
def test_transverse_wake_fp64_matches_oracle(tetm, kernel, tiling, obs):
    """40 x 36 x 70 collimator, bunch at (21, 18); observers inside a tile, on
    the last column of one warp tile and the first of the next, on a row
    boundary of the tile heights used, and on the bunch line."""
    w = collimator(40, 36, 70, "fp64", 21, 18)
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp64", pec=w.pec)
    s.set_kernel(kernel)
    if tiling:
        s.set_tiling(*tiling)
    s.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    s.set_observer(*obs)
    s.step(w.steps)
    (rx, ry), rl = oracle_transverse(w, obs)
    gx, gy = s.transverse_wake()
    assert rel_err(gx, rx) <= TOL64
    assert rel_err(gy, ry) <= TOL64
    err = rel_err(s.wake()[0], rl)
    print("wake error", kernel, tiling, obs, err)
    assert err <= TOL64, err


def test_transverse_wake_fp32_within_1e4(tetm):
    w = collimator(48, 44, 90, "fp32", 25, 21)
    s = tetm.Solver.from_workload(w)
    s.set_observer(23, 22)
    s.step(w.steps)
    (rx, ry), _ = oracle_transverse(w, (23, 22))
    gx, gy = s.transverse_wake()
    assert rel_err(gx, rx) <= TOL32_WAKE
    assert rel_err(gy, ry) <= TOL32_WAKE


@pytest.mark.parametrize("kernel,tiling", [("reference", None), ("fused", (28, 8, 5)),
                                           ("fused", (28, 20, 16))])
def test_transverse_wake_with_materials_fp64(tetm, kernel, tiling):
    """Per-cell eps_r, mu_r and PEC (the warp sweep with coefficient arrays)."""
    nx, ny, nz = 33, 29, 41
    eps, mu, pec = wl.random_materials(nx, ny, nz, 5)
    pec[:, 12:18, 14:19] = 0                       # a clear channel around the bunch line
    s = tetm.Solver(nx, ny, nz, wl.DXY, wl.DXY, wl.DZ, 0.0, "fp64", eps_r=eps, mu_r=mu, pec=pec)
    s.set_kernel(kernel)
    if tiling:
        s.set_tiling(*tiling)
    sigma = 2 * wl.DZ
    s.set_bunch(sigma, 1e-9, 16, 15)
    s.set_observer(15, 14)
    steps = nz + 30
    s.step(steps)
    o = Oracle(nx, ny, nz, wl.DXY, wl.DXY, wl.DZ, 0.0, eps_r=eps, mu_r=mu, pec=pec)
    o.set_bunch(sigma, 1e-9, 16, 15)
    o.set_observer(15, 14)
    o.step(steps)
    rx, ry = o.transverse_wake()
    gx, gy = s.transverse_wake()
    assert rel_err(gx, rx) <= TOL64
    assert rel_err(gy, ry) <= TOL64


def test_transverse_wake_static_start_matches_oracle(tetm):
    nx = ny = 30
    nz = 120
    w = collimator(nx, ny, nz, "fp64", 16, 14)
    w.pec = wl.radius_mask(nx, ny, nz, wl.collimator_radius(nz, 12.5, 6.5, 60, 90))
    K = 2 * math.ceil(5 * w.sigma / w.dz - 1e-12) + 2
    w.steps = nz - K + 30
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp64", pec=w.pec)
    s.set_bunch_static(w.sigma, w.charge, w.i0, w.j0, K)
    s.set_observer(14, 15)
    s.step(w.steps)
    (rx, ry), rl = oracle_transverse(w, (14, 15), static_k=K)
    gx, gy = s.transverse_wake()
    assert rel_err(gx, rx) <= TOL64
    assert rel_err(gy, ry) <= TOL64
    err = rel_err(s.wake()[0], rl)
    print("wake error static", err)
    assert err <= TOL64, err


def test_batch_member_transverse_wake_equals_solo(tetm):
    ws = wl.batch_solves(count=3, seed=77, n_lo=20, n_hi=36, precision="fp32")
    obs = [(w.i0 + 2, w.j0 - 1) for w in ws]
    solo = []
    for w, ob in zip(ws, obs):
        s = tetm.Solver.from_workload(w)
        s.set_observer(*ob)
        s.step(w.steps)
        solo.append(s.transverse_wake())
        s.close()
    members = []
    for w, ob in zip(ws, obs):
        s = tetm.Solver.from_workload(w)
        s.set_observer(*ob)
        members.append(s)
    b = tetm.Batch(members, [w.steps for w in ws], graph_steps=8)
    b.step(max(w.steps for w in ws))
    b.sync()
    for s, ref in zip(members, solo):
        got = s.transverse_wake()
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    b.close()


def test_checkpoint_carries_the_transverse_wake(tetm):
    w = wl.scaled_collimator(32, 64, sigma_cells=3.0, precision="fp32")
    a = tetm.Solver.from_workload(w)
    a.set_observer(w.i0 + 1, w.j0)
    a.step(50)
    buf = a.save()
    a.step(30)
    b = tetm.Solver.from_workload(w)
    b.set_observer(w.i0 + 1, w.j0)
    b.load(buf)
    b.step(30)
    for x, y in zip(a.transverse_wake(), b.transverse_wake()):
        assert np.array_equal(x, y)
    c = tetm.Solver.from_workload(w)            # another observer: not the same solve
    c.set_observer(w.i0, w.j0 + 1)
    with pytest.raises(tetm.TetmError) as e:
        c.load(buf)
    assert e.value.code == tetm.TETM_E_ARG
    d = tetm.Solver.from_workload(w)            # no observer at all
    with pytest.raises(tetm.TetmError) as e:
        d.load(buf)
    assert e.value.code == tetm.TETM_E_ARG


def test_observer_arguments_and_state(tetm):
    w = wl.plain_pipe(nz=40, n=12, steps=10, precision="fp64")
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp64", pec=w.pec)
    with pytest.raises(tetm.TetmError) as e:
        s.set_observer(3, 3)                       # no bunch
    assert e.value.code == tetm.TETM_E_STATE
    with pytest.raises(tetm.TetmError) as e:
        s.transverse_wake()
    assert e.value.code == tetm.TETM_E_STATE
    s.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    with pytest.raises(tetm.TetmError) as e:
        s.transverse_wake()                        # not turned on (no observer)
    assert e.value.code == tetm.TETM_E_STATE
    for bad in ((-1, 3), (w.nx, 3), (3, w.ny)):
        with pytest.raises(tetm.TetmError) as e:
            s.set_observer(*bad)
        assert e.value.code == tetm.TETM_E_ARG
    s.set_observer(w.nx - 1, w.ny - 1)
    s.step(1)
    with pytest.raises(tetm.TetmError) as e:
        s.set_observer(3, 3)                       # after the first step
    assert e.value.code == tetm.TETM_E_STATE


@pytest.mark.parametrize("tiling", [None, (28, 20, 16)])
def test_transverse_wake_with_materials_fp32(tetm, tiling):
    """Per-cell eps_r, mu_r and PEC in float32: the slab kernel with coefficient
    arrays (the default) and the warp-tiled one, within 1e-4 of the peak."""
    nx, ny, nz = 70, 41, 60
    eps, mu, pec = wl.random_materials(nx, ny, nz, 12)
    pec[:, 15:27, 28:42] = 0                       # a clear channel around the bunch line
    s = tetm.Solver(nx, ny, nz, wl.DXY, wl.DXY, wl.DZ, 0.0, "fp32", eps_r=eps, mu_r=mu, pec=pec)
    if tiling:
        s.set_tiling(*tiling)
    sigma = 2.5 * wl.DZ
    s.set_bunch(sigma, 1e-9, 35, 21)
    s.set_observer(34, 20)
    steps = nz + 30
    s.step(steps)
    o = Oracle(nx, ny, nz, wl.DXY, wl.DXY, wl.DZ, 0.0, eps_r=eps, mu_r=mu, pec=pec)
    o.set_bunch(sigma, 1e-9, 35, 21)
    o.set_observer(34, 20)
    o.step(steps)
    rx, ry = o.transverse_wake()
    gx, gy = s.transverse_wake()
    assert rel_err(gx, rx) <= TOL32_WAKE
    assert rel_err(gy, ry) <= TOL32_WAKE
    assert rel_err(s.wake()[0], o.wake()[0]) <= TOL32_WAKE
