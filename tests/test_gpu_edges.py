"""Degenerate cases of the Cartesian path against the FP64 oracle: a box that is
PEC throughout (no work items at all), a bunch on the first node line off the
wall with a bunch shorter than a cell, a bunch whose wake window is longer than
the box, zero steps, and the smallest grids, for the float32 default kernel
(slab) and the float64 default (warp-tiled)."""
import math

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


def run_both(tetm, nx, ny, nz, precision, sigma, i0, j0, steps, pec=None):
    s = tetm.Solver(nx, ny, nz, wl.DXY, wl.DXY, wl.DZ, 0.0, precision, pec=pec)
    s.set_bunch(sigma, 1e-9, i0, j0)
    s.step(steps)
    s.sync()
    o = Oracle(nx, ny, nz, wl.DXY, wl.DXY, wl.DZ, 0.0, pec=pec)
    o.set_bunch(sigma, 1e-9, i0, j0)
    o.step(steps)
    return s, o


def wake_err(s, o):
    g, r = s.wake()[0], o.wake()[0]
    peak = np.max(np.abs(r))
    return float(np.max(np.abs(g - r)) / peak) if peak > 0 else float(np.max(np.abs(g)))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_all_pec_box_has_no_work_and_no_field(tetm, precision):
    nx, ny, nz = 20, 18, 40
    pec = np.ones((nz, ny, nx), np.uint8)
    s, o = run_both(tetm, nx, ny, nz, precision, 2 * wl.DZ, 10, 9, 60, pec=pec)
    assert s.info()["work_items"] == 0
    for c in COMPONENTS:
        assert np.all(s.get(c) == 0.0)
    assert np.all(s.wake()[0] == 0.0) and np.all(o.wake()[0] == 0.0)
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("fp64", 1e-12)])
def test_short_bunch_on_the_first_node_line(tetm, precision, tol):
    """sigma = 0.15 dz (c0 = 1, a three-sample window) on node line (1, 1)."""
    s, o = run_both(tetm, 9, 7, 12, precision, 0.15 * wl.DZ, 1, 1, 30)
    info = o.bunch_info()
    assert info["c0"] == 1
    err = wake_err(s, o)
    print("wake error", precision, err)
    assert err <= tol, err
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("fp64", 1e-12)])
def test_window_longer_than_the_box(tetm, precision, tol):
    """sigma = 8 dz on a 12-cell box: the window (-41 .. 120) is far longer than
    the grid, most samples see no plane."""
    nx, ny, nz = 12, 12, 12
    s, o = run_both(tetm, nx, ny, nz, precision, 8 * wl.DZ, 6, 6, 200)
    assert len(s.wake()[0]) == len(o.wake()[0]) > 10 * nz
    err = wake_err(s, o)
    print("wake error", precision, err)
    assert err <= tol, err
    s.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_zero_steps_leave_the_state(tetm, precision):
    w = wl.plain_pipe(nz=20, n=8, steps=0, precision=precision)
    s = tetm.Solver.from_workload(w)
    rng = np.random.default_rng(4)
    init = {c: rng.standard_normal(s.shape) for c in COMPONENTS}
    for c, a in init.items():
        s.set(c, a)
    before = {c: s.get(c) for c in COMPONENTS}
    s.step(0)
    for c in COMPONENTS:
        assert np.array_equal(s.get(c), before[c])
    assert np.all(s.wake()[0] == 0.0) and s.info()["step"] == 0
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-5), ("fp64", 1e-12)])
@pytest.mark.parametrize("dims", [(2, 2, 2), (2, 3, 4), (3, 2, 5)])
def test_smallest_grids_with_random_fields(tetm, precision, tol, dims):
    nx, ny, nz = dims
    s = tetm.Solver(nx, ny, nz, wl.DXY, wl.DXY, wl.DZ, 0.0, precision)
    o = Oracle(nx, ny, nz, wl.DXY, wl.DXY, wl.DZ, 0.0)
    rng = np.random.default_rng(sum(dims))
    for c in COMPONENTS:
        a = rng.standard_normal(s.shape)
        s.set(c, a)
        o.set(c, a)
    s.step(25)
    o.step(25)
    for fam in (("ex", "ey", "ez"), ("hx", "hy", "hz")):
        peak = max(np.max(np.abs(o.get(c))) for c in fam)
        for c in fam:
            assert np.max(np.abs(s.get(c) - o.get(c))) <= tol * peak, c
    s.close()
