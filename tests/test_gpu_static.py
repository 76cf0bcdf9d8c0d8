"""GPU parity of the static start (tetm_set_bunch_static): the bunch begins in
a uniform entry pipe with its discrete TEM field (Sec. 4.5, Sec. 5). Checked
against the FP64 oracle's own static start: fields and wake to 1e-12 (FP64),
wake to 1e-4 (FP32); and against physics: in a smooth pipe the field moves
rigidly and the wake vanishes."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from oracle import Oracle
from paper_0901_1053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MM = 1e-3
DXY = math.sqrt(2.0) * MM


@pytest.fixture(scope="module")
def tetm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_1053_gb300 import tetm as t
    return t


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def family_err(s, o):
    g = {c: s.get(c) for c in oracle.COMPONENTS}
    r = {c: o.get(c) for c in oracle.COMPONENTS}
    out = 0.0
    for fam in (("ex", "ey", "ez"), ("hx", "hy", "hz")):
        peak = max(np.max(np.abs(r[c])) for c in fam)
        out = max(out, max(float(np.max(np.abs(g[c] - r[c])) / peak) for c in fam))
    return out


def collimator(n, nz, precision, sigma_cells=2.5):
    """Scaled step collimator: uniform entry pipe for planes k < nz/4."""
    return wl.scaled_collimator(n, nz, sigma_cells=sigma_cells, precision=precision)


@pytest.mark.parametrize("tiling", [None, (28, 12, 16), (32, 8, 64)])
def test_static_start_collimator_matches_oracle_fp64(tetm, tiling):
    w = collimator(40, 120, "fp64")          # entry pipe uniform for k < 30, c0 = 13
    c0 = math.ceil(5 * w.sigma / w.dz - 1e-12)
    K = 2 * c0 + 2
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp64", pec=w.pec)
    if tiling:
        s.set_tiling(*tiling)
    s.set_bunch_static(w.sigma, w.charge, w.i0, w.j0, K)
    o = Oracle(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, pec=w.pec)
    o.set_bunch_static(w.sigma, w.charge, w.i0, w.j0, K)
    assert family_err(s, o) <= 1e-12                 # the initial TEM field
    n = w.nz - K + 2 * c0 + 20
    s.step(n)
    o.step(n)
    assert family_err(s, o) <= 1e-12
    assert rel(s.wake()[0], o.wake()[0]) <= 1e-12


def test_static_start_fp32_wake(tetm):
    w = collimator(48, 200, "fp32", 3.0)
    c0 = math.ceil(5 * w.sigma / w.dz - 1e-12)
    K = 2 * c0 + 4
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp32", pec=w.pec)
    s.set_bunch_static(w.sigma, w.charge, w.i0, w.j0, K)
    o = Oracle(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, pec=w.pec)
    o.set_bunch_static(w.sigma, w.charge, w.i0, w.j0, K)
    n = w.nz - K + 2 * c0 + 40
    s.step(n)
    o.step(n)
    assert rel(s.wake()[0], o.wake()[0]) <= 1e-4


def test_static_start_smooth_pipe_no_wake(tetm):
    nx = ny = 30
    nz = 160
    pec = wl.radius_mask(nx, ny, nz, lambda k: np.full(k.shape, 11.5))
    sigma, q = 3 * MM, 1e-9
    c0 = math.ceil(5 * sigma / MM - 1e-12)
    K = 2 * c0 + 2
    s = tetm.Solver(nx, ny, nz, DXY, DXY, MM, 0.0, "fp64", pec=pec)
    s.set_bunch_static(sigma, q, 15, 15, K)
    f0 = {c: s.get(c) for c in oracle.COMPONENTS}
    n = nz - K - 2
    s.step(n)
    for c in oracle.COMPONENTS:
        shifted = np.zeros_like(f0[c])
        shifted[n:] = f0[c][:-n]
        scale = max(np.max(np.abs(f0["ex"])), 1e-300) if c[0] == "e" else np.max(np.abs(f0["hx"]))
        assert np.max(np.abs(s.get(c) - shifted)) <= 1e-12 * scale, c
    cold = tetm.Solver(nx, ny, nz, DXY, DXY, MM, 0.0, "fp64", pec=pec)
    cold.set_bunch(sigma, q, 15, 15)
    cold.step(n + K)
    assert np.max(np.abs(s.wake()[0])) <= 1e-12 * np.max(np.abs(cold.wake()[0]))


def test_static_start_full_size_collimator_head(tetm):
    """256x256x2048 step collimator, float32, benchmark tiling: the static
    field and 60 steps of it against the oracle on the first 160 planes."""
    w = wl.step_collimator(precision="fp32")
    c0 = math.ceil(5 * w.sigma / w.dz - 1e-12)
    K = 2 * c0 + 8
    n = 60
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp32", pec=w.pec)
    s.set_tiling(28, 20, 32)
    s.set_bunch_static(w.sigma, w.charge, w.i0, w.j0, K)
    s.step(n)
    head = dataclasses.replace(w, nz=K + n + 20, pec=w.pec[:K + n + 20].copy())
    o = Oracle(head.nx, head.ny, head.nz, head.dx, head.dy, head.dz, head.cdt, pec=head.pec)
    o.set_bunch_static(w.sigma, w.charge, w.i0, w.j0, K)
    o.step(n)
    rows = K + n + 1
    for fam in (("ex", "ey", "ez"), ("hx", "hy", "hz")):
        g = {c: s.get(c)[:rows] for c in fam}
        r = {c: o.get(c)[:rows] for c in fam}
        peak = max(np.max(np.abs(r[c])) for c in fam)
        for c in fam:
            assert np.max(np.abs(g[c] - r[c])) <= 2e-5 * peak, c


def test_static_start_errors(tetm):
    w = collimator(24, 80, "fp64", 3.0)
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp64", pec=w.pec)
    with pytest.raises(tetm.TetmError) as e:
        s.set_bunch_static(w.sigma, w.charge, w.i0, w.j0, 50)   # entry pipe ends at k = 20
    assert e.value.code == tetm.TETM_E_ARG
    with pytest.raises(tetm.TetmError):
        s.set_bunch_static(w.sigma, w.charge, w.i0, w.j0, 5)    # K < 2 c0 + 2
    s.step(1)
    with pytest.raises(tetm.TetmError) as e:
        s.set_bunch_static(w.sigma, w.charge, w.i0, w.j0, 18)
    assert e.value.code == tetm.TETM_E_STATE
    eps = np.ones((w.nz, w.ny, w.nx)) * 2.0
    s2 = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp64", eps_r=eps, pec=w.pec)
    with pytest.raises(tetm.TetmError) as e:
        s2.set_bunch_static(w.sigma, w.charge, w.i0, w.j0, 18)
    assert e.value.code == tetm.TETM_E_UNSUPPORTED


def test_static_start_checkpoint_round_trip(tetm):
    w = collimator(32, 160, "fp64", 3.0)
    c0 = math.ceil(5 * w.sigma / w.dz - 1e-12)
    K = 2 * c0 + 2
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp64", pec=w.pec)
    s.set_bunch_static(w.sigma, w.charge, w.i0, w.j0, K)
    s.step(30)
    blob = s.save()
    s.step(40)
    ref = s.wake()[0]
    s2 = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp64", pec=w.pec)
    s2.set_bunch_static(w.sigma, w.charge, w.i0, w.j0, K)
    s2.load(blob)
    s2.step(40)
    np.testing.assert_array_equal(s2.wake()[0], ref)
