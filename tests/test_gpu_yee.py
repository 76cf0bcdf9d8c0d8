"""GPU Yee scheme (Sec. 3, Eq. (7); tetm_set_scheme) against the FP64 oracle
(``Oracle.yee_step``, pinned in tests/test_oracle_yee_pins.py by the dispersion
relation (9), the step bound (8) and the leapfrog energy).

Grids span several tiles of the fused kernel in x and y with ragged tails
(float64 tiles own 60 x 14 nodes, float32 tiles 56 x 30) and several z chunks
(including chunk lengths that do not divide nz); staircase PEC, dielectric and
magnetic materials (which run on the reference updates). Seeded random initial
fields on the entries that carry a field. Tolerances: float64 1e-12 of each
component's peak; float32 5e-5 (a few hundred single-precision roundings of a
field of order one, all steps summed)."""
import math

import numpy as np
import pytest

from oracle import Oracle
from paper_0901_1053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MM = 1e-3
DXY = math.sqrt(2.0) * MM
ETA0 = 376.730313668
TOL64 = 1e-12
TOL32 = 5e-5


@pytest.fixture(scope="module")
def tetm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_1053_gb300 import tetm as t
    return t


def yee_bound(dx, dy, dz):
    return 1.0 / math.sqrt(dx ** -2 + dy ** -2 + dz ** -2)


def initial_fields(o, seed):
    """Random e [V] and h [A] (h scaled by 1/eta0) on the active entries."""
    f = wl.random_fields(o.shape, seed)
    out = []
    for c in range(6):
        a = np.where(o.coef(c) > 0, f[c], 0.0)
        out.append(a / ETA0 if c >= 3 else a)
    return out


def rel_err(a, b):
    peak = np.max(np.abs(b))
    assert peak > 0
    return float(np.max(np.abs(a - b)) / peak)


def run_pair(tetm, nx, ny, nz, precision, steps, kernel="fused", chunk=None, seed=3, frac=0.95,
             pec=None, eps=None, mu=None, dx=DXY, dy=DXY, dz=MM):
    cdt = frac * yee_bound(dx, dy, dz)
    o = Oracle(nx, ny, nz, dx, dy, dz, cdt=cdt, eps_r=eps, mu_r=mu, pec=pec)
    f0 = initial_fields(o, seed)
    s = tetm.Solver(nx, ny, nz, dx, dy, dz, cdt, precision, eps_r=eps, mu_r=mu, pec=pec)
    s.set_scheme("yee")
    s.set_kernel(kernel)
    if chunk:
        s.set_tiling(0, 0, chunk)
    for c in range(6):
        o.set(c, f0[c])
        s.set(c, f0[c])
    o.yee_step(steps)
    s.step(steps)
    s.sync()
    got = [s.get(c) for c in range(6)]
    ref = [o.get(c) for c in range(6)]
    s.close()
    return got, ref


def collimator_pec(nx, ny, nz):
    return wl.radius_mask(nx, ny, nz, wl.collimator_radius(nz, 0.46 * min(nx, ny), 0.25 * min(nx, ny),
                                                           nz // 3, 2 * nz // 3))


@pytest.mark.parametrize("chunk", [None, 4, 13, 80])
def test_yee_fp64_fused_matches_oracle(tetm, chunk):
    """130 x 33 x 70: three tiles in x (60, 60, 10) and three in y (14, 14, 5)."""
    nx, ny, nz = 130, 33, 70
    got, ref = run_pair(tetm, nx, ny, nz, "fp64", 45, chunk=chunk, pec=collimator_pec(nx, ny, nz))
    for c in range(6):
        assert rel_err(got[c], ref[c]) <= TOL64, c


def test_yee_fp64_reference_with_materials_matches_oracle(tetm):
    nx, ny, nz = 37, 29, 33
    eps, mu, pec = wl.random_materials(nx, ny, nz, 8)
    for kernel in ("reference", "fused"):       # material arrays run on the reference updates
        got, ref = run_pair(tetm, nx, ny, nz, "fp64", 30, kernel=kernel, eps=eps, mu=mu, pec=pec,
                            dx=1.3 * MM, dy=1.6 * MM, dz=0.9 * MM, frac=0.9)
        for c in range(6):
            assert rel_err(got[c], ref[c]) <= TOL64, (kernel, c)


def test_yee_fp64_reference_uniform_matches_oracle(tetm):
    nx, ny, nz = 61, 17, 40
    got, ref = run_pair(tetm, nx, ny, nz, "fp64", 35, kernel="reference", pec=collimator_pec(nx, ny, nz))
    for c in range(6):
        assert rel_err(got[c], ref[c]) <= TOL64, c


@pytest.mark.parametrize("chunk", [None, 7])
def test_yee_fp32_fused_matches_oracle(tetm, chunk):
    """120 x 70 x 64 in float32: three tiles in x (56, 56, 8), three in y (30, 30, 10)."""
    nx, ny, nz = 120, 70, 64
    got, ref = run_pair(tetm, nx, ny, nz, "fp32", 40, chunk=chunk, pec=collimator_pec(nx, ny, nz))
    for c in range(6):
        assert rel_err(got[c], ref[c]) <= TOL32, c


def test_yee_fp32_fused_equals_reference_and_is_chunk_independent(tetm):
    nx, ny, nz = 90, 61, 50
    pec = collimator_pec(nx, ny, nz)
    runs = {}
    for kernel, chunk in (("reference", None), ("fused", None), ("fused", 5), ("fused", 64)):
        runs[(kernel, chunk)], ref = run_pair(tetm, nx, ny, nz, "fp32", 25, kernel=kernel, chunk=chunk,
                                              pec=pec, seed=9)
    base = runs[("fused", None)]
    for key in (("fused", 5), ("fused", 64)):
        for c in range(6):
            assert np.array_equal(runs[key][c], base[c]), (key, c)
    for c in range(6):
        assert rel_err(base[c], runs[("reference", None)][c]) <= 1e-6, c
        assert rel_err(base[c], ref[c]) <= TOL32, c


def test_yee_fp32_materials_run_on_reference_updates(tetm):
    nx, ny, nz = 40, 36, 30
    eps, mu, pec = wl.random_materials(nx, ny, nz, 4)
    got, ref = run_pair(tetm, nx, ny, nz, "fp32", 25, eps=eps, mu=mu, pec=pec, frac=0.9)
    for c in range(6):
        assert rel_err(got[c], ref[c]) <= TOL32, c


def test_yee_api_states(tetm):
    nx, ny, nz = 20, 20, 30
    b = yee_bound(DXY, DXY, MM)
    s = tetm.Solver(nx, ny, nz, DXY, DXY, MM, MM, "fp32")       # the TE/TM scheme's magic step
    with pytest.raises(tetm.TetmError) as e:
        s.set_scheme("yee")                                      # beyond Eq. (8)
    assert e.value.code == tetm.TETM_E_UNSTABLE
    with pytest.raises(tetm.TetmError) as e:
        s.set_scheme(7)
    assert e.value.code == tetm.TETM_E_ARG
    s.close()
    s = tetm.Solver(nx, ny, nz, DXY, DXY, MM, 0.99 * b, "fp32")
    info0 = s.info()
    s.set_scheme("yee")
    for call in (lambda: s.energy(), lambda: s.save(), lambda: s.set_balance_every(10),
                 lambda: s.set_bunch(2 * MM, 1e-9, 10, 10), lambda: s.set_tiling(28, 20, 16)):
        with pytest.raises(tetm.TetmError) as e:
            call()
        assert e.value.code == tetm.TETM_E_UNSUPPORTED
    s.set_tiling(0, 0, 16)                                       # the chunk length is free
    s.set_scheme("tetm")                                         # back, before any step
    assert s.info()["tile_x"] == info0["tile_x"] and s.info()["tile_y"] == info0["tile_y"]
    s.set_scheme("yee")
    s.step(2)
    with pytest.raises(tetm.TetmError) as e:
        s.set_scheme("tetm")                                     # after the first step
    assert e.value.code == tetm.TETM_E_STATE
    with pytest.raises(tetm.TetmError) as e:
        tetm.Batch([s], [10])                                    # batches run the TE/TM scheme
    assert e.value.code == tetm.TETM_E_UNSUPPORTED
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp32", TOL32), ("fp64", TOL64)])
def test_yee_full_size_collimator_head_matches_oracle(tetm, precision, tol):
    """256x256x2048 step collimator at Yee's bound, the benchmark's launch
    configuration. The initial field fills planes 0..9 only; one step spreads
    it by at most one plane, so after n steps the oracle on the first 72 planes
    of the same geometry reproduces the full box: planes 0..60 entry by entry,
    nothing beyond plane 11 + n."""
    w = wl.step_collimator(precision=precision)
    n = 40
    cdt = yee_bound(w.dx, w.dy, w.dz)
    o = Oracle(w.nx, w.ny, 72, w.dx, w.dy, w.dz, cdt=cdt, pec=w.pec[:72].copy())
    f0 = initial_fields(o, 31)
    for c in range(6):
        f0[c][10:] = 0.0
        o.set(c, f0[c])
    o.yee_step(n)
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, cdt, precision, pec=w.pec)
    s.set_scheme("yee")
    full = np.zeros((w.nz + 1, w.ny + 1, w.nx + 1))
    for c in range(6):
        full[:73] = f0[c]
        s.set(c, full)
    s.step(n)
    s.sync()
    for c in range(6):
        g = s.get(c)
        r = o.get(c)
        assert np.all(g[12 + n:] == 0.0), c
        assert rel_err(g[:61], r[:61]) <= tol, c
    s.close()
