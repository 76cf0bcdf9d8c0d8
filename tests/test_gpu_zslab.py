"""One solve split along z into slabs on one GPU (tetm_create_slab,
tetm_export_plane, tetm_import_plane, paper_0901_1053_gb300/zslab.py): the
slabs exchange their ghost planes through host buffers before every step and
must reproduce the whole-grid solve: fields bit for bit on every owned plane
(the same arithmetic per plane), the longitudinal and transverse wakes up to
the order of the final sum over slabs (1e-14 of their peak). Slab boundaries
off the kernels' z-chunks, the bunch crossing them, random initial fields."""
import numpy as np
import pytest

from paper_0901_1053_gb300 import workloads as wl
from paper_0901_1053_gb300 import zslab

pytestmark = pytest.mark.gpu

COMPONENTS = ("ex", "ey", "ez", "hx", "hy", "hz")


@pytest.fixture(scope="module")
def tetm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_1053_gb300 import tetm as t
    return t


def collimator(n, nz, precision):
    w = wl.scaled_collimator(n, nz, sigma_cells=3.0, precision=precision)
    w.steps = nz + 30
    return w


def run_whole(tetm, w, init, steps, tiling=None):
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, w.precision, pec=w.pec)
    if tiling:
        s.set_tiling(*tiling)
    for c in COMPONENTS:
        s.set(c, init[c])
    s.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    s.set_observer(w.i0 + 1, w.j0)
    s.step(steps)
    return s


def run_split(tetm, w, init, steps, ranges, tiling=None):
    slabs = []
    for a, b in ranges:
        s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, w.precision, pec=w.pec, k_range=(a, b))
        if tiling:
            s.set_tiling(*tiling)
        for c in COMPONENTS:
            s.set(c, init[c][a:b + 1])
        s.set_bunch(w.sigma, w.charge, w.i0, w.j0)
        s.set_observer(w.i0 + 1, w.j0)
        slabs.append(s)
    chain = zslab.LocalChain(slabs)
    chain.step(steps)
    return chain


@pytest.mark.parametrize("precision,tiling,ranges", [
    ("fp32", None, [(0, 23), (23, 70)]),                     # slab kernel, 56 x 28 x 32
    ("fp32", (28, 20, 16), [(0, 17), (17, 40), (40, 70)]),   # warp-tiled kernel
    ("fp64", None, [(0, 35), (35, 37), (37, 70)]),           # float64 warp kernel, a two-plane slab
])
def test_slabs_reproduce_the_whole_grid(tetm, precision, tiling, ranges):
    w = collimator(40, 70, precision)
    rng = np.random.default_rng(17)
    shape = (w.nz + 1, w.ny + 1, w.nx + 1)
    init = {c: rng.standard_normal(shape) for c in COMPONENTS}
    ref = run_whole(tetm, w, init, w.steps, tiling)
    chain = run_split(tetm, w, init, w.steps, ranges, tiling)
    for (a, b), s in zip(ranges, chain.slabs):
        for c in COMPONENTS:
            got, exp = s.get(c)[: b - a], ref.get(c)[a:b]
            assert np.array_equal(got, exp), (a, b, c, np.max(np.abs(got - exp)))
    wk = chain.wake()[0]
    r = ref.wake()[0]
    assert np.max(np.abs(wk - r)) <= 1e-14 * np.max(np.abs(r))
    tx = sum(s.transverse_wake()[0] for s in chain.slabs)
    rx = ref.transverse_wake()[0]
    assert np.max(np.abs(tx - rx)) <= 1e-14 * np.max(np.abs(rx))


def test_slab_without_exchange_differs(tetm):
    """The comparison is sharp: slabs stepped without their ghost planes differ."""
    w = collimator(40, 70, "fp64")
    w.steps = 20
    rng = np.random.default_rng(3)
    shape = (w.nz + 1, w.ny + 1, w.nx + 1)
    init = {c: rng.standard_normal(shape) for c in COMPONENTS}
    ref = run_whole(tetm, w, init, w.steps)
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp64", pec=w.pec, k_range=(35, 70))
    for c in COMPONENTS:
        s.set(c, init[c][35:71])
    s.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    s.step(w.steps)
    assert not np.array_equal(s.get("ex")[:35], ref.get("ex")[35:70])


def test_slab_limits(tetm):
    w = collimator(24, 40, "fp64")
    lo = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp64", pec=w.pec, k_range=(0, 20))
    hi = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp64", pec=w.pec, k_range=(20, 40))
    buf = np.zeros(lo.plane_bytes(tetm.TETM_PLANES_UP), np.uint8)
    for s, d, code in ((lo, tetm.TETM_PLANES_UP, tetm.TETM_E_STATE),      # nothing below the first slab
                       (hi, tetm.TETM_PLANES_DOWN, tetm.TETM_E_STATE)):   # nothing above the last
        with pytest.raises(tetm.TetmError) as e:
            s.import_plane(d, buf)
        assert e.value.code == code
    with pytest.raises(tetm.TetmError) as e:
        hi.set_kernel("reference")
    assert e.value.code == tetm.TETM_E_UNSUPPORTED
    with pytest.raises(tetm.TetmError) as e:
        hi.set_balance_every(10)
    assert e.value.code == tetm.TETM_E_UNSUPPORTED
    assert lo.plane_bytes(tetm.TETM_PLANES_UP) == 3 * lo.plane_bytes(tetm.TETM_PLANES_DOWN)
    with pytest.raises(tetm.TetmError) as e:
        tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp64", pec=w.pec, k_range=(39, 40))
    assert e.value.code == tetm.TETM_E_ARG
