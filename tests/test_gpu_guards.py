"""The canary of out-of-place writes (tetm_check_guards): after runs of every
kernel path on ragged grids with staircase PEC, no entry that carries no field
(the zero guard ring around the cells, the entries of PEC objects) holds a
value, in either field set. The detector itself is checked with a checkpoint
whose guard entry was set on the host."""
import math

import numpy as np
import pytest

from paper_0901_1053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

COMPONENTS = ("ex", "ey", "ez", "hx", "hy", "hz")


@pytest.fixture(scope="module")
def tetm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_1053_gb300 import tetm as t
    return t


def collimator(nx, ny, nz):
    r = min(nx, ny)
    return wl.radius_mask(nx, ny, nz, wl.collimator_radius(nz, 0.45 * r, 0.2 * r, nz // 4, nz // 2))


def randomise(s, seed):
    rng = np.random.default_rng(seed)
    for c in COMPONENTS:
        s.set(c, rng.standard_normal(s.shape))


CASES = [
    ("fp32", None, None, False),                  # slab kernel
    ("fp32", (28, 20, 16), None, False),          # warp-tiled
    ("fp32", (32, 8, 7), None, False),            # block-tiled
    ("fp32", None, "materials", False),           # slab kernel with coefficient arrays
    ("fp32", (28, 12, 16), "materials", False),   # warp-tiled with coefficient arrays
    ("fp64", None, None, False),                  # warp-tiled (float64)
    ("fp64", None, "reference", False),           # one launch per update
    ("fp32", None, None, True),                   # Yee, fused
    ("fp64", None, None, True),
    ("fp32", None, "materials", True),            # Yee on the reference updates
]


@pytest.mark.parametrize("precision,tiling,variant,yee", CASES)
def test_no_write_lands_outside_the_field_entries(tetm, precision, tiling, variant, yee):
    nx, ny, nz = 130, 61, 45
    pec = collimator(nx, ny, nz)
    eps = mu = None
    if variant == "materials":
        eps, mu, pec2 = wl.random_materials(nx, ny, nz, 3)
        pec = np.maximum(pec, pec2)
    cdt = 0.0
    if yee:
        cdt = 0.95 / math.sqrt(2.0 / wl.DXY ** 2 + 1.0 / wl.DZ ** 2)
    s = tetm.Solver(nx, ny, nz, wl.DXY, wl.DXY, wl.DZ, cdt, precision, eps_r=eps, mu_r=mu, pec=pec)
    if yee:
        s.set_scheme("yee")
    if variant == "reference":
        s.set_kernel("reference")
    if tiling:
        s.set_tiling(*tiling)
    randomise(s, nx + ny + nz)
    if not yee:
        s.set_bunch(2.5 * wl.DZ, 1e-9, nx // 2, ny // 2)
    s.step(nz + 13)
    s.sync()
    assert s.check_guards() == 0
    s.close()


def test_static_start_and_observer_keep_the_guards(tetm):
    nx, ny, nz = 70, 66, 90
    w = wl.scaled_collimator(max(nx, ny), nz, sigma_cells=2.5, precision="fp32")
    r = min(nx, ny)
    pec = wl.radius_mask(nx, ny, nz, wl.collimator_radius(nz, 0.45 * r, 0.2 * r, 45, 70))
    s = tetm.Solver(nx, ny, nz, w.dx, w.dy, w.dz, w.cdt, "fp32", pec=pec)
    k_head = 2 * math.ceil(5 * w.sigma / w.dz - 1e-12) + 2     # inside the uniform entry section
    s.set_bunch_static(w.sigma, w.charge, nx // 2, ny // 2, k_head)
    s.set_observer(nx // 2 + 1, ny // 2)
    s.step(80)
    s.sync()
    assert s.check_guards() == 0
    s.close()


def layout_count(nx, ny, nz, esz):
    """Entries per device array: planes -1..nz+1, rows -2..ny+1, padded rows."""
    ox = 8 if esz == 4 else 2
    align = 16 if esz == 4 else 32 // esz
    px = -(-(ox + nx + 3) // align) * align
    return (nz + 3) * (ny + 4) * px


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_the_canary_sees_a_value_in_the_guard_ring(tetm, precision):
    nx, ny, nz = 20, 18, 24
    s = tetm.Solver(nx, ny, nz, wl.DXY, wl.DXY, wl.DZ, 0.0, precision)
    randomise(s, 5)
    s.step(3)
    assert s.check_guards() == 0
    buf = bytearray(s.save())
    esz = 4 if precision == "fp32" else 8
    fb = layout_count(nx, ny, nz, esz) * esz
    header = len(buf) - 6 * fb                   # no bunch: no wake accumulators
    assert header > 0
    one = np.array([1.0], dtype=np.float32 if esz == 4 else np.float64).tobytes()
    buf[header:header + esz] = one               # e_x at (i, j, k) = (-ox, -2, -1): guard
    t = tetm.Solver(nx, ny, nz, wl.DXY, wl.DXY, wl.DZ, 0.0, precision)
    t.load(np.frombuffer(bytes(buf), dtype=np.uint8))
    assert t.check_guards() == 1
    s.close()
    t.close()


@pytest.mark.parametrize("kernel", ["async", "register", "bulk", "bulk2"])
@pytest.mark.parametrize("start", ["cold", "scattered"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_rz_kernels_keep_the_guards(tetm, kernel, start, precision):
    """Every r-z step kernel, cold and in the scattered-field form, modes 0..2,
    on a two-cell chain whose radial size leaves a ragged last window."""
    w = wl.cavity_chain_rz(70, 160, 0, 2, sigma_cells=3.0, precision=precision, n_cells=2, i0=3)
    s = tetm.RzSolver(w.nr, w.nz, w.m_lo, w.m_hi, w.dr, w.dz, w.cdt, precision, pec=w.pec)
    s.set_kernel(kernel)
    if start == "cold":
        s.set_bunch(w.sigma, w.charge, w.i0)
    else:
        s.set_bunch_scattered(w.sigma, w.charge, w.i0, 2 * math.ceil(5 * w.sigma / w.dz - 1e-12) + 2)
    s.step(w.nz // 2 + 1)
    s.sync()
    assert s.check_guards() == 0
    s.close()
