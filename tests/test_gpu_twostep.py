"""Two steps per pass (TETM_KERNEL_TWOSTEP, temporal blocking of the sweep):
Eq. (23) applied twice per pass over the fields must give the fields of the
one-step block-tiled kernel bit for bit (the same arithmetic per node), the
float64 oracle's fields and wakes to 1e-12, and the same periodic balances;
ragged grids, short chunks (every chunk boundary inside the bunch's path),
random initial fields, the bunch on."""
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


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def make(tetm, w, init, tile, kernel):
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, w.precision, pec=w.pec)
    s.set_tiling(*tile)
    s.set_kernel(kernel)
    for c in COMPONENTS:
        s.set(c, init[c])
    s.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    return s


def collimator(nx, nz, precision):
    w = wl.scaled_collimator(nx, nz, sigma_cells=3.0, precision=precision)
    w.steps = nz + 25
    return w


@pytest.mark.parametrize("precision,tile", [("fp32", (32, 4, 5)), ("fp32", (32, 8, 7)), ("fp32", (64, 4, 32)),
                                            ("fp64", (32, 4, 6)), ("fp64", (32, 8, 5)), ("fp64", (64, 4, 9))])
def test_two_steps_equal_the_one_step_kernel(tetm, precision, tile):
    w = collimator(42, 50, precision)
    rng = np.random.default_rng(5)
    shape = (w.nz + 1, w.ny + 1, w.nx + 1)
    init = {c: rng.standard_normal(shape) for c in COMPONENTS}
    one = make(tetm, w, init, tile, "fused")
    two = make(tetm, w, init, tile, "twostep")
    for n in (7, 2, 1, 40, 25):       # odd and even calls: pairs, then single steps
        one.step(n)
        two.step(n)
    assert two.info()["step"] == one.info()["step"] == w.steps
    for c in COMPONENTS:
        assert np.array_equal(two.get(c), one.get(c)), c
    assert rel(two.wake()[0], one.wake()[0]) <= 1e-13
    for s in (one, two):
        assert s.check_guards() == 0
    e1, e2 = one.energy(), two.energy()
    assert abs(e1 - e2) <= 1e-12 * abs(e1)
    one.close()
    two.close()


def test_two_steps_against_the_oracle(tetm):
    w = collimator(30, 40, "fp64")
    rng = np.random.default_rng(9)
    shape = (w.nz + 1, w.ny + 1, w.nx + 1)
    init = {c: rng.standard_normal(shape) for c in COMPONENTS}
    s = make(tetm, w, init, (32, 4, 6), "twostep")
    o = Oracle(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, pec=w.pec)
    for c in COMPONENTS:
        o.set(c, init[c])
    o.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    s.step(w.steps)
    o.step(w.steps)
    for c in COMPONENTS:
        assert rel(s.get(c), o.get(c)) <= 1e-12, c
    assert rel(s.wake()[0], o.wake()[0]) <= 1e-12
    s.close()


def test_two_steps_keep_the_balances(tetm):
    """Balances every 5 steps: pairs stop short of each balance step (which
    keeps the state before it for the charges), and the recorded history
    equals the one-step kernel's."""
    w = collimator(36, 48, "fp64")
    w.steps = 40
    init = {c: np.zeros((w.nz + 1, w.ny + 1, w.nx + 1)) for c in COMPONENTS}
    one = make(tetm, w, init, (32, 8, 8), "fused")
    two = make(tetm, w, init, (32, 8, 8), "twostep")
    for s in (one, two):
        s.set_balance_every(5)
        s.step(w.steps)
    h1, h2 = one.balance_history(), two.balance_history()
    assert len(h1) == len(h2) == 8
    assert np.array_equal(h2, h1)    # the same fields, balanced by the same kernels
    one.close()
    two.close()


def test_two_step_limits(tetm):
    w = collimator(30, 40, "fp32")
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp32", pec=w.pec)
    with pytest.raises(tetm.TetmError) as e:    # the default shape is the slab kernel's
        s.set_kernel("twostep")
    assert e.value.code == tetm.TETM_E_UNSUPPORTED
    s.set_tiling(32, 8, 16)
    s.set_kernel("twostep")
    with pytest.raises(tetm.TetmError) as e:    # a shape the two-step sweep does not have
        s.set_tiling(32, 16, 16)
    assert e.value.code == tetm.TETM_E_UNSUPPORTED
    with pytest.raises(tetm.TetmError) as e:
        s.set_scheme("yee")
    assert e.value.code == tetm.TETM_E_UNSUPPORTED
    eps = np.ones((w.nz, w.ny, w.nx))
    eps[:, :, : w.nx // 2] = 2.0
    m = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp32", eps_r=eps, pec=w.pec)
    m.set_tiling(28, 20, 16)
    with pytest.raises(tetm.TetmError) as e:    # one material only
        m.set_kernel("twostep")
    assert e.value.code == tetm.TETM_E_UNSUPPORTED
    s.close()
    m.close()
