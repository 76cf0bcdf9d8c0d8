"""GPU float64 balances as the periodic path runs them (tetm_set_balance_every,
tetm_balance_history): the discrete energy of Sec. 4.4 and the charge
residuals of Eqs. (35) and (34), record by record, against the oracle's
energy() and qbar_e / qbar_h of the same states.

With a random initial field the electric and magnetic "charges" of Eqs. (35)
and (34) are O(1) quantities that the scheme carries unchanged, so the
recorded maxima are sharp values (not roundoff) that GPU and oracle must
agree on to 1e-12 of their size. With the bunch on from a cold start the
residual is roundoff and must stay below 1e-12 of the bunch charge.
"""
import numpy as np
import pytest

import oracle as orc
from oracle import Oracle
from paper_0901_1053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def tetm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_1053_gb300 import tetm as t
    return t


def interior_nodes(o):
    """Nodes with all six incident edges non-PEC (where Eq. (35) is checked)."""
    a = [o.coef(c) != 0 for c in range(3)]
    m = np.zeros(o.shape, bool)
    m[1:, 1:, 1:] = (a[0][1:, 1:, 1:] & a[0][1:, 1:, :-1] & a[1][1:, 1:, 1:] & a[1][1:, :-1, 1:] &
                     a[2][1:, 1:, 1:] & a[2][:-1, 1:, 1:])
    return m


def interior_cells(o):
    """Cells (by their lower node) with all six faces non-PEC (Eq. (34))."""
    a = [o.coef(c) != 0 for c in range(3, 6)]
    m = np.zeros(o.shape, bool)
    m[:-1, :-1, :-1] = (a[0][:-1, :-1, :-1] & a[0][:-1, :-1, 1:] & a[1][:-1, :-1, :-1] &
                        a[1][:-1, 1:, :-1] & a[2][:-1, :-1, :-1] & a[2][1:, :-1, :-1])
    return m


def random_fields(o, seed):
    """N(0,1) values on the entries that carry a field, zero elsewhere."""
    rng = np.random.default_rng(seed)
    return {c: rng.standard_normal(o.shape) * (o.coef(c) != 0) for c in orc.COMPONENTS}


def oracle_balances(o, f1, f0):
    """(energy, max |qe|, max |qh|) of the state f1 following f0, no bunch,
    and the largest electric and magnetic edge flux (M e, M h) of f1."""
    for c in orc.COMPONENTS:
        o.set(c, f1[c])
    qe = o.qbar_e(f1["ex"], f0["ex"], f1["ey"], f0["ey"], f1["ez"])
    qh = o.qbar_h(f1["hx"], f0["hx"], f1["hy"], f0["hy"], f0["hz"])

    def flux(c):
        m = o.coef(c)
        return float(np.max(np.abs(f1[c][m != 0] / m[m != 0])))
    return (o.energy(), float(np.max(np.abs(qe[interior_nodes(o)]))),
            float(np.max(np.abs(qh[interior_cells(o)]))), flux("ex"), flux("hx"))


def close(a, b, tol=TOL64):
    return abs(a - b) <= tol * abs(b), (a, b, abs(a - b) / abs(b))


@pytest.mark.parametrize("eps", [False, True], ids=["vacuum", "materials"])
def test_periodic_balances_fp64_random_field(tetm, eps):
    """Every record of the periodic history (float64 fields, every 5 steps)
    against the oracle run side by side from the same random field."""
    w = wl.scaled_collimator(40, 48, sigma_cells=3.0, precision="fp64")
    eps_r = None
    if eps:
        eps_r = 1.0 + 2.0 * np.random.default_rng(5).random((w.nz, w.ny, w.nx))
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp64", eps_r=eps_r, pec=w.pec)
    o = Oracle(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, eps_r=eps_r, pec=w.pec)
    f = random_fields(o, 41)
    for c in orc.COMPONENTS:
        s.set(c, f[c])
        o.set(c, f[c])
    s.set_balance_every(5)
    s.step(23)
    hist = s.balance_history()
    assert [int(r[0]) for r in hist] == [5, 10, 15, 20]
    chk = Oracle(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, eps_r=eps_r, pec=w.pec)
    done = 0
    for rec in hist:
        n = int(rec[0])
        o.step(n - 1 - done)
        f0 = o.fields()
        o.step(1)
        done = n
        ew, ee, eh, de, bh = oracle_balances(chk, o.fields(), f0)
        assert ee > 0.1 * de and eh > 0.1 * bh    # charges of the size of the fluxes: a sharp comparison
        for got, ref in ((rec[1], ew), (rec[2], ee), (rec[3], eh)):
            ok, info = close(got, ref)
            assert ok, (n, info)


@pytest.mark.parametrize("eps", [False, True], ids=["vacuum", "materials"])
def test_periodic_balances_fp32_fields_against_oracle_on_the_same_state(tetm, eps):
    """Float32 fields (the benchmark's precision), one material or per-cell
    eps_r: each record equals the oracle's float64 energy and charges
    evaluated on the GPU's own float32 states (read back exactly), to 1e-12."""
    w = wl.scaled_collimator(40, 48, sigma_cells=3.0, precision="fp32")
    eps_r = None
    if eps:
        eps_r = 1.0 + 2.0 * np.random.default_rng(6).random((w.nz, w.ny, w.nx))
    s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp32", eps_r=eps_r, pec=w.pec)
    chk = Oracle(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, eps_r=eps_r, pec=w.pec)
    f = random_fields(chk, 43)
    for c in orc.COMPONENTS:
        s.set(c, f[c])
    s.set_balance_every(4)
    for target in (4, 12, 20):
        s.step(target - 1 - s.info()["step"])
        f0 = s.fields()
        s.step(1)
        rec = s.balance_history()[-1]
        assert int(rec[0]) == target
        ew, ee, eh, de, bh = oracle_balances(chk, s.fields(), f0)
        assert ee > 0.1 * de and eh > 0.1 * bh
        for got, ref in ((rec[1], ew), (rec[2], ee), (rec[3], eh)):
            ok, info = close(got, ref)
            assert ok, (target, info)


def test_periodic_balances_with_bunch_fp64(tetm):
    """Cold start with the bunch: recorded energies equal the oracle's at the
    same steps; the charge residuals of Eq. (35) (after the bunch's own
    charge) and of Eq. (34) stay below 1e-12 of the bunch charge; the
    recorded charge scale is the bunch's largest node charge."""
    w = wl.scaled_collimator(40, 80, sigma_cells=3.0, precision="fp64")
    s = tetm.Solver.from_workload(w)
    s.set_balance_every(15)
    s.step(75)
    hist = s.balance_history()
    assert [int(r[0]) for r in hist] == [15, 30, 45, 60, 75]
    o = Oracle(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, pec=w.pec)
    o.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    done = 0
    qcell = o.bunch_info()["qcell"]
    for rec in hist:
        n = int(rec[0])
        o.step(n - done)
        done = n
        ok, info = close(rec[1], o.energy())
        assert ok, (n, info)
        assert rec[4] > 0.1 * np.max(qcell)
        assert rec[2] <= 1e-12 * rec[4] and rec[3] <= 1e-12 * rec[4], (n, rec)
