"""Material arrays of the rotationally symmetric solver (Sec. 4.3, Eq. (24)
with per-cell eps_r, mu_r): the per-radian material matrices built on the
device from the staircase averages must reproduce the float64 oracle's
fields and wakes to 1e-12 for every mode (ring bunch and a random initial
state), its energy and charges, and the periodic balances; float32 wakes
within 1e-4 of their peak; arrays of ones are the vacuum; the options that
need one material are refused."""
import numpy as np
import pytest

from oracle import RzOracle
from paper_0901_1053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
NAMES = ("er", "ephi", "ez", "hr", "hphi", "hz")


@pytest.fixture(scope="module")
def tetm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_1053_gb300 import tetm as t
    return t


def dielectric_chain(nr, nz, m_lo, m_hi, precision, seed, i0=4):
    """The two-cell chain with a random eps_r in [1, 4) and mu_r in [1, 2)
    per cell outside a clear beam channel of radius i0 + 3 cells."""
    w = wl.cavity_chain_rz(nr, nz, m_lo, m_hi, sigma_cells=2.5, precision=precision, n_cells=2, i0=i0)
    rng = np.random.default_rng(seed)
    eps = rng.uniform(1.0, 4.0, (nz, nr))
    mu = rng.uniform(1.0, 2.0, (nz, nr))
    eps[:, : i0 + 3] = 1.0
    mu[:, : i0 + 3] = 1.0
    return w, eps, mu


def fam_err(g, o):
    out = 0.0
    for fam in (NAMES[:3], NAMES[3:]):
        peak = max(np.max(np.abs(o[c])) for c in fam)
        for c in fam:
            out = max(out, float(np.max(np.abs(g[c] - o[c])) / peak))
    return out


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("chunk", [7, 32])
def test_ring_bunch_in_a_dielectric_chain_matches_oracle(tetm, chunk):
    w, eps, mu = dielectric_chain(36, 90, 0, 2, "fp64", 5)
    s = tetm.RzSolver(w.nr, w.nz, w.m_lo, w.m_hi, w.dr, w.dz, w.cdt, "fp64", pec=w.pec, eps_r=eps, mu_r=mu)
    assert s.info()["kernel"] == tetm.TETM_RZ_KERNEL_REGISTER
    s.set_tiling(chunk)
    s.set_bunch(w.sigma, w.charge, w.i0)
    s.step(w.steps)
    for m in range(3):
        o = RzOracle(w.nr, w.nz, m, w.dr, w.dz, w.cdt, eps_r=eps, mu_r=mu, pec=w.pec)
        o.set_bunch(w.sigma, w.charge, w.i0)
        o.step(w.steps)
        assert fam_err(s.fields(m), o.fields()) <= TOL64, m
        wo = o.wake()[0]
        assert np.max(np.abs(wo)) > 0
        assert rel(s.wake(m)[0], wo) <= TOL64, m
    s.close()


def test_random_state_energy_and_charges_match_oracle(tetm):
    """Random fields of mode 1 (set_fields keeps what the geometry makes
    active), 40 steps: fields, energy and both charge maxima as the oracle's."""
    w, eps, mu = dielectric_chain(30, 60, 1, 1, "fp64", 9)
    s = tetm.RzSolver(w.nr, w.nz, 1, 1, w.dr, w.dz, w.cdt, "fp64", pec=w.pec, eps_r=eps, mu_r=mu)
    o = RzOracle(w.nr, w.nz, 1, w.dr, w.dz, w.cdt, eps_r=eps, mu_r=mu, pec=w.pec)
    rng = np.random.default_rng(12)
    for c in NAMES:
        a = rng.standard_normal(o.shape)
        s.set(1, c, a)
        o.set(c, a)
        np.testing.assert_array_equal(s.get(1, c), o.get(c))
    assert s.energy(1) == pytest.approx(o.energy(), rel=TOL64)
    s.step(39)
    o.step(39)
    f0 = o.fields()
    s.step(1)
    o.step(1)
    assert fam_err(s.fields(1), o.fields()) <= TOL64
    assert s.energy(1) == pytest.approx(o.energy(), rel=TOL64)
    f1 = o.fields()
    qe = o.qbar_e(f1["er"], f0["er"], f1["ephi"], f0["ephi"], f1["ez"])
    qh = o.qbar_h(f1["hphi"], f0["hphi"], f1["hr"], f0["hr"], f0["hz"])
    me, mh, _ = s.charge_residual(1)
    # the device takes the maxima over the nodes (cells) whose every edge
    # (face) carries a field; the oracle's charges there are the same values
    a = {c: o.coef(c) != 0 for c in NAMES}
    node = a["ez"].copy()
    node[1:, :] &= a["ez"][:-1, :]
    node[0, :] = False
    node &= a["er"] & a["ephi"]
    node[:, 1:] &= a["er"][:, :-1]
    cell = a["hz"].copy()
    cell[:-1, :] &= a["hz"][1:, :]
    cell[-1, :] = False
    outward = np.zeros_like(cell)
    outward[:, :-1] = a["hr"][:, 1:]
    inward = a["hr"].copy()
    inward[:, 0] = True
    cell &= outward & inward & a["hphi"]
    ref_e, ref_h = float(np.max(np.abs(qe[node]))), float(np.max(np.abs(qh[cell])))
    assert ref_e > 0 and ref_h > 0
    assert abs(me - ref_e) <= TOL64 * ref_e, (me, ref_e)
    assert abs(mh - ref_h) <= TOL64 * ref_h, (mh, ref_h)
    s.close()


def test_periodic_balances_with_materials(tetm):
    """Bunch from a cold start: every record's charge residual is roundoff
    (below 1e-12 of the bunch charge) and the energy is the oracle's."""
    w, eps, mu = dielectric_chain(30, 70, 0, 1, "fp64", 21)
    s = tetm.RzSolver(w.nr, w.nz, 0, 1, w.dr, w.dz, w.cdt, "fp64", pec=w.pec, eps_r=eps, mu_r=mu)
    s.set_bunch(w.sigma, w.charge, w.i0)
    s.set_balance_every(10)
    s.step(60)
    rows = s.balance_history()
    assert len(rows) == 12
    for r in rows:
        assert r[3] <= 1e-12 * abs(w.charge) and r[4] <= 1e-12 * abs(w.charge), r
    for m in (0, 1):
        o = RzOracle(w.nr, w.nz, m, w.dr, w.dz, w.cdt, eps_r=eps, mu_r=mu, pec=w.pec)
        o.set_bunch(w.sigma, w.charge, w.i0)
        o.step(60)
        last = rows[(rows[:, 0] == 60) & (rows[:, 1] == m)][0]
        assert last[2] == pytest.approx(o.energy(), rel=TOL64)
    s.close()


def test_fp32_wakes_in_a_dielectric_chain(tetm):
    w, eps, mu = dielectric_chain(40, 120, 0, 2, "fp32", 33)
    s = tetm.RzSolver(w.nr, w.nz, 0, 2, w.dr, w.dz, w.cdt, "fp32", pec=w.pec, eps_r=eps, mu_r=mu)
    s.set_bunch(w.sigma, w.charge, w.i0)
    s.step(w.steps)
    for m in range(3):
        o = RzOracle(w.nr, w.nz, m, w.dr, w.dz, w.cdt, eps_r=eps, mu_r=mu, pec=w.pec)
        o.set_bunch(w.sigma, w.charge, w.i0)
        o.step(w.steps)
        err = rel(s.wake(m)[0], o.wake()[0])
        print("m", m, "fp32 wake error", err)
        assert err <= 1e-4, (m, err)
    s.close()


def test_unit_arrays_are_the_vacuum_and_limits(tetm):
    w, eps, mu = dielectric_chain(24, 40, 0, 1, "fp64", 2)
    ones = np.ones((w.nz, w.nr))
    v = tetm.RzSolver(w.nr, w.nz, 0, 1, w.dr, w.dz, w.cdt, "fp64", pec=w.pec, eps_r=ones, mu_r=ones)
    p = tetm.RzSolver(w.nr, w.nz, 0, 1, w.dr, w.dz, w.cdt, "fp64", pec=w.pec)
    assert v.info()["kernel"] == p.info()["kernel"]
    for s in (v, p):
        s.set_bunch(w.sigma, w.charge, w.i0)
        s.step(30)
    for m in (0, 1):
        np.testing.assert_array_equal(v.wake(m)[0], p.wake(m)[0])
    m_ = tetm.RzSolver(w.nr, w.nz, 0, 1, w.dr, w.dz, w.cdt, "fp64", pec=w.pec, eps_r=eps)
    for kern in ("async", "bulk", "bulk2"):
        with pytest.raises(tetm.TetmError) as e:
            m_.set_kernel(kern)
        assert e.value.code == tetm.TETM_E_UNSUPPORTED
    m_.set_kernel("register")
    with pytest.raises(tetm.TetmError) as e:
        m_.set_bunch_static(w.sigma, w.charge, w.i0, 20)
    assert e.value.code == tetm.TETM_E_UNSUPPORTED
    bad = eps.copy()
    bad[3, 3] = 0.5
    with pytest.raises(tetm.TetmError) as e:
        tetm.RzSolver(w.nr, w.nz, 0, 1, w.dr, w.dz, w.cdt, "fp64", pec=w.pec, eps_r=bad)
    assert e.value.code == tetm.TETM_E_ARG
    for s in (v, p, m_):
        s.close()
