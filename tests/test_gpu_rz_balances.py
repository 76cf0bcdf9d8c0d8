"""GPU balances and checkpoints of the rotationally symmetric solver (Sec. 4.3,
Eq. (24)): the charges of every azimuthal mode (tetm_rz_charge_residual, the
analogue of Eqs. (35)/(34) per mode) and the energy (Sec. 4.4), directly and
through the periodic history (tetm_rz_set_balance_every), against the oracle's
rz qbar_e / qbar_h / energy of the same states; tetm_rz_save / tetm_rz_load
as a bitwise split run.

With a random initial field the charges are flux-sized quantities that the
scheme carries unchanged, so they are compared as values (1e-12 of their
size); with the bunch from a cold start the residual against the bunch's
share of its node charges is roundoff, below 1e-12 of the bunch charge.
"""
import math

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


def chain(nr, nz, m_lo, m_hi, precision, i0=None):
    return wl.cavity_chain_rz(nr, nz, m_lo, m_hi, sigma_cells=2.5, precision=precision, n_cells=2, i0=i0)


def interior_nodes(o):
    a = {c: o.coef(c) != 0 for c in NAMES}
    ok = a["ez"].copy()
    ok[1:, :] &= a["ez"][:-1, :]
    ok[0, :] = False
    ok &= a["er"]
    inward = np.ones_like(ok)
    inward[:, 1:] = a["er"][:, :-1]
    ok &= inward
    if o.m > 0:
        ok &= a["ephi"]
    return ok


def interior_cells(o):
    a = {c: o.coef(c) != 0 for c in NAMES}
    ok = a["hz"].copy()
    ok[:-1, :] &= a["hz"][1:, :]
    ok[-1, :] = False
    outward = np.zeros_like(ok)
    outward[:, :-1] = a["hr"][:, 1:]
    ok &= outward
    inward = a["hr"].copy()
    inward[:, 0] = True
    ok &= inward
    if o.m > 0:
        ok &= a["hphi"]
    return ok


def oracle_charges(o, f1, f0):
    """(energy, max |qe|, max |qh|) of the state f1 following f0 (no bunch),
    the oracle of mode o.m set to f1."""
    for c in NAMES:
        o.set(c, f1[c])
    qe = o.qbar_e(f1["er"], f0["er"], f1["ephi"], f0["ephi"], f1["ez"])
    qh = o.qbar_h(f1["hphi"], f0["hphi"], f1["hr"], f0["hr"], f0["hz"])
    return o.energy(), float(np.max(np.abs(qe[interior_nodes(o)]))), float(np.max(np.abs(qh[interior_cells(o)])))


def close(a, b, tol=TOL64):
    return abs(a - b) <= tol * abs(b), (a, b, abs(a - b) / abs(b))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_rz_balances_of_a_random_field_every_mode(tetm, precision):
    """Modes 0..3 from a random field: every periodic record (every 5 steps,
    the two-step kernel, which takes single steps into the records) equals the
    oracle's energy and charges of the GPU's own states, read back exactly."""
    w = chain(30, 80, 0, 3, precision)
    s = tetm.RzSolver(w.nr, w.nz, w.m_lo, w.m_hi, w.dr, w.dz, w.cdt, precision, pec=w.pec)
    s.set_kernel("bulk2")
    rng = np.random.default_rng(71)
    oracles = {m: RzOracle(w.nr, w.nz, m, w.dr, w.dz, w.cdt, pec=w.pec) for m in range(4)}
    for m in range(4):
        for c in NAMES:
            s.set(m, c, rng.standard_normal(s.shape) * (oracles[m].coef(c) != 0))
    s.set_balance_every(5)
    for target in (5, 15):
        s.step(target - 1 - s.info()["step"])
        f0 = {m: s.fields(m) for m in range(4)}
        s.step(1)
        rows = s.balance_history()
        rows = rows[rows[:, 0] == target]
        assert sorted(int(r[1]) for r in rows) == [0, 1, 2, 3]
        for r in rows:
            m = int(r[1])
            ew, ee, eh = oracle_charges(oracles[m], s.fields(m), f0[m])
            assert ee > 0 and eh > 0
            for got, ref in ((r[2], ew), (r[3], ee), (r[4], eh)):
                ok, info = close(got, ref)
                assert ok, (target, m, info)
            e, h, q = s.charge_residual(m)
            assert (e, h, q) == (r[3], r[4], 0.0)


@pytest.mark.parametrize("kernel", ["async", "bulk2"])
def test_rz_charge_residual_with_the_bunch(tetm, kernel):
    """Cold start, bunch on the ring i0 = 3 (modes 0..2), float64: the node
    charge equals the bunch's share of its node charges to 1e-12 of the bunch
    charge, the cell charge stays zero; periodic records at odd steps under
    the two-step kernel; the recorded energy equals the oracle's."""
    w = chain(24, 90, 0, 2, "fp64", i0=3)
    s = tetm.RzSolver(w.nr, w.nz, w.m_lo, w.m_hi, w.dr, w.dz, w.cdt, "fp64", pec=w.pec)
    s.set_kernel(kernel)
    s.set_bunch(w.sigma, w.charge, w.i0)
    s.set_balance_every(7)
    s.step(64)
    rows = s.balance_history()
    steps = sorted({int(r[0]) for r in rows})
    assert steps == [7, 14, 21, 28, 35, 42, 49, 56, 63]
    for m in range(3):
        o = RzOracle(w.nr, w.nz, m, w.dr, w.dz, w.cdt, pec=w.pec)
        o.set_bunch(w.sigma, w.charge, w.i0)
        # the share of the largest node charge of the bunch (centre on a node)
        scale = (1.0 if m == 0 else 2.0) / (2 * np.pi) * w.charge * math.erf(0.5 * w.dz / (w.sigma * math.sqrt(2)))
        done = 0
        for r in rows[rows[:, 1] == m]:
            n = int(r[0])
            o.step(n - done)
            done = n
            ok, info = close(r[2], o.energy())
            assert ok, (m, n, info)
            assert 0 < r[5] <= scale * (1 + 1e-12)
            assert r[3] <= 1e-12 * scale and r[4] <= 1e-12 * scale, (m, n, r)
        assert np.max(rows[rows[:, 1] == m][:, 5]) > 0.5 * scale


def test_rz_charge_residual_scattered_form(tetm):
    """The scattered-field form (stored field = total minus the bunch's TEM
    field of the entry pipe): the charges of the total field against the
    bunch, modes 0..2, float64."""
    w = chain(24, 90, 0, 2, "fp64", i0=3)
    s = tetm.RzSolver(w.nr, w.nz, w.m_lo, w.m_hi, w.dr, w.dz, w.cdt, "fp64", pec=w.pec)
    K = 2 * int(np.ceil(5 * w.sigma / w.dz - 1e-12)) + 2
    s.set_bunch_scattered(w.sigma, w.charge, w.i0, K)
    s.step(40)
    for m in range(3):
        e, h, q = s.charge_residual(m)
        print("scattered form residual", m, e / q, h / q)
        assert q > 0
        assert e <= 1e-12 * q and h <= 1e-12 * q, (m, e / q, h / q)


@pytest.mark.parametrize("start", ["cold", "scattered"])
def test_rz_checkpoint_split_run_is_bitwise_equal(tetm, start):
    w = chain(30, 96, 0, 2, "fp32", i0=3)
    K = 2 * int(np.ceil(5 * w.sigma / w.dz - 1e-12)) + 2

    def make():
        s = tetm.RzSolver(w.nr, w.nz, w.m_lo, w.m_hi, w.dr, w.dz, w.cdt, "fp32", pec=w.pec)
        s.set_kernel("bulk2")
        if start == "cold":
            s.set_bunch(w.sigma, w.charge, w.i0)
        else:
            s.set_bunch_scattered(w.sigma, w.charge, w.i0, K)
        return s
    a = make()
    a.step(41)
    buf = a.save()
    a.step(37)
    b = make()
    b.load(buf)
    assert b.info()["step"] == 41
    b.step(37)
    for m in range(3):
        assert np.array_equal(a.wake(m)[0], b.wake(m)[0]), m
        assert np.array_equal(a.transverse_wake(m), b.transverse_wake(m)), m
        for c in NAMES:
            assert np.array_equal(a.get(m, c), b.get(m, c)), (m, c)
    c = tetm.RzSolver(w.nr, w.nz, w.m_lo, w.m_hi, w.dr, w.dz, w.cdt, "fp32", pec=w.pec)
    with pytest.raises(tetm.TetmError) as e:
        c.load(buf)                                    # no bunch set: not the same solve
    assert e.value.code == tetm.TETM_E_ARG
