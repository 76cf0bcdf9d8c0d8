"""Pins of the rotationally symmetric FP64 oracle (oracle/tetm_rz_oracle.c,
Sec. 4.3, Eq. (24)) against what the paper and the mathematics fix: the dense
two-level form (24) assembled from the per-mode curl, the stability bound of
Sec. 4.4 (c*dt <= min(dr, dz) for every mode m), the energy law (19), the
pillbox eigenfrequencies of the continuous problem (Bessel zeros), the exact
one-cell shift of a coaxial TEM pulse at c*dt = dz (Sec. 4.5), Gauss's law
for an on-axis bunch and the loss-factor identity of the wake."""
import math

import numpy as np
import pytest
import scipy.special as sp

import oracle
from oracle import RzOracle, C_LIGHT, MU0, EPS0
from dense24 import Dense24

MM = 1e-3
NAMES = oracle.RZ_COMPONENTS


def _coefs(o):
    return [o.coef(c) for c in range(6)]


def _random_state(o, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    for c in NAMES:
        o.set(c, scale * rng.standard_normal(o.shape))


def _cavity_pec(nr, nz, r_pipe, k1, k2):
    """Staircase pillbox between pipes: cells with ci >= r_pipe are PEC outside
    the cavity cells k1 <= ck < k2."""
    pec = np.zeros((nz, nr), np.uint8)
    for k in range(nz):
        if not (k1 <= k < k2):
            pec[k, r_pipe:] = 1
    return pec


def _materials(nr, nz, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(1.0, 4.0, (nz, nr)), rng.uniform(1.0, 4.0, (nz, nr))


# ---------------------------------------------------------------------------
# Metric
# ---------------------------------------------------------------------------

def test_vacuum_metric_per_radian():
    nr, nz, dr, dz = 5, 4, 1.3 * MM, 0.9 * MM
    for m in (0, 2):
        o = RzOracle(nr, nz, m, dr, dz)
        c = {n: o.coef(n) for n in NAMES}
        i, k = 3, 2
        ri, rh = i * dr, (i + 0.5) * dr
        assert c["er"][k, i] == pytest.approx(dr / (EPS0 * rh * dz), rel=1e-15)
        assert c["ephi"][k, i] == pytest.approx(ri / (EPS0 * dr * dz), rel=1e-15)
        assert c["ez"][k, i] == pytest.approx(dz / (EPS0 * ri * dr), rel=1e-15)
        assert c["hphi"][k, i] == pytest.approx(rh / (MU0 * dr * dz), rel=1e-15)
        assert c["hr"][k, i] == pytest.approx(dr / (MU0 * ri * dz), rel=1e-15)
        assert c["hz"][k, i] == pytest.approx(dz / (MU0 * rh * dr), rel=1e-15)
        # axis: no e_phi, no h_r; e_z only for m = 0; PEC wall r = nr dr and z ends
        assert not c["ephi"][:, 0].any() and not c["hr"][:, 0].any()
        assert bool(c["ez"][0, 0]) == (m == 0)
        assert not c["ez"][:, nr].any() and not c["ephi"][:, nr].any()
        assert not c["er"][0].any() and not c["er"][nz].any() and not c["hz"][0].any()
        assert not c["ephi"][0].any() and not c["ephi"][nz].any()


# ---------------------------------------------------------------------------
# Ten detailed updates == dense two-level form (24)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m,seed", [(0, 0), (1, 1), (2, 2), (4, 3)])
def test_step_equals_dense_form(m, seed):
    nr, nz = 4, 4
    eps, mu = _materials(nr, nz, seed)
    pec = np.zeros((nz, nr), np.uint8)
    pec[2, 3] = 1
    dr, dz = 1.2 * MM, MM
    cdt = 0.95 * dz
    o = RzOracle(nr, nz, m, dr, dz, cdt=cdt, eps_r=eps, mu_r=mu, pec=pec)
    d = Dense24(nr, nz, m, _coefs(o), cdt)
    assert d.skew_ok < 1e-9 * np.max(np.abs(d.l))
    assert np.max(np.abs(d.qe - d.qe.T)) <= 1e-12 * np.max(np.abs(d.qe))   # Q^{e,r} symmetric
    _random_state(o, 100 + seed)
    rng = np.random.default_rng(200 + seed)
    y = d.y_from_fields(o.fields())
    for _ in range(3):
        jz = rng.standard_normal(o.shape) * 1e-3
        o.step_custom(jz)
        y = d.step(y, d.f_vec(jz))
        y_or = d.y_from_fields(o.fields())
        assert np.max(np.abs(y_or - y)) <= 1e-12 * np.max(np.abs(y))


def test_energy_formula_equals_dense_quadratic_form():
    for m in (0, 3):
        nr, nz = 4, 5
        eps, mu = _materials(nr, nz, 5 + m)
        o = RzOracle(nr, nz, m, 1.1 * MM, MM, eps_r=eps, mu_r=mu)
        d = Dense24(nr, nz, m, _coefs(o), o.dt * C_LIGHT)
        _random_state(o, 7 + m)
        assert o.energy() == pytest.approx(d.energy(d.y_from_fields(o.fields())), rel=1e-12)


# ---------------------------------------------------------------------------
# Stability (Sec. 4.4): c*dt <= min(dr, dz) independent of m
# ---------------------------------------------------------------------------

def _oracle_propagator(o, d):
    ny_ = d.be.shape[0]
    g = np.empty((ny_, ny_))
    for col in range(ny_):
        y = np.zeros(ny_)
        y[col] = 1.0
        f = d.fields_from_y(y)
        for c in range(6):
            o.set(c, f[c].reshape(o.shape))
        o.step_custom()
        g[:, col] = d.y_from_fields(o.fields())
    return g


@pytest.mark.parametrize("dr,dz", [(MM, MM), (0.8 * MM, MM), (MM, 0.7 * MM)])
def test_stable_at_the_bound_for_every_mode(dr, dz):
    nr, nz = 7, 8
    pec = _cavity_pec(nr, nz, 4, 3, 6)
    cdt = min(dr, dz)
    assert oracle.rz_stable(dr, dz, cdt) and not oracle.rz_stable(dr, dz, 1.01 * cdt)
    for m in range(5):
        o = RzOracle(nr, nz, m, dr, dz, cdt=cdt, pec=pec)
        d = Dense24(nr, nz, m, _coefs(o), cdt)
        g = _oracle_propagator(o, d) if m in (0, 3) else d.propagator()
        if m in (0, 3):
            np.testing.assert_allclose(g, d.propagator(), atol=1e-11)
        lam = np.linalg.eigvals(g)
        assert np.max(np.abs(lam)) < 1.0 + 1e-8, (m, np.max(np.abs(lam)))
        # strictly inside the bound the discrete energy is a norm (Q^{e,r} > 0)
        d2 = Dense24(nr, nz, m, _coefs(RzOracle(nr, nz, m, dr, dz, cdt=0.98 * cdt, pec=pec)),
                     0.98 * cdt)
        assert np.min(np.linalg.eigvalsh(0.5 * (d2.qe + d2.qe.T))) > 0


def test_time_step_above_the_bound_grows():
    nr, nz, dr, dz = 6, 6, MM, 1.5 * MM
    grew = []
    for m in (0, 2):
        cdt = 1.08 * dr
        o = RzOracle(nr, nz, m, dr, dz, cdt=cdt)
        d = Dense24(nr, nz, m, _coefs(o), cdt)
        grew.append(np.max(np.abs(np.linalg.eigvals(d.propagator()))))
    assert min(grew) > 1.0 + 1e-3


def test_high_modes_do_not_reduce_the_step():
    """At c*dt = min(dr, dz) the modes m = 8 and 16 stay bounded; the Yee
    limit quoted in Sec. 4.4 would need a step several times smaller."""
    nr, nz, dr, dz = 6, 5, MM, MM
    for m in (8, 16):
        o = RzOracle(nr, nz, m, dr, dz)
        d = Dense24(nr, nz, m, _coefs(o), o.dt * C_LIGHT)
        assert np.max(np.abs(np.linalg.eigvals(d.propagator()))) < 1.0 + 1e-8
        yee = 1.0 / math.sqrt((1.2 + 0.4 * m * m) / dr ** 2 + 1.2 / dz ** 2)
        assert yee < 0.25 * o.dt * C_LIGHT


# ---------------------------------------------------------------------------
# Energy law (19)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m", [0, 1, 3])
def test_energy_conserved_without_current(m):
    nr, nz = 10, 14
    o = RzOracle(nr, nz, m, MM, MM, pec=_cavity_pec(nr, nz, 6, 4, 10))
    _random_state(o, 11 + m)
    w0 = o.energy()
    for _ in range(10):
        o.step(30)
        assert o.energy() == pytest.approx(w0, rel=1e-12)


def test_energy_law_with_current():
    o = RzOracle(8, 12, 1, 1.2 * MM, MM)
    _random_state(o, 12)
    rng = np.random.default_rng(13)
    for _ in range(10):
        w0 = o.energy()
        ez0 = o.get("ez")
        jz = rng.standard_normal(o.shape)
        o.step_custom(jz)
        ez1 = o.get("ez")
        rhs = -o.dt * np.sum(jz * 0.5 * (ez0 + ez1) * (o.coef("ez") != 0))
        assert o.energy() - w0 == pytest.approx(rhs, rel=1e-9, abs=1e-12 * abs(w0))


# ---------------------------------------------------------------------------
# Pillbox eigenfrequencies converge to the Bessel-zero closed form
# ---------------------------------------------------------------------------

def _lowest_angles(nr, nz, m, radius, length, family=None):
    dr, dz = radius / nr, length / nz
    cdt = min(dr, dz)
    o = RzOracle(nr, nz, m, dr, dz, cdt=cdt)
    d = Dense24(nr, nz, m, _coefs(o), cdt)
    lam, vec = np.linalg.eig(d.propagator())
    ang = np.angle(lam)
    keep = ang > 1e-6
    if family is not None:
        # share of each eigenvector in the e_phi/h_r/h_z (TE) components
        x = np.zeros_like(vec)
        x[d.perm] = vec
        comp = d.comp
        te = np.isin(comp, (1, 3, 5))
        share = np.sum(np.abs(x[te]) ** 2, axis=0) / np.sum(np.abs(x) ** 2, axis=0)
        keep &= (share > 0.5) if family == "TE" else (share < 0.5)
    return np.sort(ang[keep]) / (cdt / C_LIGHT), cdt


@pytest.mark.parametrize("m", [0, 1, 2])
def test_pillbox_tm_m10_converges_second_order(m):
    """TM_{m,1,0} of a pillbox of radius R: omega = c j_{m,1} / R."""
    radius, length = 20 * MM, 2 * MM
    exact = C_LIGHT * sp.jn_zeros(m, 1)[0] / radius
    errs = []
    for nr in (16, 32, 64):
        w, _ = _lowest_angles(nr, 2, m, radius, length)
        errs.append(abs(w[0] / exact - 1.0))
    assert errs[-1] < 1e-3
    assert errs[0] > errs[1] > errs[2] and 3.5 < errs[1] / errs[2] < 4.5


def test_pillbox_te_011_converges_second_order():
    """TE_{0,1,1}: omega = c sqrt((j'_{0,1}/R)^2 + (pi/L)^2), j'_{0,1} = j_{1,1}."""
    radius, length = 10 * MM, 10 * MM
    exact = C_LIGHT * math.hypot(sp.jnp_zeros(0, 1)[0] / radius, math.pi / length)
    errs = []
    for n in (6, 12, 24):
        w, _ = _lowest_angles(n, n, 0, radius, length, family="TE")
        errs.append(abs(w[0] / exact - 1.0))
    assert errs[-1] < 5e-3
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0


# ---------------------------------------------------------------------------
# Zero dispersion along z: a coaxial TEM pulse shifts one cell per step
# ---------------------------------------------------------------------------

def test_coaxial_tem_pulse_shifts_one_cell_per_step():
    nr, nz, dr, dz = 12, 40, 1.3 * MM, MM
    pec = np.zeros((nz, nr), np.uint8)
    pec[:, :3] = 1                               # inner conductor r < 3 dr
    eta0 = MU0 * C_LIGHT
    kk = np.arange(nz + 1)
    rh = (np.arange(nr + 1) + 0.5) * dr

    def F(k):
        x = (np.asarray(k, dtype=float) - 8.0) / 3.0
        return np.where(np.abs(x) < 1.0, (1 - x * x) ** 3, 0.0)

    o = RzOracle(nr, nz, 0, dr, dz, cdt=dz, pec=pec)
    sh = o.shape
    o.set("er", (dr / rh)[None, :] * F(kk)[:, None] * np.ones(sh))
    o.set("hphi", -F(kk + 1)[:, None] / eta0 * np.ones(sh))
    nsteps = 20
    o.step(nsteps)
    er_exp = (dr / rh)[None, :] * F(kk - nsteps)[:, None] * (o.coef("er") != 0)
    hp_exp = -F(kk + 1 - nsteps)[:, None] / eta0 * (o.coef("hphi") != 0)
    escale, hscale = np.max(np.abs(er_exp)), np.max(np.abs(hp_exp))
    assert np.max(np.abs(o.get("er") - er_exp)) <= 1e-13 * escale
    assert np.max(np.abs(o.get("hphi") - hp_exp)) <= 1e-13 * hscale
    assert np.max(np.abs(o.get("ez"))) <= 1e-13 * escale
    for c in ("ephi", "hr", "hz"):
        assert not o.get(c).any()


# ---------------------------------------------------------------------------
# Gauss's law and the wake for an on-axis bunch (m = 0)
# ---------------------------------------------------------------------------

def _node_charge_closed_form(q, sigma, dz, zc, k):
    a = max(k * dz - 0.5 * dz - zc, -5 * sigma)
    b = min(k * dz + 0.5 * dz - zc, 5 * sigma)
    if b <= a:
        return 0.0
    return q * 0.5 * (math.erf(b / (sigma * math.sqrt(2))) - math.erf(a / (sigma * math.sqrt(2))))


def _rz_interior_nodes(o):
    """Nodes whose incident edges all carry a field: e_z below and above, e_r
    outward and inward (the axis node has no inward e_r), e_phi for m >= 1."""
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


def _rz_interior_cells(o):
    """Cells (by lower node) whose faces all carry a field: h_z below and
    above, h_r outward and inward (none on the axis), h_phi for m >= 1."""
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


@pytest.mark.parametrize("m", [0, 1, 2, 3])
def test_rz_charges_with_random_fields_and_currents(m):
    """The mode-m charges of the oracle (qbar_e, qbar_h) obey the discrete
    charge laws of Sec. 4.5 for scheme (24): with a current j_z the node
    charge changes by dt P_z^T j_z per step, the cell charge does not change;
    on a pillbox between pipes, random fields (charges of the size of the
    fluxes) and random currents."""
    nr, nz = 12, 30
    o = RzOracle(nr, nz, m, MM, MM, pec=_cavity_pec(nr, nz, 6, 10, 20))
    _random_state(o, 40 + m)
    rng = np.random.default_rng(50 + m)
    jz = [rng.standard_normal(o.shape) * (o.coef("ez") != 0) for _ in range(3)]
    hist = [o.fields()]
    for n in range(3):
        o.step_custom(jz[n])
        hist.append(o.fields())
    inode, icell = _rz_interior_nodes(o), _rz_interior_cells(o)
    assert inode.sum() > 20 and icell.sum() > 20
    qe = [o.qbar_e(hist[n + 1]["er"], hist[n]["er"], hist[n + 1]["ephi"], hist[n]["ephi"], hist[n + 1]["ez"])
          for n in range(3)]
    for n in (1, 2):
        ptz = -jz[n]
        ptz[1:, :] += jz[n][:-1, :]
        res = (qe[n] - qe[n - 1]) - o.dt * ptz
        assert np.max(np.abs(res[inode])) <= 1e-12 * np.max(np.abs(qe[n][inode]))
    qh = [o.qbar_h(hist[n + 1]["hphi"], hist[n]["hphi"], hist[n + 1]["hr"], hist[n]["hr"], hist[n]["hz"])
          for n in range(3)]
    scale = np.max(np.abs(qh[0][icell]))
    d_scale = np.max(np.abs(hist[0]["hz"] / np.where(o.coef("hz") != 0, o.coef("hz"), np.inf)))
    assert scale > 0.1 * d_scale
    for n in (1, 2):
        assert np.max(np.abs(qh[n][icell] - qh[0][icell])) <= 1e-12 * scale


@pytest.mark.parametrize("m", [1, 2])
def test_rz_charge_keeps_the_m_part_out_of_the_z_flux(m):
    """Reading of Sec. 4.3: the m-part of the splitting operator stays in
    B^{e,r}, so the conserved z-flux is corrected by the radial part only.
    Adding the m-part (alpha^2 m^2 M_hr^-1 e_z) to the corrected flux breaks
    the conservation at O(1)."""
    nr, nz = 12, 30
    o = RzOracle(nr, nz, m, MM, MM, pec=_cavity_pec(nr, nz, 6, 10, 20))
    _random_state(o, 60 + m)
    hist = [o.fields()]
    for n in range(3):
        o.step(1)
        hist.append(o.fields())
    inode = _rz_interior_nodes(o)

    def alt(n):
        q = o.qbar_e(hist[n + 1]["er"], hist[n]["er"], hist[n + 1]["ephi"], hist[n]["ephi"], hist[n + 1]["ez"])
        extra = o.alpha ** 2 * m * m * o.coef("hr") * hist[n + 1]["ez"] * (o.coef("ez") != 0)
        ptz = -extra
        ptz[1:, :] += extra[:-1, :]
        return q - ptz, q
    a0, q0 = alt(0)
    a2, q2 = alt(2)
    scale = np.max(np.abs(q0[inode]))
    assert np.max(np.abs(q2[inode] - q0[inode])) <= 1e-12 * scale
    assert np.max(np.abs(a2[inode] - a0[inode])) > 1e-3 * scale


@pytest.mark.parametrize("m,i0", [(0, 0), (1, 3), (2, 3)])
def test_gauss_law_for_the_bunch(m, i0):
    """The node charge of the mode equals the bunch's share of the truncated
    Gaussian's node charges on the ring: (2 - delta_m0)/(2 pi) per radian."""
    nr, nz = 10, 40
    q, sigma = 1e-9, 2.5 * MM
    pec = _cavity_pec(nr, nz, 5, 15, 25)
    share = (1.0 if m == 0 else 2.0) / (2 * math.pi)
    for n in (6, 13, 20, 29):
        o = RzOracle(nr, nz, m, MM, MM, pec=pec)
        o.set_bunch(sigma, q, i0)
        c0 = math.ceil(5 * sigma / MM - 1e-12)
        o.step(n)
        er0, ep0 = o.get("er"), o.get("ephi")
        o.step(1)
        qe = o.qbar_e(o.get("er"), er0, o.get("ephi"), ep0, o.get("ez"))
        zc = (n + 0.5 - c0) * MM
        expect = np.zeros(o.shape)
        for k in range(1, nz):
            expect[k, i0] = share * _node_charge_closed_form(q, sigma, MM, zc, k)
        inner = _rz_interior_nodes(o)
        assert inner[:, i0].sum() > nz // 2
        assert np.max(np.abs(qe[inner] - expect[inner])) <= 1e-12 * q
        if n >= 13:
            assert np.max(np.abs(expect)) > 0.05 * share * q


@pytest.mark.parametrize("m,i0", [(0, 0), (1, 3), (2, 4)])
def test_loss_factor_identity(m, i0):
    """Energy law (19) summed over the passage: the energy left behind per
    radian equals w_m Q/2 sum_d Q_cell(d) [W(-d) + W(-d-1)], with the mode
    share w_m = (2 - delta_m0)/(2 pi) of the source."""
    nr, nz = 8, 30
    sigma, q = 2.0 * MM, 1e-9
    o = RzOracle(nr, nz, m, MM, MM, pec=_cavity_pec(nr, nz, 6, 10, 18))
    o.set_bunch(sigma, q, i0)
    c0 = math.ceil(5 * sigma / MM - 1e-12)
    m_max = math.ceil(15 * sigma / MM - 1e-12)
    o.step(nz + 2 * c0 + m_max)
    wk, s0, ds = o.wake()
    m_min = -c0 - 1
    assert s0 == pytest.approx(m_min * MM)
    edges = np.arange(-c0, c0 + 1) * MM
    qcell = q * np.diff(0.5 * (1 + sp.erf(np.clip(edges, -5 * sigma, 5 * sigma) / (sigma * math.sqrt(2)))))
    rhs = 0.0
    for d in range(-c0, c0):
        rhs += 0.5 * q * qcell[d + c0] * (wk[-d - m_min] + wk[-d - 1 - m_min])
    w_m = (1.0 if m == 0 else 2.0) / (2 * math.pi)
    assert o.energy() == pytest.approx(w_m * rhs, rel=1e-11)
    assert o.energy() > 0


def test_no_field_ahead_of_the_bunch():
    nr, nz = 8, 50
    o = RzOracle(nr, nz, 0, MM, MM)
    o.set_bunch(3 * MM, 1e-9, 0)
    for n in (10, 25, 40):
        o.step(n - o.step_count)
        for c in NAMES:
            f = o.get(c)
            assert np.all(f[n + 1:] == 0.0), (c, n)
    assert o.get("ez").any()


def test_bad_bunch_and_grid_arguments():
    with pytest.raises(ValueError):
        RzOracle(1, 4, 0, MM, MM)
    o = RzOracle(6, 6, 1, MM, MM)
    with pytest.raises(ValueError):
        o.set_bunch(MM, 1e-9, 0)        # only m = 0 lives on the axis
    with pytest.raises(ValueError):
        o.set_bunch(MM, 1e-9, 6)        # the ring must lie inside the wall


def _numpy_step(f, c, alpha, m, factor_e, factor_h):
    """The ten updates of (24) with the implicit diagonal factors passed in."""
    er, ep, ez, hr, hp, hz = [x.copy() for x in f]
    cer, cep, cez, chr_, chp, chz = c

    def pz(v):
        out = -v.copy(); out[:-1] += v[1:]; return out

    def pr(v):
        out = -v.copy(); out[:, :-1] += v[:, 1:]; return out

    def pzt(v):
        out = -v.copy(); out[1:] += v[:-1]; return out

    def prt(v):
        out = -v.copy(); out[:, 1:] += v[:, :-1]; return out

    a = alpha
    hp += a * chp * (pz(er) - pr(ez)); hr += a * chr_ * (-pz(ep) + m * ez)
    ez += 2 * a * cez * (prt(hp) - m * hr) / (1 + a * a * m * m * factor_e)
    hp += a * chp * (pz(er) - pr(ez)); hr += a * chr_ * (-pz(ep) + m * ez)
    ep += a * cep * (pzt(hr) - prt(hz)); er += a * cer * (-pzt(hp) + m * hz)
    hz += 2 * a * chz * (pr(ep) - m * er) / (1 + a * a * m * m * factor_h)
    ep += a * cep * (pzt(hr) - prt(hz)); er += a * cer * (-pzt(hp) + m * hz)
    return [er, ep, ez, hr, hp, hz]


def test_factor_pairing_reading():
    """The diagonal factor of the e_z update pairs M_eps_z^-1 with M_mu_r^-1 of
    the same entry (the h_r that the m-terms couple to e_z), and the h_z factor
    pairs M_mu_z^-1 with M_eps_r^-1. With the labels as printed in (24)
    (mu_z eps_r for e_z, eps_z mu_r for h_z) the scheme is not of the form
    (24) and grows at c*dt = min(dr, dz)."""
    nr, nz = 6, 6
    for m in (1, 2):
        o = RzOracle(nr, nz, m, MM, MM)
        c = _coefs(o)
        d = Dense24(nr, nz, m, c, o.dt * C_LIGHT)
        n = d.be.shape[0]
        grow = {}
        for name, fe, fh in (("derived", c[2] * c[3], c[5] * c[0]),
                             ("printed", c[5] * c[0], c[2] * c[3])):
            g = np.empty((n, n))
            for col in range(n):
                y = np.zeros(n)
                y[col] = 1.0
                f = [x.reshape(o.shape) for x in d.fields_from_y(y)]
                g[:, col] = d.y_from_fields(_numpy_step(f, c, o.alpha, m, fe, fh))
            grow[name] = np.max(np.abs(np.linalg.eigvals(g)))
            if name == "derived":
                np.testing.assert_allclose(g, d.propagator(), atol=1e-12)
        assert grow["derived"] < 1.0 + 1e-9
        assert grow["printed"] > 1.5


# ---------------------------------------------------------------------------
# Transverse wake (Sec. 5: the dipole wake of the transverse deflecting
# structure) and the Panofsky-Wenzel theorem, dW_perp/ds = grad_perp W_par
# (with W_par = -(1/Q) int E_z): in the scheme at c*dt = dz it holds exactly
# between the radial wake at r_{i+1/2} and the longitudinal wakes at the
# rings i and i+1, with the half-sample average the staggering asks for:
#   W_r(m+1) - W_r(m) = dz/dr * [(W_{i+1} - W_i)(m) + (W_{i+1} - W_i)(m+1)] / 2
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m,i0,obs", [(1, 3, 3), (1, 3, 6), (2, 4, 5), (0, 0, 2)])
def test_discrete_panofsky_wenzel(m, i0, obs):
    nr, nz = 20, 100
    pec = _cavity_pec(nr, nz, 7, 40, 70)
    o = RzOracle(nr, nz, m, MM, MM, pec=pec)
    o.set_bunch(2.5 * MM, 1e-9, i0)
    o.set_observer(obs)
    c0 = math.ceil(5 * 2.5 - 1e-12)
    o.step(nz + 2 * c0 + math.ceil(15 * 2.5) + 2)
    wr = o.transverse_wake()
    w0, w1 = o.wake_at_observer()
    grad = (w1 - w0) * (MM / MM)
    rhs = 0.5 * (grad[:-1] + grad[1:])
    lhs = np.diff(wr)
    assert np.max(np.abs(rhs)) > 0
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-11 * np.max(np.abs(rhs)))
    # the bunch-ring wake of the main accumulator is the one at ring i0
    if obs == i0:
        np.testing.assert_array_equal(w0, o.wake()[0])


def test_transverse_wake_vanishes_for_the_tem_field_of_a_smooth_pipe():
    """E_r - c mu0 H_phi of the bunch's own field cancels along the path: in a
    coaxial smooth pipe the TEM pulse of the shift test exerts no force."""
    nr, nz, dr, dz = 12, 40, 1.3 * MM, MM
    pec = np.zeros((nz, nr), np.uint8)
    pec[:, :3] = 1
    eta0 = MU0 * C_LIGHT
    kk = np.arange(nz + 1)
    rh = (np.arange(nr + 1) + 0.5) * dr
    x = (kk - 8.0) / 3.0
    F = np.where(np.abs(x) < 1.0, (1 - x * x) ** 3, 0.0)
    x1 = (kk + 1 - 8.0) / 3.0
    F1 = np.where(np.abs(x1) < 1.0, (1 - x1 * x1) ** 3, 0.0)
    o = RzOracle(nr, nz, 0, dr, dz, cdt=dz, pec=pec)
    o.set("er", (dr / rh)[None, :] * F[:, None] * np.ones(o.shape))
    o.set("hphi", -F1[:, None] / eta0 * np.ones(o.shape))
    er = o.get("er")
    for _ in range(20):
        er_n = o.get("er")
        o.step(1)
        hp = o.get("hphi")
        force = er_n / dr + eta0 * hp / rh[None, :]
        assert np.max(np.abs(force)) <= 1e-12 * np.max(np.abs(er / dr))


# ---------------------------------------------------------------------------
# Static start (infinite ingoing pipe, Sec. 5): the discrete TEM field of the
# ring bunch, mode by mode, moves one cell per step (Sec. 4.5)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("m,i0", [(0, 0), (0, 3), (1, 3), (2, 4), (4, 2)])
def test_static_start_moves_rigidly_and_leaves_no_wake(m, i0):
    nr, nz, K = 16, 90, 34
    pec = _cavity_pec(nr, nz, 10, nz, nz)          # smooth pipe of radius 10 cells
    o = RzOracle(nr, nz, m, MM, MM, pec=pec)
    o.set_bunch_static(3 * MM, 1e-9, i0, K)
    f0 = o.fields()
    assert not f0["ez"].any() and not f0["hz"].any()
    n = 40
    o.step(n)
    escale = max(np.max(np.abs(f0["er"])), np.max(np.abs(f0["ephi"])))
    hscale = max(np.max(np.abs(f0["hphi"])), np.max(np.abs(f0["hr"])))
    for c in NAMES:
        shifted = np.zeros_like(f0[c])
        shifted[n:] = f0[c][:-n]
        assert np.max(np.abs(o.get(c) - shifted)) <= 1e-13 * (escale if c[0] == "e" else hscale), c
    cold = RzOracle(nr, nz, m, MM, MM, pec=pec)
    cold.set_bunch(3 * MM, 1e-9, i0)
    cold.step(n + K)
    assert np.max(np.abs(o.wake()[0])) <= 1e-13 * np.max(np.abs(cold.wake()[0]))
    assert np.max(np.abs(o.transverse_wake())) <= 1e-13 * np.max(np.abs(cold.transverse_wake()))


def test_static_start_energy_identity_in_a_cavity():
    nr, nz, K = 14, 70, 24
    pec = _cavity_pec(nr, nz, 6, 32, 46)
    sigma, q, m, i0 = 2 * MM, 1e-9, 1, 3
    o = RzOracle(nr, nz, m, MM, MM, pec=pec)
    o.set_bunch_static(sigma, q, i0, K)
    w0 = o.energy()
    c0 = math.ceil(5 * sigma / MM - 1e-12)
    o.step(nz - (K - 2 * c0) + 1)
    wk = o.wake()[0]
    edges = np.arange(-c0, c0 + 1) * MM
    qcell = q * np.diff(0.5 * (1 + sp.erf(np.clip(edges, -5 * sigma, 5 * sigma) / (sigma * math.sqrt(2)))))
    m_min = -c0 - 1
    rhs = sum(0.5 * q * qcell[d + c0] * (wk[-d - m_min] + wk[-d - 1 - m_min]) for d in range(-c0, c0))
    assert o.energy() - w0 == pytest.approx(rhs / math.pi, rel=1e-10, abs=1e-12 * w0)
    assert abs(rhs) > 1e-6 * w0


def test_static_start_rejections():
    nr, nz = 12, 60
    pec = _cavity_pec(nr, nz, 6, 20, 40)
    with pytest.raises(ValueError):
        RzOracle(nr, nz, 1, MM, MM, pec=pec).set_bunch_static(2 * MM, 1e-9, 3, 30)  # K past k = 20
    with pytest.raises(ValueError):
        RzOracle(nr, nz, 1, MM, MM, pec=pec).set_bunch_static(2 * MM, 1e-9, 3, 10)  # K < 2 c0 + 2
    with pytest.raises(ValueError):
        RzOracle(nr, nz, 1, MM, MM, eps_r=np.ones((nz, nr)), pec=pec).set_bunch_static(MM, 1e-9, 3, 14)
