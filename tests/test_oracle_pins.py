"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle (oracle/tetm_oracle.c) against something other
than itself: the dense two-level form (23) assembled from the operator
definitions of Sec. 2 and Sec. 4.2, the closed-form dispersion relation (27),
the energy law (19), the charge laws (34)/(35), Gauss's law for the bunch,
the exact one-cell shift of a TEM pulse at c*dt = dz (Sec. 4.5), causality,
and the loss-factor identity that ties the wake of Sec. 5 to the field energy.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import Oracle, C_LIGHT, MU0, EPS0
from dense23 import Dense23
from paper_0901_1053_gb300 import workloads as wl

MM = 1e-3
DXY = math.sqrt(2.0) * MM


def _random_state(o, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    for c in oracle.COMPONENTS:
        o.set(c, scale * rng.standard_normal(o.shape))


def _coefs(o):
    return [o.coef(c) for c in range(6)]


# ---------------------------------------------------------------------------
# Geometry (staircase reading of the material matrices)
# ---------------------------------------------------------------------------

def test_vacuum_box_active_counts_and_values():
    nx, ny, nz = 3, 4, 5
    o = Oracle(nx, ny, nz, 1.3 * MM, 1.7 * MM, 0.9 * MM)
    dx, dy, dz = 1.3 * MM, 1.7 * MM, 0.9 * MM
    counts = [int(np.count_nonzero(o.coef(c))) for c in range(6)]
    assert counts == [nx * (ny - 1) * (nz - 1), (nx - 1) * ny * (nz - 1), (nx - 1) * (ny - 1) * nz,
                      (nx - 1) * ny * nz, nx * (ny - 1) * nz, nx * ny * (nz - 1)]
    expect = [dx / (EPS0 * dy * dz), dy / (EPS0 * dx * dz), dz / (EPS0 * dx * dy),
              dx / (MU0 * dy * dz), dy / (MU0 * dx * dz), dz / (MU0 * dx * dy)]
    for c in range(6):
        v = o.coef(c)
        np.testing.assert_allclose(v[v != 0], expect[c], rtol=1e-15)


def test_pec_cell_deactivates_its_edges_and_faces():
    nx = ny = nz = 4
    pec = np.zeros((nz, ny, nx), np.uint8)
    pec[1, 2, 1] = 1                    # cell (ci=1, cj=2, ck=1)
    o0 = Oracle(nx, ny, nz, MM, MM, MM)
    o1 = Oracle(nx, ny, nz, MM, MM, MM, pec=pec)
    # brute force from the cell side: the 12 edges and 6 faces of the cell
    ci, cj, ck = 1, 2, 1
    edges = {0: [(ci, cj + b, ck + c) for b in (0, 1) for c in (0, 1)],
             1: [(ci + a, cj, ck + c) for a in (0, 1) for c in (0, 1)],
             2: [(ci + a, cj + b, ck) for a in (0, 1) for b in (0, 1)],
             3: [(ci + a, cj, ck) for a in (0, 1)],
             4: [(ci, cj + b, ck) for b in (0, 1)],
             5: [(ci, cj, ck + c) for c in (0, 1)]}
    for comp in range(6):
        a0, a1 = o0.coef(comp) != 0, o1.coef(comp) != 0
        lost = set(zip(*np.nonzero(a0 & ~a1)))
        lost = {(int(i), int(j), int(k)) for (k, j, i) in lost}
        expect = {e for e in edges[comp] if a0[e[2], e[1], e[0]]}
        assert lost == expect, (comp, lost, expect)
        assert not np.any(a1 & ~a0)


def test_material_averaging():
    nx = ny = nz = 3
    eps = np.full((nz, ny, nx), 2.0)
    eps[1, 1, 1] = 4.0
    mu = np.full((nz, ny, nx), 1.0)
    mu[1, 1, 1] = 3.0
    o = Oracle(nx, ny, nz, MM, MM, MM, eps_r=eps, mu_r=mu)
    # ez edge (1,1,k=1+1/2) touches cells (0..1, 0..1, 1): one of them eps 4
    ez = o.coef(2)
    assert ez[1, 1, 1] == pytest.approx(MM / (EPS0 * (2.0 + 2.0 + 2.0 + 4.0) / 4.0 * MM * MM), rel=1e-15)
    # hx face x=1 between cells (0,1,1) and (1,1,1): 1/mu_bar = (1 + 1/3)/2
    hx = o.coef(3)
    assert hx[1, 1, 1] == pytest.approx(MM * ((1.0 + 1.0 / 3.0) / 2.0) / (MU0 * MM * MM), rel=1e-15)


# ---------------------------------------------------------------------------
# Brute force: ten detailed updates == dense two-level form (23)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1])
def test_step_equals_dense_form_with_materials_and_currents(seed):
    nx, ny, nz = 3, 3, 4
    eps, mu, pec = wl.random_materials(nx, ny, nz, seed)
    pec[:] = 0
    pec[1, 1, 1] = 1
    dx, dy, dz = 1.1 * DXY, DXY, MM
    cdt = 0.9 * dz
    o = Oracle(nx, ny, nz, dx, dy, dz, cdt=cdt, eps_r=eps, mu_r=mu, pec=pec)
    d = Dense23(nx, ny, nz, _coefs(o), cdt)
    assert d.skew_ok < 1e-9 * np.max(np.abs(d.l))
    _random_state(o, 100 + seed)
    rng = np.random.default_rng(200 + seed)
    y = d.y_from_fields(o.fields())
    for _ in range(3):
        jz, jx, jy = (rng.standard_normal(o.shape) * 1e-3 for _ in range(3))
        o.step_custom(jz, jx, jy)
        y = d.step(y, d.f_vec(jz, jx, jy))
        y_or = d.y_from_fields(o.fields())
        assert np.max(np.abs(y_or - y)) <= 1e-12 * np.max(np.abs(y))


def test_energy_formula_equals_dense_quadratic_form():
    nx, ny, nz = 3, 4, 3
    eps, mu, pec = wl.random_materials(nx, ny, nz, 5)
    pec[:] = 0
    o = Oracle(nx, ny, nz, DXY, 1.2 * DXY, MM, eps_r=eps, mu_r=mu, pec=pec)
    d = Dense23(nx, ny, nz, _coefs(o), MM)
    assert np.max(np.abs(d.qe - d.qe.T)) <= 1e-12 * np.max(np.abs(d.qe))   # Q^e = Q^e*
    _random_state(o, 7)
    y = d.y_from_fields(o.fields())
    w_dense = d.energy(y)
    assert o.energy() == pytest.approx(w_dense, rel=1e-12)


# ---------------------------------------------------------------------------
# Dispersion relation (27) and stability (25)
# ---------------------------------------------------------------------------

def _oracle_propagator(o, d):
    """Columns = one oracle step applied to each unit vector of y."""
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


def _closed_form_angles(nx, ny, nz, dx, dy, dz, cdt):
    """Eq. (27): sin^2 W / dtau^2 = sin^2 Kz/dz^2 + (sin^2 Kx/dx^2 + sin^2 Ky/dy^2)
    (1 - dtau^2/dz^2 sin^2 Kz), K = p*pi/(2N) for the standing waves of a PEC box;
    one step turns a mode by 2W. Multiplicity 2 if p, q, r >= 1, 1 if exactly one is 0."""
    out = []
    for p in range(nx):
        for q in range(ny):
            for r in range(nz):
                zeros = (p == 0) + (q == 0) + (r == 0)
                mult = {0: 2, 1: 1}.get(zeros, 0)
                if not mult:
                    continue
                sx = math.sin(p * math.pi / (2 * nx)) ** 2 / dx ** 2
                sy = math.sin(q * math.pi / (2 * ny)) ** 2 / dy ** 2
                sz = math.sin(r * math.pi / (2 * nz)) ** 2 / dz ** 2
                s2 = cdt ** 2 * (sz + (sx + sy) * (1.0 - cdt ** 2 * sz))
                out += [2.0 * math.asin(math.sqrt(s2))] * mult
    return np.sort(np.array(out))


@pytest.mark.parametrize("dims,ratio", [((3, 4, 5), (DXY, DXY, MM)), ((4, 3, 4), (1.7 * MM, 1.5 * MM, MM))])
def test_eigen_angles_match_dispersion_relation(dims, ratio):
    nx, ny, nz = dims
    dx, dy, dz = ratio
    cdt = dz
    assert oracle.stable(dx, dy, dz, cdt)
    o = Oracle(nx, ny, nz, dx, dy, dz, cdt=cdt)
    d = Dense23(nx, ny, nz, _coefs(o), cdt)
    g = _oracle_propagator(o, d)
    np.testing.assert_allclose(g, d.propagator(), atol=1e-12)
    lam = np.linalg.eigvals(g)
    assert np.max(np.abs(np.abs(lam) - 1.0)) < 1e-9
    ang = np.angle(lam)
    pos = np.sort(ang[ang > 1e-7])
    expect = _closed_form_angles(nx, ny, nz, dx, dy, dz, cdt)
    assert len(pos) == len(expect)
    np.testing.assert_allclose(pos, expect, atol=1e-9)


def test_cubic_mesh_at_magic_step_is_unstable():
    """Eq. (25) is necessary (Sec. 4.5): dx = dy = dz with c*dt = dz grows."""
    nx, ny, nz = 4, 4, 4
    assert not oracle.stable(MM, MM, MM, MM)
    o = Oracle(nx, ny, nz, MM, MM, MM, cdt=MM)
    d = Dense23(nx, ny, nz, _coefs(o), MM)
    lam = np.linalg.eigvals(_oracle_propagator(o, d))
    assert np.max(np.abs(lam)) > 1.5
    # and the amended mesh of the same box is not
    o2 = Oracle(nx, ny, nz, DXY, DXY, MM, cdt=MM)
    d2 = Dense23(nx, ny, nz, _coefs(o2), MM)
    lam2 = np.linalg.eigvals(_oracle_propagator(o2, d2))
    assert np.max(np.abs(lam2)) < 1.0 + 1e-9


# ---------------------------------------------------------------------------
# Energy law (19)
# ---------------------------------------------------------------------------

def test_energy_conserved_without_current():
    o = Oracle(6, 5, 8, DXY, 1.1 * DXY, MM)
    _random_state(o, 11)
    w0 = o.energy()
    for _ in range(20):
        o.step(25)
        assert o.energy() == pytest.approx(w0, rel=1e-13)


def test_energy_law_with_current():
    """W^{n+1} - W^n = -dt sum jj_z^n (ez^{n+1/2} + ez^{n-1/2})/2, Eq. (19)."""
    o = Oracle(6, 6, 10, DXY, DXY, MM)
    _random_state(o, 12)
    rng = np.random.default_rng(13)
    for _ in range(10):
        w0 = o.energy()
        ez0 = o.get("ez")
        jz = rng.standard_normal(o.shape)
        o.step_custom(jz)
        ez1 = o.get("ez")
        w1 = o.energy()
        rhs = -o.dt * np.sum(jz * 0.5 * (ez0 + ez1) * (o.coef("ez") != 0))
        assert w1 - w0 == pytest.approx(rhs, rel=1e-9, abs=1e-12 * abs(w0))


# ---------------------------------------------------------------------------
# Charge laws (34), (35) and Gauss's law for the bunch
# ---------------------------------------------------------------------------

def _interior_nodes(o):
    """Nodes whose six incident edges are all non-PEC."""
    ae = [o.coef(c) != 0 for c in range(3)]
    m = np.zeros(o.shape, bool)
    m[1:, 1:, 1:] = (ae[0][1:, 1:, 1:] & ae[0][1:, 1:, :-1] & ae[1][1:, 1:, 1:] &
                     ae[1][1:, :-1, 1:] & ae[2][1:, 1:, 1:] & ae[2][:-1, 1:, 1:])
    return m


def _interior_cells(o):
    """Cells (indexed by their lower node) whose six faces are all active."""
    ah = [o.coef(c) != 0 for c in range(3, 6)]
    m = np.zeros(o.shape, bool)
    m[:-1, :-1, :-1] = (ah[0][:-1, :-1, :-1] & ah[0][:-1, :-1, 1:] & ah[1][:-1, :-1, :-1] &
                        ah[1][:-1, 1:, :-1] & ah[2][:-1, :-1, :-1] & ah[2][1:, :-1, :-1])
    return m


def test_charge_laws_with_random_fields_and_currents():
    nx, ny, nz = 5, 5, 6
    pec = np.zeros((nz, ny, nx), np.uint8)
    pec[2, 3, 3] = 1
    o = Oracle(nx, ny, nz, DXY, DXY, MM, pec=pec)
    _random_state(o, 21)
    rng = np.random.default_rng(22)
    jx = [rng.standard_normal(o.shape) for _ in range(3)]
    jy = [rng.standard_normal(o.shape) for _ in range(3)]
    jz = [rng.standard_normal(o.shape) for _ in range(3)]
    hist = [o.fields()]
    for n in range(3):
        o.step_custom(jz[n], jx[n], jy[n])
        hist.append(o.fields())
    inode, icell = _interior_nodes(o), _interior_cells(o)
    assert inode.sum() > 10 and icell.sum() > 10
    # (35): qe^{n+1/2} - qe^{n-1/2} = dt (P_x^T jbar_x + P_y^T jbar_y + P_z^T jz^n)
    for n in (1, 2):
        qe1 = o.qbar_e(hist[n + 1]["ex"], hist[n]["ex"], hist[n + 1]["ey"], hist[n]["ey"], hist[n + 1]["ez"])
        qe0 = o.qbar_e(hist[n]["ex"], hist[n - 1]["ex"], hist[n]["ey"], hist[n - 1]["ey"], hist[n]["ez"])
        jbx = 0.5 * (jx[n] + jx[n - 1]) * (o.coef("ex") != 0)
        jby = 0.5 * (jy[n] + jy[n - 1]) * (o.coef("ey") != 0)
        jbz = jz[n] * (o.coef("ez") != 0)
        div = np.zeros(o.shape)
        # (P^T v)[node] = v[node - s] - v[node], written on the 3-D array
        div += -jbx
        div[:, :, 1:] += jbx[:, :, :-1]
        div += -jby
        div[:, 1:, :] += jby[:, :-1, :]
        div += -jbz
        div[1:, :, :] += jbz[:-1, :, :]
        res = (qe1 - qe0) - o.dt * div
        scale = np.max(np.abs(qe1[inode]))
        assert np.max(np.abs(res[inode])) <= 1e-12 * scale
    # (34): qh^n constant
    qh = [o.qbar_h(hist[n + 1]["hx"], hist[n]["hx"], hist[n + 1]["hy"], hist[n]["hy"], hist[n]["hz"])
          for n in range(3)]
    scale = np.max(np.abs(qh[0][icell]))
    for n in (1, 2):
        assert np.max(np.abs(qh[n][icell] - qh[0][icell])) <= 1e-12 * scale


def test_sign_of_the_r_term_in_the_charge():
    """The printed (I + alpha^2 r_0) does not give a conserved charge; the
    reading (I - alpha^2 r_0) does (previous test). Flip the correction and
    the residual becomes O(1)."""
    nx, ny, nz = 5, 5, 6
    o = Oracle(nx, ny, nz, DXY, DXY, MM)
    _random_state(o, 31)
    h = [o.fields()]
    for _ in range(2):
        o.step_custom()
        h.append(o.fields())
    inode = _interior_nodes(o)

    def qe_plus(n):
        # the same charge but with the alpha^2 correction added instead of subtracted:
        base = o.qbar_e(h[n + 1]["ex"], h[n]["ex"], h[n + 1]["ey"], h[n]["ey"], h[n + 1]["ez"])
        ez = h[n + 1]["ez"]
        zero = np.zeros_like(ez)
        plain = o.qbar_e(zero, zero, zero, zero, ez)          # -P_z^T dz~ only
        no_r = -_ptz(ez * _inv(o.coef("ez")))                 # -P_z^T M_eps ez
        return base - 2.0 * (plain - no_r)

    res_plus = qe_plus(1) - qe_plus(0)
    scale = np.max(np.abs(qe_plus(0)[inode]))
    assert np.max(np.abs(res_plus[inode])) > 1e-3 * scale


def _inv(c):
    out = np.zeros_like(c)
    out[c != 0] = 1.0 / c[c != 0]
    return out


def _ptz(v):
    out = -v.copy()
    out[1:, :, :] += v[:-1, :, :]
    return out


def _node_charge_closed_form(q, sigma, dz, zc, k):
    """Charge of the truncated Gaussian inside the dual cell [z_k - dz/2, z_k + dz/2]."""
    a = max(k * dz - 0.5 * dz - zc, -5 * sigma)
    b = min(k * dz + 0.5 * dz - zc, 5 * sigma)
    if b <= a:
        return 0.0
    return q * 0.5 * (math.erf(b / (sigma * math.sqrt(2))) - math.erf(a / (sigma * math.sqrt(2))))


def test_gauss_law_for_the_bunch():
    """Cold start: qe^{n+1/2} equals the bunch charge in each node's dual cell
    on the bunch line and vanishes at every other interior node (Eq. (35)
    summed over the steps)."""
    nx, ny, nz = 10, 10, 40
    q = 1e-9
    sigma = 2.5 * MM
    o = Oracle(nx, ny, nz, DXY, DXY, MM)
    o.set_bunch(sigma, q, 5, 5)
    c0 = o.bunch_info()["c0"]
    inode = _interior_nodes(o)
    for n in (6, 13, 20, 29):
        o2 = Oracle(nx, ny, nz, DXY, DXY, MM)
        o2.set_bunch(sigma, q, 5, 5)
        o2.step(n)
        f0 = o2.fields()
        o2.step(1)
        f1 = o2.fields()
        qe = o2.qbar_e(f1["ex"], f0["ex"], f1["ey"], f0["ey"], f1["ez"])
        zc = (n + 0.5 - c0) * MM
        expect = np.zeros(o.shape)
        for k in range(nz + 1):
            expect[k, 5, 5] = _node_charge_closed_form(q, sigma, MM, zc, k)
        assert np.max(np.abs(qe[inode] - expect[inode])) <= 1e-12 * q
        if n >= 13:
            assert np.max(np.abs(expect[inode])) > 0.05 * q


# ---------------------------------------------------------------------------
# Zero dispersion along z (Sec. 4.5): exact one-cell shift of a TEM pulse
# ---------------------------------------------------------------------------

def _tem_potential(nx, ny, dx, dy, i0, j0):
    """phi on the nodes of the cross-section: (dy/dx P_x^T P_x + dx/dy P_y^T P_y) phi
    = delta(i0, j0) at interior nodes, phi = 0 on the PEC wall."""
    idx = {}
    for j in range(1, ny):
        for i in range(1, nx):
            idx[(i, j)] = len(idx)
    a = np.zeros((len(idx), len(idx)))
    wx, wy = dy / dx, dx / dy
    for (i, j), r in idx.items():
        a[r, r] = 2 * wx + 2 * wy
        for (ii, jj), w in (((i + 1, j), wx), ((i - 1, j), wx), ((i, j + 1), wy), ((i, j - 1), wy)):
            if (ii, jj) in idx:
                a[r, idx[(ii, jj)]] -= w
    b = np.zeros(len(idx))
    b[idx[(i0, j0)]] = 1.0
    x = np.linalg.solve(a, b)
    phi = np.zeros((ny + 1, nx + 1))
    for (i, j), r in idx.items():
        phi[j, i] = x[r]
    return phi


def test_tem_pulse_shifts_one_cell_per_step():
    nx, ny, nz = 6, 5, 40
    dx, dy, dz = DXY, 1.2 * DXY, MM
    i0, j0 = 3, 2
    phi = _tem_potential(nx, ny, dx, dy, i0, j0)
    pxp = np.zeros_like(phi)
    pyp = np.zeros_like(phi)
    pxp[:, :-1] = phi[:, 1:] - phi[:, :-1]
    pyp[:-1, :] = phi[1:, :] - phi[:-1, :]
    eta0 = MU0 * C_LIGHT
    kk = np.arange(nz + 1)

    def F(k):
        k = np.asarray(k, dtype=float)
        x = (k - 8.0) / 3.0
        return np.where(np.abs(x) < 1.0, (1 - x * x) ** 3, 0.0)

    o = Oracle(nx, ny, nz, dx, dy, dz)
    sh = o.shape
    f0 = F(kk)[:, None, None]
    f1 = F(kk + 1)[:, None, None]
    o.set("ex", -pxp[None] * f0 * np.ones(sh))
    o.set("ey", -pyp[None] * f0 * np.ones(sh))
    o.set("hx", (dx / dy) * pyp[None] * f1 / eta0 * np.ones(sh))
    o.set("hy", -(dy / dx) * pxp[None] * f1 / eta0 * np.ones(sh))
    nsteps = 20
    for n in range(nsteps):
        jz = np.zeros(sh)
        jz[:nz, j0, i0] = 0.5 * (F(kk[:nz] + 1 - n) + F(kk[:nz] - n)) / eta0
        o.step_custom(jz)
    fN = F(kk - nsteps)[:, None, None]
    fN1 = F(kk + 1 - nsteps)[:, None, None]
    ex_exp = -pxp[None] * fN * (o.coef("ex") != 0)
    ey_exp = -pyp[None] * fN * (o.coef("ey") != 0)
    hx_exp = (dx / dy) * pyp[None] * fN1 / eta0 * (o.coef("hx") != 0)
    hy_exp = -(dy / dx) * pxp[None] * fN1 / eta0 * (o.coef("hy") != 0)
    escale = np.max(np.abs(ex_exp))
    hscale = np.max(np.abs(hx_exp))
    assert np.max(np.abs(o.get("ex") - ex_exp)) <= 1e-13 * escale
    assert np.max(np.abs(o.get("ey") - ey_exp)) <= 1e-13 * escale
    assert np.max(np.abs(o.get("hx") - hx_exp)) <= 1e-13 * hscale
    assert np.max(np.abs(o.get("hy") - hy_exp)) <= 1e-13 * hscale
    assert np.max(np.abs(o.get("ez"))) <= 1e-13 * escale
    assert np.max(np.abs(o.get("hz"))) <= 1e-13 * hscale


# ---------------------------------------------------------------------------
# Bunch, causality and the wake
# ---------------------------------------------------------------------------

def test_bunch_profile_closed_form():
    o = Oracle(8, 8, 30, DXY, DXY, MM)
    sigma, q = 3.3 * MM, 2e-9
    o.set_bunch(sigma, q, 4, 4)
    info = o.bunch_info()
    assert info["c0"] == math.ceil(5 * 3.3)
    assert info["qcell"].sum() == pytest.approx(q * math.erf(5 / math.sqrt(2)), rel=1e-13)
    # current of step n on edge k is c*Q_cell(k - n + c0)/dz
    n = 7
    jz = o.current(n)
    c0 = info["c0"]
    for k in range(30):
        d = k - n + c0
        qc = info["qcell"][d + c0] if -c0 <= d < c0 else 0.0
        assert jz[k, 4, 4] == pytest.approx(C_LIGHT * qc / MM, rel=1e-15, abs=0)


def test_no_field_ahead_of_the_bunch():
    w = wl.plain_pipe(nz=60, n=10, steps=0)
    o = Oracle(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt)
    o.set_bunch(w.sigma, w.charge, w.i0, w.j0)
    for n in (10, 25, 40):
        o.step(n - o.step_count)
        for c in oracle.COMPONENTS:
            f = o.get(c)
            assert np.all(f[n + 1:] == 0.0), (c, n)
            assert np.any(f[:n] != 0.0)
    wk, s0, ds = o.wake()
    info = o.bunch_info()
    assert s0 == pytest.approx(info["m_min"] * MM)
    # samples ahead of the head are exactly zero
    c0 = info["c0"]
    assert wk[0] == 0.0 and wk[1] == 0.0          # m = -c0-1 and m = -c0


def test_loss_factor_identity():
    """Energy law (19) summed over the whole passage: the field energy left
    behind equals Q/2 * sum_d Q_cell(d) [W(-d) + W(-d-1)]."""
    nx, ny, nz = 8, 8, 30
    sigma = 2.0 * MM
    o = Oracle(nx, ny, nz, DXY, DXY, MM)
    q = 1e-9
    o.set_bunch(sigma, q, 4, 4)
    info = o.bunch_info()
    c0 = info["c0"]
    o.step(nz + 2 * c0 + info["m_max"])
    wk, s0, ds = o.wake()
    m_min = info["m_min"]
    rhs = 0.0
    for d in range(-c0, c0):
        qc = info["qcell"][d + c0]
        rhs += 0.5 * q * qc * (wk[-d - m_min] + wk[-d - 1 - m_min])
    assert o.energy() == pytest.approx(rhs, rel=1e-12)
    assert o.energy() > 0


def test_wake_independent_of_charge_and_symmetric():
    w = wl.plain_pipe(nz=40, n=8, steps=0)
    res = []
    for q in (1e-9, 3e-12):
        o = Oracle(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz)
        o.set_bunch(3 * MM, q, 4, 4)
        o.step(90)
        res.append(o)
    w1, w2 = res[0].wake()[0], res[1].wake()[0]
    np.testing.assert_allclose(w1, w2, rtol=1e-12, atol=1e-12 * np.max(np.abs(w1)))
    # square pipe, on-axis bunch: ex(i+1/2, j) = ey(j, i+1/2) (x <-> y mirror)
    ex, ey = res[0].get("ex"), res[0].get("ey")
    np.testing.assert_allclose(ex, np.swapaxes(ey, 1, 2), atol=1e-12 * np.max(np.abs(ex)))


def test_as_written_cubic_config_fails_stability_check():
    w = wl.plain_pipe_cubic()
    assert not oracle.stable(w.dx, w.dy, w.dz, w.cdt)
    w2 = wl.plain_pipe()
    assert oracle.stable(w2.dx, w2.dy, w2.dz, w2.cdt)


# ---------------------------------------------------------------------------
# Static start: the bunch enters from an infinite ingoing pipe (Sec. 5) with
# its discrete TEM field; at c*dt = dz that field moves one cell per step
# (Sec. 4.5), so a smooth pipe radiates nothing
# ---------------------------------------------------------------------------

def _round_pipe(nx, ny, nz, radius_of_k):
    return wl.radius_mask(nx, ny, nz, radius_of_k)


def test_static_start_moves_rigidly_and_leaves_no_wake_in_a_smooth_pipe():
    nx = ny = 14
    nz = 90
    pec = _round_pipe(nx, ny, nz, lambda k: np.full(k.shape, 5.5))
    sigma, q, K = 3 * MM, 1e-9, 34
    o = Oracle(nx, ny, nz, DXY, DXY, MM, pec=pec)
    o.set_bunch_static(sigma, q, 7, 7, K)
    assert o.kshift == K
    f0 = o.fields()
    assert not f0["ez"].any() and not f0["hz"].any()
    n = 40
    o.step(n)
    escale, hscale = np.max(np.abs(f0["ex"])), np.max(np.abs(f0["hx"]))
    for c in oracle.COMPONENTS:
        shifted = np.zeros_like(f0[c])
        shifted[n:] = f0[c][:-n]
        scale = escale if c[0] == "e" else hscale
        assert np.max(np.abs(o.get(c) - shifted)) <= 1e-13 * scale, c
    cold = Oracle(nx, ny, nz, DXY, DXY, MM, pec=pec)
    cold.set_bunch(sigma, q, 7, 7)
    cold.step(n + K)
    assert np.max(np.abs(o.wake()[0])) <= 1e-13 * np.max(np.abs(cold.wake()[0]))


def test_static_start_gauss_law():
    """The static field carries the bunch charge from the first step on: the
    node charges of Eq. (35) equal the closed-form charges of the shifted
    bunch at the bunch nodes and vanish elsewhere."""
    nx = ny = 12
    nz = 70
    pec = _round_pipe(nx, ny, nz, lambda k: np.where((k >= 40) & (k < 50), 5.5, 4.5))
    q, sigma, K = 1e-9, 2.5 * MM, 30
    c0 = math.ceil(5 * sigma / MM - 1e-12)
    for n in (0, 7, 21):
        o = Oracle(nx, ny, nz, DXY, DXY, MM, pec=pec)
        o.set_bunch_static(sigma, q, 6, 6, K)
        o.step(n)
        f0 = o.fields()
        o.step(1)
        f1 = o.fields()
        qe = o.qbar_e(f1["ex"], f0["ex"], f1["ey"], f0["ey"], f1["ez"])
        zc = (n + K + 0.5 - c0) * MM
        expect = np.zeros(o.shape)
        for k in range(nz + 1):
            expect[k, 6, 6] = _node_charge_closed_form(q, sigma, MM, zc, k)
        inode = _interior_nodes(o)
        assert np.max(np.abs(qe[inode] - expect[inode])) <= 1e-12 * q
        assert np.max(np.abs(expect[inode])) > 0.05 * q


def test_static_start_energy_identity_in_a_cavity():
    """Energy law (19) summed over the passage (until the bunch has left the
    grid): W^N - W^0 = Q/2 sum_d Q_cell(d) [W(m_d) + W(m_d - 1)], with the
    static field's own energy in W^0."""
    nx = ny = 12
    nz = 60
    pec = _round_pipe(nx, ny, nz, lambda k: np.where((k >= 30) & (k < 40), 5.5, 3.5))
    q, sigma, K = 1e-9, 2.0 * MM, 24
    o = Oracle(nx, ny, nz, DXY, DXY, MM, pec=pec)
    o.set_bunch_static(sigma, q, 6, 6, K)
    w0 = o.energy()
    assert w0 > 0
    o.step(nz - (K - 2 * math.ceil(5 * sigma / MM - 1e-12)) + 1)
    wk, s0, ds = o.wake()
    info = o.bunch_info()
    c0, m_min = info["c0"], info["m_min"]
    rhs = 0.0
    for d in range(-c0, c0):
        rhs += 0.5 * q * info["qcell"][d + c0] * (wk[-d - m_min] + wk[-d - 1 - m_min])
    assert o.energy() - w0 == pytest.approx(rhs, rel=1e-10, abs=1e-12 * w0)
    assert abs(rhs) > 1e-6 * w0                       # the cavity takes energy from the bunch


def test_static_start_rejects_what_it_cannot_represent():
    nx = ny = 10
    nz = 60
    pec = _round_pipe(nx, ny, nz, lambda k: np.where(k < 20, 4.5, 3.5))
    o = Oracle(nx, ny, nz, DXY, DXY, MM, pec=pec)
    with pytest.raises(ValueError):
        o.set_bunch_static(2 * MM, 1e-9, 5, 5, 30)        # entry section not uniform up to K
    with pytest.raises(ValueError):
        Oracle(nx, ny, nz, DXY, DXY, MM, pec=pec).set_bunch_static(2 * MM, 1e-9, 5, 5, 12)  # K < 2 c0 + 2
    eps = np.ones((nz, ny, nx))
    with pytest.raises(ValueError):
        Oracle(nx, ny, nz, DXY, DXY, MM, eps_r=eps, pec=pec).set_bunch_static(MM, 1e-9, 5, 5, 15)


# ---------------------------------------------------------------------------
# Transverse wake (Sec. 5: the dipole wake of off-axis bunches and deflecting
# structures), W_perp = (1/Q) integral of (E + c z^ x B)_perp along the path.
# The Panofsky-Wenzel theorem dW_perp/ds = grad_perp W_par holds exactly in
# the scheme at c*dt = dz between W_x on the x-edge line (i+1/2, j) and the
# longitudinal wakes on the node lines i and i+1, with the half-sample
# average the staggering asks for (likewise W_y with the lines j and j+1):
#   W_x(m+1) - W_x(m) = dz/dx * [(W_{i+1} - W_i)(m) + (W_{i+1} - W_i)(m+1)] / 2
# ---------------------------------------------------------------------------

def _cavity_box(nx, ny, nz, ic, jc, r_pipe, r_cav, k_lo, k_hi):
    jj, ii = np.mgrid[0:ny, 0:nx]
    pec = np.zeros((nz, ny, nx), np.uint8)
    for k in range(nz):
        r = r_cav if k_lo <= k < k_hi else r_pipe
        pec[k] = ((ii + 0.5 - ic) ** 2 + (jj + 0.5 - jc) ** 2) > r * r
    return pec


@pytest.mark.parametrize("bunch,obs", [((6, 5), (5, 5)), ((5, 5), (5, 5)), ((5, 6), (4, 4)),
                                       ((6, 4), (6, 6))])
def test_discrete_panofsky_wenzel_3d(bunch, obs):
    nx, ny, nz = 10, 10, 60
    pec = _cavity_box(nx, ny, nz, 5, 5, 3.2, 4.4, 25, 35)
    sigma = 2 * MM
    o = Oracle(nx, ny, nz, DXY, DXY, MM, pec=pec)
    o.set_bunch(sigma, 1e-9, *bunch)
    o.set_observer(*obs)
    c0 = math.ceil(5 * sigma / MM - 1e-12)
    o.step(nz + 2 * c0 + math.ceil(15 * sigma / MM) + 2)
    wx, wy = o.transverse_wake()
    w00, w10, w01 = o.wake_at_observer()
    for w, nb in ((wx, w10), (wy, w01)):
        grad = (nb - w00) * (MM / DXY)
        rhs = 0.5 * (grad[:-1] + grad[1:])
        assert np.max(np.abs(rhs)) > 0
        np.testing.assert_allclose(np.diff(w), rhs, rtol=0, atol=1e-12 * np.max(np.abs(rhs)))
    if tuple(obs) == tuple(bunch):  # the default observer is the bunch line
        np.testing.assert_array_equal(w00, o.wake()[0])


def test_transverse_wake_mirror_antisymmetry():
    """Geometry and bunch symmetric about the planes x = x_i0 and y = y_j0:
    the x-edge lines i0 +- 1/2 are mirror images, so W_x there is equal and
    opposite (likewise W_y on j0 +- 1/2)."""
    nx = ny = 10
    nz = 50
    pec = _cavity_box(nx, ny, nz, 5, 5, 3.2, 4.4, 20, 30)
    pec[20:30, 2, 1:4] = 1                       # a symmetric set of posts breaks the
    pec[20:30, 2, 6:9] = 1                       # rotational symmetry, not the mirror ones
    pec[20:30, 7, 1:4] = 1
    pec[20:30, 7, 6:9] = 1
    out = {}
    for obs in ((5, 5), (4, 5), (5, 4)):
        o = Oracle(nx, ny, nz, DXY, DXY, MM, pec=pec)
        o.set_bunch(2 * MM, 1e-9, 5, 5)
        o.set_observer(*obs)
        o.step(nz + 20 + 30 + 2)
        out[obs] = o.transverse_wake()
    # W_x on (5 + 1/2, 5) mirrors W_x on (4 + 1/2, 5); W_y on (5, 5 + 1/2) mirrors (5, 4 + 1/2)
    for c, mirror in ((0, (4, 5)), (1, (5, 4))):
        a, b = out[(5, 5)][c], out[mirror][c]
        assert np.max(np.abs(a)) > 0
        np.testing.assert_allclose(a, -b, rtol=0, atol=1e-12 * np.max(np.abs(a)))


def test_transverse_wake_of_the_static_tem_field_vanishes():
    """The bunch's own discrete TEM field (static start) exerts no force on a
    test charge moving with it: in a smooth pipe the transverse wake of an
    off-axis bunch stays zero, while the cold start's entry transient gives
    one."""
    nx = ny = 14
    nz = 90
    pec = _round_pipe(nx, ny, nz, lambda k: np.full(k.shape, 5.5))
    sigma, q, K = 3 * MM, 1e-9, 34
    o = Oracle(nx, ny, nz, DXY, DXY, MM, pec=pec)
    o.set_bunch_static(sigma, q, 8, 7, K)
    o.set_observer(6, 7)
    o.step(40)
    cold = Oracle(nx, ny, nz, DXY, DXY, MM, pec=pec)
    cold.set_bunch(sigma, q, 8, 7)
    cold.set_observer(6, 7)
    cold.step(40 + K)
    for a, b in zip(o.transverse_wake(), cold.transverse_wake()):
        assert np.max(np.abs(b)) > 0
        assert np.max(np.abs(a)) <= 1e-13 * np.max(np.abs(b))


def test_observer_arguments_and_state():
    o = Oracle(6, 6, 20, DXY, DXY, MM)
    with pytest.raises(ValueError):
        o.set_observer(2, 2)                      # no bunch
    o.set_bunch(MM, 1e-9, 3, 3)
    for bad in ((-1, 2), (6, 2), (2, 6)):
        with pytest.raises(ValueError):
            o.set_observer(*bad)
    o.set_observer(5, 5)
    o.step(1)
    with pytest.raises(ValueError):
        o.set_observer(2, 2)                      # after the first step


def test_cavity_mode_frequency_converges_at_second_order():
    """The continuous limit of the scheme: the TM_111 frequency of a rectangular
    PEC box, c pi ((1/a)^2 + (1/b)^2 + (1/d)^2)^(1/2) (Maxwell's equations, no
    discretisation), is approached as O(h^2) when the mesh is refined at fixed
    c dt = dz. The frequency is measured from the time series of the e_z
    pattern's projection by the three-term recurrence p(n+1) + p(n-1) =
    2 cos(w dt) p(n) + const (the constant carries the static part)."""
    errs = []
    for f in (1, 2, 4):
        nx, ny, nz = 6 * f, 6 * f, 8 * f
        dx, dy, dz = DXY / f, DXY / f, MM / f
        o = Oracle(nx, ny, nz, dx, dy, dz)
        i, j, k = np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1)
        ez = (np.cos(np.pi * (k + 0.5) / nz)[:, None, None] * np.sin(np.pi * j / ny)[None, :, None]
              * np.sin(np.pi * i / nx)[None, None, :])
        ez = np.where(o.coef("ez") > 0, ez, 0.0)
        o.set("ez", ez)
        p = []
        for _ in range(160 * f):
            o.step(1)
            p.append(float(np.sum(o.get("ez") * ez)))
        p = np.array(p)
        a = np.column_stack([2.0 * p[1:-1], np.ones(len(p) - 2)])
        (c, _), *_ = np.linalg.lstsq(a, p[2:] + p[:-2], rcond=None)
        w = math.acos(c) / o.dt
        w_cont = C_LIGHT * math.pi * math.sqrt((nx * dx) ** -2 + (ny * dy) ** -2 + (nz * dz) ** -2)
        errs.append(abs(w - w_cont) / w_cont)
    assert errs[0] < 0.05
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs
