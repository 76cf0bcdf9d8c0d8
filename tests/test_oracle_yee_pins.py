"""Pins of the oracle's Yee scheme (Sec. 3, Eq. (7)), the E/M leapfrog the paper
measures the TE/TM scheme against, on the same grid doublet and material
matrices (oracle/tetm_oracle.c, ``oracle_yee_step``).

What fixes it, other than itself:
* the eigen-angles of its one-step propagator on a PEC box against the
  closed-form dispersion relation (9) (standing waves K = p*pi/(2N));
* the step bound (8): no growth at the bound, growth above it, and growth at
  the TE/TM scheme's step c*dt = dz on the paper's mesh dx = dy = sqrt(2) dz;
* the leapfrog energy 1/2 e^{n+1/2} M_eps e^{n+1/2} + 1/2 h^n M_mu h^{n+1},
  conserved exactly (to rounding) by the exact skew form of Eq. (7);
* the z-dispersion of a TEM pulse on a coaxial line against the closed form of
  Eq. (10), and its phase error against the dispersion-free motion (Eq. (11)).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import Oracle

MM = 1e-3
DXY = math.sqrt(2.0) * MM


def yee_bound(dx, dy, dz):
    return 1.0 / math.sqrt(dx ** -2 + dy ** -2 + dz ** -2)


def active_index(o):
    """(component, flat index) of every entry with a non-zero coefficient."""
    out = []
    for c in range(6):
        nz = np.nonzero(o.coef(c).ravel() > 0)[0]
        out += [(c, int(q)) for q in nz]
    return out


def yee_propagator(o, act):
    n = len(act)
    g = np.empty((n, n))
    for col, (c, q) in enumerate(act):
        for cc in range(6):
            o.set(cc, np.zeros(o.shape))
        f = np.zeros(o.shape).ravel()
        f[q] = 1.0
        o.set(c, f.reshape(o.shape))
        o.yee_step(1)
        fl = [o.get(cc).ravel() for cc in range(6)]
        g[:, col] = [fl[cc][qq] for cc, qq in act]
    return g


def closed_form_angles_9(nx, ny, nz, dx, dy, dz, cdt):
    """Eq. (9): sin^2 W / dtau^2 = sum_a sin^2 K_a / d_a^2 with W = omega dtau/(2c),
    K_a = p_a pi/(2 N_a) for the standing waves of the box; one step turns a
    mode by 2W. Two polarisations if p, q, r >= 1, one if exactly one is 0."""
    out = []
    for p in range(nx):
        for q in range(ny):
            for r in range(nz):
                zeros = (p == 0) + (q == 0) + (r == 0)
                mult = {0: 2, 1: 1}.get(zeros, 0)
                if not mult:
                    continue
                s2 = cdt ** 2 * (math.sin(p * math.pi / (2 * nx)) ** 2 / dx ** 2
                                 + math.sin(q * math.pi / (2 * ny)) ** 2 / dy ** 2
                                 + math.sin(r * math.pi / (2 * nz)) ** 2 / dz ** 2)
                out += [2.0 * math.asin(math.sqrt(s2))] * mult
    return np.sort(np.array(out))


@pytest.mark.parametrize("dims,steps,frac", [((3, 4, 5), (DXY, DXY, MM), 0.97),
                                             ((4, 3, 4), (1.7 * MM, 1.5 * MM, MM), 0.6)])
def test_yee_eigen_angles_match_dispersion_relation_9(dims, steps, frac):
    nx, ny, nz = dims
    dx, dy, dz = steps
    cdt = frac * yee_bound(dx, dy, dz)
    assert oracle.yee_stable(dx, dy, dz, cdt)
    o = Oracle(nx, ny, nz, dx, dy, dz, cdt=cdt)
    g = yee_propagator(o, active_index(o))
    lam = np.linalg.eigvals(g)
    assert np.max(np.abs(lam)) < 1.0 + 1e-9
    ang = np.angle(lam)
    pos = np.sort(ang[ang > 1e-7])
    expect = closed_form_angles_9(nx, ny, nz, dx, dy, dz, cdt)
    assert len(pos) == len(expect)
    np.testing.assert_allclose(pos, expect, atol=1e-9)
    # the rotating modes sit on the unit circle
    rot = lam[np.abs(np.angle(lam)) > 1e-7]
    np.testing.assert_allclose(np.abs(rot), 1.0, atol=1e-9)


def test_yee_step_bound_8():
    nx, ny, nz = 3, 4, 5
    b = yee_bound(DXY, DXY, MM)
    assert abs(b - MM / math.sqrt(2.0)) < 1e-15
    assert oracle.yee_stable(DXY, DXY, MM, b) and not oracle.yee_stable(DXY, DXY, MM, 1.001 * b)
    o = Oracle(nx, ny, nz, DXY, DXY, MM, cdt=b)
    assert np.max(np.abs(np.linalg.eigvals(yee_propagator(o, active_index(o))))) < 1.0 + 1e-9
    # above the bound the highest standing wave of this box grows (it needs
    # c*dt > 1.082 b here, Eq. (9) with |sin W| > 1)
    o = Oracle(nx, ny, nz, DXY, DXY, MM, cdt=1.2 * b)
    assert np.max(np.abs(np.linalg.eigvals(yee_propagator(o, active_index(o))))) > 1.05
    # the TE/TM scheme's "magic" step c*dt = dz is beyond Yee's bound on this mesh
    o = Oracle(nx, ny, nz, DXY, DXY, MM, cdt=MM)
    assert oracle.stable(DXY, DXY, MM, MM)
    assert np.max(np.abs(np.linalg.eigvals(yee_propagator(o, active_index(o))))) > 1.5


def test_yee_leapfrog_energy_is_conserved():
    nx, ny, nz = 6, 5, 7
    pec = np.zeros((nz, ny, nx), np.uint8)
    pec[2:4, 1:3, 3:5] = 1                           # an interior PEC block
    eps = np.ones((nz, ny, nx))
    eps[4:, :, :] = 2.5                              # a dielectric half
    o = Oracle(nx, ny, nz, DXY, 1.1 * DXY, MM, cdt=0.9 * yee_bound(DXY, 1.1 * DXY, MM),
               eps_r=eps, pec=pec)
    rng = np.random.default_rng(5)
    coef = [o.coef(c) for c in range(6)]
    for c in range(6):
        o.set(c, np.where(coef[c] > 0, rng.standard_normal(o.shape), 0.0))

    def energy_after_step():
        h0 = [o.get(c) for c in (3, 4, 5)]
        o.yee_step(1)
        w = 0.0
        for c in (0, 1, 2):
            a = coef[c] > 0
            w += 0.5 * np.sum(o.get(c)[a] ** 2 / coef[c][a])
        for c, hn in zip((3, 4, 5), h0):
            a = coef[c] > 0
            w += 0.5 * np.sum(hn[a] * o.get(c)[a] / coef[c][a])
        return w

    w0 = energy_after_step()
    for _ in range(12):
        o.yee_step(17)
        assert energy_after_step() == pytest.approx(w0, rel=1e-12)


def test_yee_keeps_inactive_entries_zero_and_refuses_a_bunch():
    o = Oracle(5, 5, 6, DXY, DXY, MM, cdt=0.7 * MM)
    rng = np.random.default_rng(2)
    coef = [o.coef(c) for c in range(6)]
    for c in range(6):
        o.set(c, np.where(coef[c] > 0, rng.standard_normal(o.shape), 0.0))
    o.yee_step(9)
    for c in range(6):
        assert np.all(o.get(c)[coef[c] == 0] == 0.0)
    b = Oracle(5, 5, 6, DXY, DXY, MM)
    b.set_bunch(2 * MM, 1e-9, 2, 2)
    with pytest.raises(ValueError):
        b.yee_step(1)


def test_yee_tem_pulse_on_a_coaxial_line_follows_eq_10():
    """The z-dispersion of Yee's scheme, Eq. (10). On a coaxial line (a PEC rod
    through the box) the discrete TEM field e = e0(x, y) a_k is curl-free and
    divergence-free across the section, so from h = 0 the 3D scheme keeps the
    fields separable and a_k follows a 1D leapfrog whose standing waves
    sin(r pi k / nz) turn with sin W = (c dt/dz) sin(r pi / (2 nz)) per half step:
    a^{n-1/2} = sum_r A_r cos((2n - 1) W_r) / cos(W_r) sin(r pi k / nz) from the
    sine coefficients A_r of the initial a^{-1/2}."""
    from paper_0901_1053_gb300 import workloads as wl
    nx = ny = 10
    nz = 240
    rod = (4, 6, 4, 6)
    cdt = 0.9 * yee_bound(DXY, DXY, MM)
    o = Oracle(nx, ny, nz, DXY, DXY, MM, cdt=cdt, pec=wl.coax_pec(nx, ny, nz, rod))
    e0x, e0y = wl.coax_tem_e(nx, ny, DXY, DXY, rod)
    k = np.arange(nz + 1)
    a0 = np.exp(-0.5 * ((k - 70.0) / 4.0) ** 2)
    a0[0] = a0[-1] = 0.0
    o.set(0, e0x[None] * a0[:, None, None])
    o.set(1, e0y[None] * a0[:, None, None])
    n = 150
    o.yee_step(n)
    ex, ey = o.get(0), o.get(1)
    j, i = np.unravel_index(np.argmax(np.abs(e0x)), e0x.shape)
    a = ex[:, j, i] / e0x[j, i]
    # separable: every e_x, e_y edge carries e0 * a_k; no e_z, h_z
    np.testing.assert_allclose(ex, e0x[None] * a[:, None, None], atol=1e-12 * np.abs(ex).max())
    np.testing.assert_allclose(ey, e0y[None] * a[:, None, None], atol=1e-12 * np.abs(ex).max())
    assert np.abs(o.get(2)).max() <= 1e-12 * np.abs(ex).max()
    assert np.abs(o.get(5)).max() <= 1e-12 * np.abs(o.get(3)).max()
    # closed form of Eq. (10)
    r = np.arange(1, nz)
    modes = np.sin(np.pi * np.outer(r, k) / nz)            # (nz-1, nz+1)
    amp = (2.0 / nz) * modes @ a0
    w = np.arcsin((cdt / MM) * np.sin(np.pi * r / (2 * nz)))
    pred = (amp * np.cos((2 * n - 1) * w) / np.cos(w)) @ modes
    assert np.max(np.abs(a - pred)) <= 1e-11 * np.max(np.abs(a0))
    # and it is not the dispersion-free motion (c dt < dz): the phase error of
    # Eq. (11) is visible after 150 steps
    w_exact = (cdt / MM) * np.pi * r / (2 * nz)
    exact = (amp * np.cos((2 * n - 1) * w_exact) / np.cos(w_exact)) @ modes
    assert np.max(np.abs(a - exact)) > 1e-3 * np.max(np.abs(a0))


def test_tetm_moves_the_coaxial_tem_pulse_without_dispersion():
    """The same pulse under the TE/TM scheme at c dt = dz (its "magic" step,
    Sec. 4.5): every standing wave turns at the exact frequency c k, so the
    field equals the dispersion-free motion of the initial e^0 (h^{-1/2} = 0):
    a^n = sum_r A_r cos((2n + 1) W_r) / cos(W_r) sin(r pi k / nz), W_r = r pi / (2 nz)."""
    from paper_0901_1053_gb300 import workloads as wl
    nx = ny = 10
    nz = 240
    rod = (4, 6, 4, 6)
    o = Oracle(nx, ny, nz, DXY, DXY, MM, cdt=MM, pec=wl.coax_pec(nx, ny, nz, rod))
    e0x, e0y = wl.coax_tem_e(nx, ny, DXY, DXY, rod)
    k = np.arange(nz + 1)
    a0 = np.exp(-0.5 * ((k - 70.0) / 4.0) ** 2)
    a0[0] = a0[-1] = 0.0
    o.set(0, e0x[None] * a0[:, None, None])
    o.set(1, e0y[None] * a0[:, None, None])
    n = 150
    o.step(n)
    j, i = np.unravel_index(np.argmax(np.abs(e0x)), e0x.shape)
    a = o.get(0)[:, j, i] / e0x[j, i]
    r = np.arange(1, nz)
    modes = np.sin(np.pi * np.outer(r, k) / nz)
    amp = (2.0 / nz) * modes @ a0
    w = np.pi * r / (2 * nz)
    exact = (amp * np.cos((2 * n + 1) * w) / np.cos(w)) @ modes
    assert np.max(np.abs(a - exact)) <= 1e-11 * np.max(np.abs(a0))
