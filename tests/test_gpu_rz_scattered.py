"""Scattered-field form of the rotationally symmetric static start
(tetm_rz_set_bunch_scattered, include/tetm_rz.h).

The device keeps the total field minus the incident field, the discrete TEM
field of the ring bunch in the entry section moving one plane per step
(Sec. 4.5). In exact arithmetic the solve is the static start's (Sec. 5), so:
the FP64 path matches the oracle's static start (oracle/tetm_rz_oracle.c) to
1e-12 of each field family, wake and energy; the four step kernels and any
chunk length give bit-identical results; and since the stored field carries
no near field of the bunch, FP32 wakes of every mode stay within 1e-4 of their
peak against the FP64 static start."""
import math

import numpy as np
import pytest

from oracle import RzOracle
from paper_0901_1053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32_WAKE = 1e-4
E_NAMES, H_NAMES = ("er", "ephi", "ez"), ("hr", "hphi", "hz")
KERNELS = ("async", "register", "bulk", "bulk2")


@pytest.fixture(scope="module")
def tetm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_1053_gb300 import tetm as t
    return t


def k_head(w):
    return 2 * math.ceil(5 * w.sigma / w.dz - 1e-12) + 2


def solver(tetm, w, chunk=None, kernel="async", precision=None):
    s = tetm.RzSolver(w.nr, w.nz, w.m_lo, w.m_hi, w.dr, w.dz, w.cdt, precision or w.precision,
                      pec=w.pec)
    s.set_kernel(kernel)
    if chunk:
        s.set_tiling(chunk)
    return s


def family_errors(gf, of):
    out = {}
    for fam in (E_NAMES, H_NAMES):
        peak = max(np.max(np.abs(of[c])) for c in fam)
        for c in fam:
            out[c] = float(np.max(np.abs(gf[c] - of[c])) / peak)
    return out


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("kernel", KERNELS)
def test_scattered_fp64_matches_oracle_static_start(tetm, kernel):
    """Three-cell chain, modes 0..4, the bunch through all cells and into the
    exit wall: total fields (incident part added back on readout), both wakes
    and the energy against the oracle's total-field static start."""
    w = wl.cavity_chain_rz(45, 160, 0, 4, sigma_cells=3.0, precision="fp64", n_cells=3, i0=4)
    K = k_head(w)
    s = solver(tetm, w, 20, kernel)
    s.set_bunch_scattered(w.sigma, w.charge, w.i0, K)
    n = w.steps - K + 41                     # odd: the two-step kernel ends on a one-step pass
    s.step(n)
    for m in range(5):
        o = RzOracle(w.nr, w.nz, m, w.dr, w.dz, w.cdt, pec=w.pec)
        o.set_bunch_static(w.sigma, w.charge, w.i0, K)
        o.step(n)
        errs = family_errors(s.fields(m), o.fields())
        assert max(errs.values()) <= TOL64, (m, errs)
        assert rel(s.wake(m)[0], o.wake()[0]) <= TOL64, m
        assert rel(s.transverse_wake(m), o.transverse_wake()) <= TOL64, m
        assert s.energy(m) == pytest.approx(o.energy(), rel=TOL64), m


def test_scattered_fp32_kernels_and_chunks_bitwise_identical(tetm):
    w = wl.cavity_chain_rz(96, 600, 0, 4, sigma_cells=4.0, precision="fp32", n_cells=4)
    K = k_head(w)
    n = 301
    ref = None
    for kernel in KERNELS:
        for chunk in (7, 32):
            s = solver(tetm, w, chunk, kernel)
            s.set_bunch_scattered(w.sigma, w.charge, w.i0, K)
            s.step(n)
            got = [np.concatenate([s.wake(m)[0], s.transverse_wake(m)]) for m in range(5)]
            got += [s.get(m, c) for m in (0, 4) for c in E_NAMES + H_NAMES]
            s.close()
            if ref is None:
                ref = got
                continue
            for a, b in zip(got, ref):
                assert np.array_equal(a, b), (kernel, chunk)


def test_scattered_fp32_wakes_of_every_mode_within_1e4(tetm):
    """Nine-cell chain scaled to 128 x 2048 (ring at nr/64, sigma = 8 dz, as
    the full workload): every longitudinal and transverse wake of modes 0..4
    in float32 within 1e-4 of its peak, against the float64 total-field static
    start (itself held to the oracle in tests/test_gpu_rz.py)."""
    w = wl.cavity_chain_rz(128, 2048, 0, 4, precision="fp32")
    K = k_head(w)
    n = w.steps - K
    s = solver(tetm, w, 32, "bulk2")
    s.set_bunch_scattered(w.sigma, w.charge, w.i0, K)
    s.step(n)
    r = solver(tetm, w, 32, "bulk", precision="fp64")
    r.set_bunch_static(w.sigma, w.charge, w.i0, K)
    r.step(n)
    for m in range(5):
        assert rel(s.wake(m)[0], r.wake(m)[0]) <= TOL32_WAKE, m
        assert rel(s.transverse_wake(m), r.transverse_wake(m)) <= TOL32_WAKE, m


def test_scattered_fields_round_trip(tetm):
    """Total fields read and written back (the incident part subtracted on
    the way in) continue the solve as if uninterrupted."""
    w = wl.cavity_chain_rz(40, 140, 1, 2, sigma_cells=3.0, precision="fp64", n_cells=2, i0=3)
    K = k_head(w)
    a, b = solver(tetm, w), solver(tetm, w)
    for s in (a, b):
        s.set_bunch_scattered(w.sigma, w.charge, w.i0, K)
        s.step(37)
    for m in (1, 2):
        for c in E_NAMES + H_NAMES:
            b.set(m, c, b.get(m, c))
    a.step(50)
    b.step(50)
    for m in (1, 2):
        errs = family_errors(b.fields(m), a.fields(m))
        assert max(errs.values()) <= TOL64, (m, errs)
        assert rel(b.wake(m)[0], a.wake(m)[0]) <= TOL64


def test_scattered_errors(tetm):
    w = wl.cavity_chain_rz(30, 120, 0, 1, sigma_cells=3.0, precision="fp64", n_cells=2, i0=3)
    K = k_head(w)
    s = solver(tetm, w)
    with pytest.raises(tetm.TetmError) as e:
        s.set_bunch_scattered(w.sigma, w.charge, 3, K - 1)     # head too close to the wall
    assert e.value.code == tetm.TETM_E_ARG
    with pytest.raises(tetm.TetmError) as e:
        s.set_bunch_scattered(w.sigma, w.charge, 3, 100)       # past the entry pipe
    assert e.value.code == tetm.TETM_E_ARG
    s.set_bunch_scattered(w.sigma, w.charge, 3, K)
    with pytest.raises(tetm.TetmError) as e:
        s.set_bunch_scattered(w.sigma, w.charge, 3, K)
    assert e.value.code == tetm.TETM_E_STATE
    # a section narrower than the entry pipe downstream: the incident field
    # would sit inside the wall
    pec = wl.rz_radius_mask(30, 120, lambda k: np.where((k >= 60) & (k < 70), 6.0, 12.0))
    n = tetm.RzSolver(30, 120, 0, 1, w.dr, w.dz, w.cdt, "fp64", pec=pec)
    with pytest.raises(tetm.TetmError) as e:
        n.set_bunch_scattered(w.sigma, w.charge, 3, K)
    assert e.value.code == tetm.TETM_E_ARG
