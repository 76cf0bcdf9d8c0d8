"""GPU parity of the rotationally symmetric solver (Sec. 4.3, Eq. (24)): the
CUDA path through the C ABI (include/tetm_rz.h) against the FP64 CPU oracle
(oracle/tetm_rz_oracle.c), mode by mode.

Tolerances as for the 3D solver: FP64 fields and wakes within 1e-12 of the
peak of each field family or wake (the sides differ only by FMA contraction
and the order in which the diagonal factor of (24) is applied); FP32 fields
with FP64 wake sums: wakes within 1e-4 of their peak for m <= 2 (higher
modes: see test_fp32_wakes_against_oracle)."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import RzOracle
from paper_0901_1053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32_WAKE = 1e-4
E_NAMES, H_NAMES = ("er", "ephi", "ez"), ("hr", "hphi", "hz")


@pytest.fixture(scope="module")
def tetm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_1053_gb300 import tetm as t
    return t


def small_chain(nr, nz, m_lo, m_hi, sigma_cells=3.0, i0=None, steps=None, precision="fp64",
                n_cells=3):
    w = wl.cavity_chain_rz(nr, nz, m_lo, m_hi, sigma_cells=sigma_cells, precision=precision,
                           n_cells=n_cells, i0=i0)
    if steps is not None:
        w.steps = steps
    return w


def gpu_solver(tetm, w, chunk=None, kernel="async"):
    s = tetm.RzSolver(w.nr, w.nz, w.m_lo, w.m_hi, w.dr, w.dz, w.cdt, w.precision, pec=w.pec)
    s.set_kernel(kernel)
    if chunk:
        s.set_tiling(chunk)
    return s


def oracle_mode(w, m, steps=None, fields=None, bunch=True):
    o = RzOracle(w.nr, w.nz, m, w.dr, w.dz, w.cdt, pec=w.pec)
    if fields is not None:
        for c, a in fields.items():
            o.set(c, a)
    if bunch:
        o.set_bunch(w.sigma, w.charge, w.i0)
    o.step(w.steps if steps is None else steps)
    return o


def family_errors(gf, of, rows=None):
    out = {}
    for fam in (E_NAMES, H_NAMES):
        sl = slice(None) if rows is None else slice(0, rows)
        peak = max(np.max(np.abs(of[c][sl])) for c in fam)
        for c in fam:
            out[c] = float(np.max(np.abs(gf[c][sl] - of[c][sl])) / peak) if peak > 0 else \
                float(np.max(np.abs(gf[c][sl])))
    return out


def rel(a, b):
    peak = np.max(np.abs(b))
    return float(np.max(np.abs(a - b)) / peak)


# ---------------------------------------------------------------------------
# FP64 parity, field by field and wake by wake
# ---------------------------------------------------------------------------

KERNELS = ("async", "register", "bulk", "bulk2")


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("chunk", [5, 32, 200])
def test_axis_bunch_m0_matches_oracle(tetm, chunk, kernel):
    """m = 0, bunch on the axis, 3-cell chain, 61 radial entries (3 tiles, the
    last ragged), nz = 150 (chunks with a ragged tail)."""
    w = small_chain(60, 150, 0, 0, steps=None)
    s = gpu_solver(tetm, w, chunk, kernel)
    s.set_bunch(w.sigma, w.charge, w.i0)
    s.step(w.steps)
    o = oracle_mode(w, 0)
    errs = family_errors(s.fields(0), o.fields())
    assert max(errs.values()) <= TOL64, errs
    assert rel(s.wake(0)[0], o.wake()[0]) <= TOL64
    assert s.wake(0)[1] == o.wake()[1]


@pytest.mark.parametrize("kernel", KERNELS)
def test_ring_bunch_modes_0_to_3_match_oracle(tetm, kernel):
    w = small_chain(45, 120, 0, 3, i0=4, steps=150)
    s = gpu_solver(tetm, w, 16, kernel)
    s.set_bunch(w.sigma, w.charge, w.i0)
    s.step(w.steps)
    for m in range(4):
        o = oracle_mode(w, m)
        errs = family_errors(s.fields(m), o.fields())
        assert max(errs.values()) <= TOL64, (m, errs)
        wk, wo = s.wake(m)[0], o.wake()[0]
        assert rel(wk, wo) <= TOL64, m
        assert np.max(np.abs(wo)) > 0


def test_high_modes_subset(tetm):
    """A solve of modes 5..6 only (m_lo > 0)."""
    w = small_chain(30, 80, 5, 6, i0=6, steps=100)
    s = gpu_solver(tetm, w, 24)
    s.set_bunch(w.sigma, w.charge, w.i0)
    s.step(w.steps)
    for m in (5, 6):
        o = oracle_mode(w, m)
        assert max(family_errors(s.fields(m), o.fields()).values()) <= TOL64
        assert rel(s.wake(m)[0], o.wake()[0]) <= TOL64


@pytest.mark.parametrize("m", [0, 2])
def test_random_initial_state_matches_oracle(tetm, m):
    """Random fields in every component (set_fields zeroes what the mode and
    the geometry make inactive), no bunch, 60 steps."""
    w = small_chain(33, 50, m, m, steps=60)
    s = gpu_solver(tetm, w, 7)
    o = RzOracle(w.nr, w.nz, m, w.dr, w.dz, w.cdt, pec=w.pec)
    rng = np.random.default_rng(40 + m)
    for c in E_NAMES + H_NAMES:
        a = rng.standard_normal(o.shape)
        s.set(m, c, a)
        o.set(c, a)
        np.testing.assert_array_equal(s.get(m, c), o.get(c))
    s.step(60)
    o.step(60)
    errs = family_errors(s.fields(m), o.fields())
    assert max(errs.values()) <= TOL64, errs


def test_chunk_sizes_and_kernels_are_bitwise_identical(tetm):
    for prec in ("fp64", "fp32"):
        w = small_chain(70, 130, 0, 2, i0=5, steps=90, precision=prec)
        res = []
        for chunk, kernel in ((4, "async"), (13, "async"), (64, "async"), (13, "register"),
                              (64, "register"), (4, "bulk"), (13, "bulk"), (64, "bulk"),
                              (4, "bulk2"), (13, "bulk2"), (64, "bulk2")):
            s = gpu_solver(tetm, w, chunk, kernel)
            s.set_bunch(w.sigma, w.charge, w.i0)
            s.step(w.steps)
            res.append([s.get(2, c) for c in E_NAMES + H_NAMES] + [s.wake(1)[0]])
        for r in res[1:]:
            for a, b in zip(res[0], r):
                np.testing.assert_array_equal(a, b)


# ---------------------------------------------------------------------------
# Energy on the device
# ---------------------------------------------------------------------------

def test_energy_matches_oracle_and_is_conserved(tetm):
    w = small_chain(40, 60, 1, 1, steps=0)
    s = gpu_solver(tetm, w, 16)
    o = RzOracle(w.nr, w.nz, 1, w.dr, w.dz, w.cdt, pec=w.pec)
    rng = np.random.default_rng(77)
    for c in E_NAMES + H_NAMES:
        a = rng.standard_normal(o.shape)
        s.set(1, c, a)
        o.set(c, a)
    w0 = o.energy()
    assert s.energy(1) == pytest.approx(w0, rel=1e-12)
    s.step(200)
    o.step(200)
    assert s.energy(1) == pytest.approx(o.energy(), rel=1e-12)
    assert s.energy(1) == pytest.approx(w0, rel=1e-11)


# ---------------------------------------------------------------------------
# FP32 fields, FP64 wake sums
# ---------------------------------------------------------------------------

def test_fp32_wakes_against_oracle(tetm):
    """Nine-cell chain scaled to 64 x 400, ring at nr/64 as in the full
    workload. Modes 0..2 meet 1e-4 of their peak. For m >= 3 the wake is a
    small remainder of the bunch's own near field at the ring, which the e_z
    update cancels against the current every step; float32 storage of that
    field leaves a residue of up to a few 1e-4 of the (small) wake peak, so
    those modes are held to 1e-3 here and measured in the benchmark."""
    w = small_chain(64, 400, 0, 4, sigma_cells=8.0, precision="fp32")
    s = gpu_solver(tetm, w, 32)
    s.set_bunch(w.sigma, w.charge, w.i0)
    s.step(w.steps)
    for m in range(5):
        o = oracle_mode(w, m)
        assert rel(s.wake(m)[0], o.wake()[0]) <= (TOL32_WAKE if m <= 2 else 1e-3), m
        # the transverse wake at the ring meets 1e-4 for every mode
        assert rel(s.transverse_wake(m), o.transverse_wake()) <= TOL32_WAKE, m


# ---------------------------------------------------------------------------
# Full size: the 512 x 16384 nine-cell chain, modes 0..4, in the benchmark's
# launch configuration. Nothing ahead of plane n moves in n steps, so the
# oracle on the first n + 10 planes of the same geometry reproduces the head
# of the full grid entry by entry.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision,tol", [("fp32", 2e-5), ("fp64", TOL64)])
def test_full_size_chain_head_matches_oracle(tetm, precision, tol):
    from paper_0901_1053_gb300.autotune import tune_rz
    w = wl.cavity_chain_rz(precision=precision)
    n = 60
    kernel, chunk = tune_rz(w)
    s = gpu_solver(tetm, w, chunk, kernel)
    s.set_bunch(w.sigma, w.charge, w.i0)
    s.step(n)
    head = dataclasses.replace(w, nz=n + 10, pec=w.pec[:n + 10].copy(), steps=n)
    for m in range(w.m_lo, w.m_hi + 1):
        o = oracle_mode(head, m)
        g = s.fields(m)
        for c in E_NAMES + H_NAMES:
            assert not g[c][n + 2:].any(), (m, c)
        errs = family_errors({c: g[c][:n + 1] for c in g}, {c: o.get(c)[:n + 1] for c in g})
        assert max(errs.values()) <= tol, (m, errs)
        err = rel(s.wake(m)[0], o.wake()[0])
        print("wake error", precision, m, err)
        assert err <= (TOL32_WAKE if precision == "fp32" else 1e-12), (m, err)


# ---------------------------------------------------------------------------
# States and arguments
# ---------------------------------------------------------------------------

def test_state_and_argument_errors(tetm):
    w = small_chain(20, 40, 0, 2, steps=0)
    s = gpu_solver(tetm, w)
    with pytest.raises(tetm.TetmError) as e:
        s.set_bunch(w.sigma, w.charge, 0)          # the axis carries only m = 0
    assert e.value.code == tetm.TETM_E_ARG
    with pytest.raises(tetm.TetmError):
        s.wake(0)                                  # no bunch yet
    s.step(1)
    with pytest.raises(tetm.TetmError) as e:
        s.set_bunch(w.sigma, w.charge, 3)          # only at step 0
    assert e.value.code == tetm.TETM_E_STATE
    with pytest.raises(ValueError):
        s.energy(3)
    info = s.info()
    assert info["step"] == 1 and info["n_modes"] == 3 and info["wake_len"] == 0
    s2 = tetm.RzSolver(20, 40, 0, 0, 1e-3, 1.2e-3, 0.0, "fp64")   # c*dt = dr < dz
    with pytest.raises(tetm.TetmError) as e:
        s2.set_bunch(2e-3, 1e-9, 0)
    assert e.value.code == tetm.TETM_E_NOT_MAGIC


# ---------------------------------------------------------------------------
# Transverse (dipole) wake at r_{obs+1/2}
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("obs", [None, 9])
def test_transverse_wake_matches_oracle(tetm, kernel, obs):
    w = small_chain(40, 130, 0, 2, i0=4, steps=None)
    s = gpu_solver(tetm, w, 24, kernel)
    s.set_bunch(w.sigma, w.charge, w.i0)
    if obs is not None:
        s.set_observer(obs)
    s.step(w.steps)
    for m in range(3):
        o = RzOracle(w.nr, w.nz, m, w.dr, w.dz, w.cdt, pec=w.pec)
        o.set_bunch(w.sigma, w.charge, w.i0)
        if obs is not None:
            o.set_observer(obs)
        o.step(w.steps)
        wt = o.transverse_wake()
        if m == 0 and np.max(np.abs(wt)) == 0:
            continue
        assert rel(s.transverse_wake(m), wt) <= TOL64, m
        assert rel(s.wake(m)[0], o.wake()[0]) <= TOL64, m


def test_observer_state_errors(tetm):
    w = small_chain(20, 40, 0, 1, i0=3, steps=0)
    s = gpu_solver(tetm, w)
    with pytest.raises(tetm.TetmError) as e:
        s.set_observer(3)                          # no bunch yet
    assert e.value.code == tetm.TETM_E_STATE
    s.set_bunch(w.sigma, w.charge, w.i0)
    with pytest.raises(tetm.TetmError) as e:
        s.set_observer(19)                         # r_{obs+1/2} must lie inside the wall
    assert e.value.code == tetm.TETM_E_ARG
    s.set_observer(5)
    s.step(1)
    with pytest.raises(tetm.TetmError) as e:
        s.set_observer(6)
    assert e.value.code == tetm.TETM_E_STATE


# ---------------------------------------------------------------------------
# Static start: the ring bunch enters from an infinite pipe with its TEM field
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kernel", KERNELS)
def test_static_start_matches_oracle(tetm, kernel):
    w = small_chain(45, 160, 0, 3, i0=4)             # entry pipe uniform for k < 59
    K = 2 * math.ceil(5 * w.sigma / w.dz - 1e-12) + 2
    s = gpu_solver(tetm, w, 20, kernel)
    s.set_bunch_static(w.sigma, w.charge, w.i0, K)
    n = w.steps - K + 40
    s.step(n)
    for m in range(4):
        o = RzOracle(w.nr, w.nz, m, w.dr, w.dz, w.cdt, pec=w.pec)
        o.set_bunch_static(w.sigma, w.charge, w.i0, K)
        o.step(n)
        errs = family_errors(s.fields(m), o.fields())
        assert max(errs.values()) <= TOL64, (m, errs)
        assert rel(s.wake(m)[0], o.wake()[0]) <= TOL64, m
        assert rel(s.transverse_wake(m), o.transverse_wake()) <= TOL64, m


def test_static_start_smooth_pipe_moves_rigidly(tetm):
    nr, nz = 30, 150
    pec = wl.rz_radius_mask(nr, nz, lambda k: np.full(k.shape, 14.5))
    s = tetm.RzSolver(nr, nz, 0, 2, 0.25e-3, 0.25e-3, 0.0, "fp64", pec=pec)
    sigma = 3 * 0.25e-3
    K = 2 * 15 + 2
    s.set_bunch_static(sigma, 1e-9, 5, K)
    f0 = [s.fields(m) for m in range(3)]
    n = nz - K - 2
    s.step(n)
    for m in range(3):
        escale = max(np.max(np.abs(f0[m]["er"])), np.max(np.abs(f0[m]["ephi"])))
        hscale = max(np.max(np.abs(f0[m]["hphi"])), np.max(np.abs(f0[m]["hr"])))
        for c in E_NAMES + H_NAMES:
            shifted = np.zeros_like(f0[m][c])
            shifted[n:] = f0[m][c][:-n]
            tol = 1e-12 * (escale if c[0] == "e" else hscale)
            assert np.max(np.abs(s.get(m, c) - shifted)) <= tol, (m, c)
    cold = tetm.RzSolver(nr, nz, 0, 2, 0.25e-3, 0.25e-3, 0.0, "fp64", pec=pec)
    cold.set_bunch(sigma, 1e-9, 5)
    cold.step(n + K)
    for m in range(3):
        assert np.max(np.abs(s.wake(m)[0])) <= 1e-12 * np.max(np.abs(cold.wake(m)[0]))
        assert np.max(np.abs(s.transverse_wake(m))) <= 1e-12 * np.max(np.abs(cold.transverse_wake(m)))


def test_static_start_errors(tetm):
    w = small_chain(30, 120, 0, 1, i0=3, steps=0)
    s = gpu_solver(tetm, w)
    with pytest.raises(tetm.TetmError) as e:
        s.set_bunch_static(w.sigma, w.charge, 3, 100)        # past the entry pipe
    assert e.value.code == tetm.TETM_E_ARG
    with pytest.raises(tetm.TetmError) as e:
        s.set_bunch_static(w.sigma, w.charge, 0, 20)         # the axis with m = 1 solved
    assert e.value.code == tetm.TETM_E_ARG
    s.step(1)
    with pytest.raises(tetm.TetmError) as e:
        s.set_bunch_static(w.sigma, w.charge, 3, 20)
    assert e.value.code == tetm.TETM_E_STATE
