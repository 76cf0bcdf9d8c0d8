"""FP64 CPU oracle of the explicit TE/TM scheme: the 3D scheme (Sec. 4.2,
Eq. (23)) and the rotationally symmetric one (Sec. 4.3, Eq. (24)).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code
with the CUDA path (``paper_0901_1053_gb300``) and never imports it.

The arithmetic lives in ``tetm_oracle.c`` (plain loops, one function per
paper passage); this module only loads it with ctypes, marshals numpy arrays
and offers the canonical FIT layout helpers.

Component numbering: 0 ex, 1 ey, 2 ez, 3 hx, 4 hy, 5 hz. Every field array
has the canonical FIT shape ``(nz+1, ny+1, nx+1)`` (x fastest), float64, in
integral units (edge voltages [V], dual-edge currents [A]).

Parity status: every function here is pinned by the ``-m "not gpu"`` tests
(dense matrix form of Eq. (23), eigen-angles of Eq. (27), energy law (19),
charge laws (34)/(35), exact z-shift at c*dt = dz, loss-factor identity).
``Oracle.yee_step`` (Yee's scheme, Eq. (7), the paper's comparison scheme) is
pinned by the eigen-angles of the dispersion relation (9), the step bound (8),
the exactly conserved leapfrog energy and the z-dispersion (10) of a TEM pulse
on a coaxial line. ``RzOracle`` (tetm_rz_oracle.c) is pinned by its own tests: the dense form
(24), stability at c*dt = min(dr, dz) for every mode, energy law (19),
pillbox Bessel-zero frequencies, the coaxial TEM shift, Gauss's law and the
loss-factor identity.
"""
from __future__ import annotations

import ctypes
import os
import numpy as np

from .build import build_oracle, library_path

COMPONENTS = ("ex", "ey", "ez", "hx", "hy", "hz")
C_LIGHT = 299792458.0
EPS0 = 8.8541878128e-12
MU0 = 1.0 / (EPS0 * C_LIGHT * C_LIGHT)

_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        build_oracle()
    lib = ctypes.CDLL(path)
    d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    lib.oracle_new.restype = vp
    lib.oracle_new.argtypes = [i, i, i, d, d, d, d, vp, vp, vp]
    lib.oracle_free.argtypes = [vp]
    lib.oracle_stable.restype = i
    lib.oracle_stable.argtypes = [d, d, d, d]
    lib.oracle_set_bunch.restype = i
    lib.oracle_set_bunch.argtypes = [vp, d, d, i, i]
    lib.oracle_current.argtypes = [vp, ctypes.c_long, vp]
    lib.oracle_step_j.argtypes = [vp, vp, vp, vp]
    lib.oracle_step.argtypes = [vp, i]
    lib.oracle_step_custom.argtypes = [vp, vp, vp, vp]
    lib.oracle_yee_step.restype = i
    lib.oracle_yee_step.argtypes = [vp, i]
    lib.oracle_yee_stable.restype = i
    lib.oracle_yee_stable.argtypes = [d, d, d, d]
    lib.oracle_wake.restype = i
    lib.oracle_wake.argtypes = [vp, vp, i, ctypes.POINTER(i), dp, dp]
    lib.oracle_set_observer.restype = i
    lib.oracle_set_observer.argtypes = [vp, i, i]
    lib.oracle_wake_extra.restype = i
    lib.oracle_wake_extra.argtypes = [vp, i, vp, i]
    lib.oracle_energy.restype = d
    lib.oracle_energy.argtypes = [vp]
    lib.oracle_qbar_e.argtypes = [vp] + [vp] * 6
    lib.oracle_qbar_h.argtypes = [vp] + [vp] * 6
    lib.oracle_get.argtypes = [vp, i, vp]
    lib.oracle_set.argtypes = [vp, i, vp]
    lib.oracle_coef.argtypes = [vp, i, vp]
    lib.oracle_step_count.restype = ctypes.c_long
    lib.oracle_step_count.argtypes = [vp]
    lib.oracle_dt.restype = d
    lib.oracle_dt.argtypes = [vp]
    lib.oracle_set_bunch_static.restype = i
    lib.oracle_set_bunch_static.argtypes = [vp, d, d, i, i, i]
    lib.oracle_kshift.restype = ctypes.c_long
    lib.oracle_kshift.argtypes = [vp]
    lib.oracle_bunch_info.restype = i
    lib.oracle_bunch_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i),
                                      ctypes.POINTER(i), vp]
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def stable(dx, dy, dz, cdt):
    """Eq. (25): c*dt <= dz and c*dt <= (dx^-2 + dy^-2)^-1/2."""
    return bool(_load().oracle_stable(dx, dy, dz, cdt))


def yee_stable(dx, dy, dz, cdt):
    """Eq. (8), the step bound of Yee's scheme: c*dt <= (dx^-2 + dy^-2 + dz^-2)^-1/2."""
    return bool(_load().oracle_yee_stable(dx, dy, dz, cdt))


class Oracle:
    """One FP64 solve on a closed PEC box (Sec. 2, Eq. (1)), cold start.

    ``eps_r``, ``mu_r``: float64 per primary cell, shape (nz, ny, nx) or None
    (vacuum); ``pec``: uint8 per cell, 1 = PEC, or None. ``cdt`` = c*dt in
    metres, 0 means dz (the "magic" step of Sec. 4.5).
    """

    def __init__(self, nx, ny, nz, dx, dy, dz, cdt=0.0, eps_r=None, mu_r=None, pec=None):
        self.lib = _load()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dx, self.dy, self.dz = float(dx), float(dy), float(dz)
        shape_c = (self.nz, self.ny, self.nx)
        self._keep = []
        args = []
        for a, dt in ((eps_r, np.float64), (mu_r, np.float64), (pec, np.uint8)):
            if a is None:
                args.append(None)
            else:
                a = np.ascontiguousarray(a, dtype=dt).reshape(shape_c)
                self._keep.append(a)
                args.append(_ptr(a))
        h = self.lib.oracle_new(self.nx, self.ny, self.nz, self.dx, self.dy, self.dz,
                                float(cdt), *args)
        if not h:
            raise ValueError("oracle_new: invalid grid")
        self.h = ctypes.c_void_p(h)
        self.shape = (self.nz + 1, self.ny + 1, self.nx + 1)
        self.dt = self.lib.oracle_dt(self.h)
        self.alpha = 0.5 * self.dt

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and self.lib is not None:
            self.lib.oracle_free(h)
            self.h = None

    # --- fields -----------------------------------------------------------
    def get(self, comp):
        out = np.empty(self.shape, dtype=np.float64)
        self.lib.oracle_get(self.h, _comp(comp), _ptr(out))
        return out

    def set(self, comp, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.shape)
        self.lib.oracle_set(self.h, _comp(comp), _ptr(a))

    def coef(self, comp):
        out = np.empty(self.shape, dtype=np.float64)
        self.lib.oracle_coef(self.h, _comp(comp), _ptr(out))
        return out

    def fields(self):
        return {c: self.get(c) for c in COMPONENTS}

    # --- bunch, stepping, wake ---------------------------------------------
    def set_bunch(self, sigma, charge, i0, j0):
        if self.lib.oracle_set_bunch(self.h, float(sigma), float(charge), int(i0), int(j0)) != 0:
            raise ValueError("oracle_set_bunch: bad argument")

    def set_bunch_static(self, sigma, charge, i0, j0, k_head):
        """Bunch with its head at plane k_head at step 0, carrying its discrete
        TEM field (static start in a uniform vacuum entry section)."""
        if self.lib.oracle_set_bunch_static(self.h, float(sigma), float(charge), int(i0), int(j0),
                                            int(k_head)) != 0:
            raise ValueError("oracle_set_bunch_static: bad argument or non-uniform entry section")

    @property
    def kshift(self):
        return int(self.lib.oracle_kshift(self.h))

    def current(self, n):
        out = np.zeros(self.shape, dtype=np.float64)
        self.lib.oracle_current(self.h, int(n), _ptr(out))
        return out

    def step(self, n=1):
        self.lib.oracle_step(self.h, int(n))

    def step_custom(self, jz=None, jx=None, jy=None):
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape)
                for a in (jz, jx, jy)]
        self.lib.oracle_step_custom(self.h, *[_ptr(a) for a in arrs])

    def yee_step(self, n=1):
        """n steps of Yee's E/M leapfrog, Eq. (7), on this grid: state
        (e^{n-1/2}, h^n), source-free."""
        if self.lib.oracle_yee_step(self.h, int(n)) != 0:
            raise ValueError("oracle_yee_step: a solve with a bunch")

    @property
    def step_count(self):
        return int(self.lib.oracle_step_count(self.h))

    def wake(self):
        n = ctypes.c_int()
        s0 = ctypes.c_double()
        ds = ctypes.c_double()
        if self.lib.oracle_wake(self.h, None, 0, ctypes.byref(n), ctypes.byref(s0),
                                ctypes.byref(ds)) != 0:
            raise RuntimeError("no bunch set")
        out = np.empty(n.value, dtype=np.float64)
        self.lib.oracle_wake(self.h, _ptr(out), n.value, None, None, None)
        return out, s0.value, ds.value

    def set_observer(self, i, j):
        """Observer line of the transverse wake (before the first step)."""
        if self.lib.oracle_set_observer(self.h, int(i), int(j)) != 0:
            raise ValueError("oracle_set_observer: bad argument or state")

    def _extra(self, which):
        n = len(self.wake()[0])
        out = np.empty(n, dtype=np.float64)
        if self.lib.oracle_wake_extra(self.h, int(which), _ptr(out), n) != 0:
            raise RuntimeError("no bunch set")
        return out

    def transverse_wake(self):
        """(W_x on the x-edge line (i+1/2, j), W_y on the y-edge line (i, j+1/2)),
        (1/Q) sum (E_x - c mu0 H_y) dz and (1/Q) sum (E_y + c mu0 H_x) dz."""
        return self._extra(0), self._extra(1)

    def wake_at_observer(self):
        """Longitudinal wakes on the node lines (i, j), (i+1, j), (i, j+1)."""
        return self._extra(2), self._extra(3), self._extra(4)

    def bunch_info(self):
        c0, mn, mx = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        if self.lib.oracle_bunch_info(self.h, ctypes.byref(c0), ctypes.byref(mn),
                                      ctypes.byref(mx), None) != 0:
            raise RuntimeError("no bunch set")
        qcell = np.empty(2 * c0.value, dtype=np.float64)
        self.lib.oracle_bunch_info(self.h, ctypes.byref(c0), ctypes.byref(mn), ctypes.byref(mx),
                                   _ptr(qcell))
        return {"c0": c0.value, "m_min": mn.value, "m_max": mx.value, "qcell": qcell}

    # --- invariants -----------------------------------------------------------
    def energy(self):
        return float(self.lib.oracle_energy(self.h))

    def qbar_e(self, ex1, ex0, ey1, ey0, ez):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape)
                for a in (ex1, ex0, ey1, ey0, ez)]
        q = np.empty(self.shape, dtype=np.float64)
        self.lib.oracle_qbar_e(self.h, *[_ptr(a) for a in arrs], _ptr(q))
        return q

    def qbar_h(self, hx1, hx0, hy1, hy0, hz):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape)
                for a in (hx1, hx0, hy1, hy0, hz)]
        q = np.empty(self.shape, dtype=np.float64)
        self.lib.oracle_qbar_h(self.h, *[_ptr(a) for a in arrs], _ptr(q))
        return q


def _comp(c):
    if isinstance(c, str):
        return COMPONENTS.index(c)
    return int(c)


# ---------------------------------------------------------------------------
# Rotationally symmetric scheme (Sec. 4.3, Eq. (24)), one azimuthal mode
# ---------------------------------------------------------------------------

RZ_COMPONENTS = ("er", "ephi", "ez", "hr", "hphi", "hz")


def _load_rz():
    lib = _load()
    if getattr(lib, "_rz_ready", False):
        return lib
    d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    lib.rz_oracle_new.restype = vp
    lib.rz_oracle_new.argtypes = [i, i, i, d, d, d, vp, vp, vp]
    lib.rz_oracle_free.argtypes = [vp]
    lib.rz_oracle_stable.restype = i
    lib.rz_oracle_stable.argtypes = [d, d, d]
    lib.rz_oracle_set_bunch.restype = i
    lib.rz_oracle_set_bunch.argtypes = [vp, d, d, i]
    lib.rz_oracle_current.argtypes = [vp, ctypes.c_long, vp]
    lib.rz_oracle_step.argtypes = [vp, i]
    lib.rz_oracle_step_custom.argtypes = [vp, vp]
    lib.rz_oracle_wake.restype = i
    lib.rz_oracle_wake.argtypes = [vp, vp, i, ctypes.POINTER(i), dp, dp]
    lib.rz_oracle_set_bunch_static.restype = i
    lib.rz_oracle_set_bunch_static.argtypes = [vp, d, d, i, i]
    lib.rz_oracle_set_observer.restype = i
    lib.rz_oracle_set_observer.argtypes = [vp, i]
    lib.rz_oracle_wake_extra.restype = i
    lib.rz_oracle_wake_extra.argtypes = [vp, i, vp, i]
    lib.rz_oracle_energy.restype = d
    lib.rz_oracle_energy.argtypes = [vp]
    lib.rz_oracle_qbar_e.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.rz_oracle_qbar_h.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    lib.rz_oracle_get.argtypes = [vp, i, vp]
    lib.rz_oracle_set.argtypes = [vp, i, vp]
    lib.rz_oracle_coef.argtypes = [vp, i, vp]
    lib.rz_oracle_dt.restype = d
    lib.rz_oracle_dt.argtypes = [vp]
    lib.rz_oracle_step_count.restype = ctypes.c_long
    lib.rz_oracle_step_count.argtypes = [vp]
    lib._rz_ready = True
    return lib


def rz_stable(dr, dz, cdt):
    """Sec. 4.4: c*dt <= min(dr, dz), for every azimuthal mode."""
    return bool(_load_rz().rz_oracle_stable(dr, dz, cdt))


class RzOracle:
    """One FP64 solve of azimuthal mode ``m`` on an (r, z) grid of nr x nz
    cells, axis at r = 0, PEC at r = nr*dr and at both z ends, cold start.

    Field arrays have the canonical shape (nz+1, nr+1), r fastest, per-radian
    integral units. ``eps_r``, ``mu_r`` per cell (nz, nr) or None; ``pec``
    uint8 per cell or None. ``cdt`` = c*dt, 0 means min(dr, dz)."""

    def __init__(self, nr, nz, m, dr, dz, cdt=0.0, eps_r=None, mu_r=None, pec=None):
        self.lib = _load_rz()
        self.nr, self.nz, self.m = int(nr), int(nz), int(m)
        self.dr, self.dz = float(dr), float(dz)
        shape_c = (self.nz, self.nr)
        self._keep = []
        args = []
        for a, dt in ((eps_r, np.float64), (mu_r, np.float64), (pec, np.uint8)):
            if a is None:
                args.append(None)
            else:
                a = np.ascontiguousarray(a, dtype=dt).reshape(shape_c)
                self._keep.append(a)
                args.append(_ptr(a))
        h = self.lib.rz_oracle_new(self.nr, self.nz, self.m, self.dr, self.dz, float(cdt), *args)
        if not h:
            raise ValueError("rz_oracle_new: invalid grid")
        self.h = ctypes.c_void_p(h)
        self.shape = (self.nz + 1, self.nr + 1)
        self.dt = self.lib.rz_oracle_dt(self.h)
        self.alpha = 0.5 * self.dt

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and self.lib is not None:
            self.lib.rz_oracle_free(h)
            self.h = None

    def get(self, comp):
        out = np.empty(self.shape, dtype=np.float64)
        self.lib.rz_oracle_get(self.h, _rz_comp(comp), _ptr(out))
        return out

    def set(self, comp, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.shape)
        self.lib.rz_oracle_set(self.h, _rz_comp(comp), _ptr(a))

    def coef(self, comp):
        out = np.empty(self.shape, dtype=np.float64)
        self.lib.rz_oracle_coef(self.h, _rz_comp(comp), _ptr(out))
        return out

    def fields(self):
        return {c: self.get(c) for c in RZ_COMPONENTS}

    def set_bunch(self, sigma, charge, i0=0):
        if self.lib.rz_oracle_set_bunch(self.h, float(sigma), float(charge), int(i0)) != 0:
            raise ValueError("rz_oracle_set_bunch: bad argument")

    def set_bunch_static(self, sigma, charge, i0, k_head):
        """Bunch with its head at plane k_head at step 0 carrying its discrete
        TEM field (static start in a uniform vacuum entry section)."""
        if self.lib.rz_oracle_set_bunch_static(self.h, float(sigma), float(charge), int(i0),
                                               int(k_head)) != 0:
            raise ValueError("rz_oracle_set_bunch_static: bad argument or non-uniform entry section")

    def current(self, n):
        out = np.zeros(self.shape, dtype=np.float64)
        self.lib.rz_oracle_current(self.h, int(n), _ptr(out))
        return out

    def step(self, n=1):
        self.lib.rz_oracle_step(self.h, int(n))

    def step_custom(self, jz=None):
        a = None if jz is None else np.ascontiguousarray(jz, dtype=np.float64).reshape(self.shape)
        self.lib.rz_oracle_step_custom(self.h, _ptr(a))

    @property
    def step_count(self):
        return int(self.lib.rz_oracle_step_count(self.h))

    def wake(self):
        n = ctypes.c_int()
        s0 = ctypes.c_double()
        ds = ctypes.c_double()
        if self.lib.rz_oracle_wake(self.h, None, 0, ctypes.byref(n), ctypes.byref(s0),
                                   ctypes.byref(ds)) != 0:
            raise RuntimeError("no bunch set")
        out = np.empty(n.value, dtype=np.float64)
        self.lib.rz_oracle_wake(self.h, _ptr(out), n.value, None, None, None)
        return out, s0.value, ds.value

    def energy(self):
        return float(self.lib.rz_oracle_energy(self.h))

    def qbar_e(self, er1, er0, ephi1, ephi0, ez):
        """Node charge of the mode (per radian) in the form of Eq. (35) for
        scheme (24): e_r, e_phi at n+1 and n, e_z at n+1/2."""
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape)
                for a in (er1, er0, ephi1, ephi0, ez)]
        q = np.empty(self.shape, dtype=np.float64)
        self.lib.rz_oracle_qbar_e(self.h, *[_ptr(a) for a in arrs], _ptr(q))
        return q

    def qbar_h(self, hphi1, hphi0, hr1, hr0, hz):
        """Cell charge of the mode (per radian, by lower node) in the form of
        Eq. (34): h_phi, h_r at n+1/2 and n-1/2, h_z at n."""
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape)
                for a in (hphi1, hphi0, hr1, hr0, hz)]
        q = np.empty(self.shape, dtype=np.float64)
        self.lib.rz_oracle_qbar_h(self.h, *[_ptr(a) for a in arrs], _ptr(q))
        return q

    def set_observer(self, obs):
        """Transverse wake at r_{obs+1/2} (before the first step)."""
        if self.lib.rz_oracle_set_observer(self.h, int(obs)) != 0:
            raise ValueError("rz_oracle_set_observer: bad argument or state")

    def _extra(self, which):
        n = len(self.wake()[0])
        out = np.empty(n, dtype=np.float64)
        if self.lib.rz_oracle_wake_extra(self.h, int(which), _ptr(out), n) != 0:
            raise RuntimeError("no bunch set")
        return out

    def transverse_wake(self):
        """Radial transverse wake (1/Q) sum (E_r - c mu0 H_phi) dz at r_{obs+1/2}, phi = 0."""
        return self._extra(0)

    def wake_at_observer(self):
        """Longitudinal wakes at rings obs and obs+1."""
        return self._extra(1), self._extra(2)


def _rz_comp(c):
    if isinstance(c, str):
        return RZ_COMPONENTS.index(c)
    return int(c)
