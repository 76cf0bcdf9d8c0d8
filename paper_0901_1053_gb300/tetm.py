"""Thin ctypes binding of libtetm.so (include/tetm.h, include/tetm_rz.h), same
names as the C ABI.

Argument marshalling only: every step of the solve runs in the library's
CUDA kernels. Importing this module loads the in-tree library and raises
ImportError if it has not been built (``python -m paper_0901_1053_gb300.build``
or ``__graft_entry__.build()``); there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import library_path

TETM_OK = 0
TETM_E_ARG = -1
TETM_E_UNSTABLE = -2
TETM_E_NOT_MAGIC = -3
TETM_E_NOMEM = -4
TETM_E_CUDA = -5
TETM_E_STATE = -6
TETM_E_TIMEOUT = -7
TETM_E_DIVERGED = -8
TETM_E_UNSUPPORTED = -9
TETM_E_TOO_LARGE = -10
TETM_NOALLOC_MAX_ENTRIES = 33554432

TETM_FP64 = 0
TETM_FP32 = 1
TETM_KERNEL_FUSED = 0
TETM_KERNEL_REFERENCE = 1
TETM_KERNEL_TWOSTEP = 2
TETM_SCHEME_TETM = 0
TETM_SCHEME_YEE = 1
COMPONENTS = ("ex", "ey", "ez", "hx", "hy", "hz")

# Every function the header declares (checked by the CPU test suite).
EXPORTS = ("tetm_create", "tetm_set_bunch", "tetm_step", "tetm_sync", "tetm_wake",
           "tetm_destroy", "tetm_energy", "tetm_charge_residual", "tetm_get_fields",
           "tetm_set_fields", "tetm_set_stream", "tetm_set_kernel", "tetm_set_tiling", "tetm_set_scheme",
           "tetm_check_guards",
           "tetm_set_observer", "tetm_transverse_wake",
           "tetm_get_info", "tetm_bytes_needed", "tetm_save", "tetm_load", "tetm_strerror",
           "tetm_set_balance_every", "tetm_balance_history", "tetm_energy_noalloc",
           "tetm_batch_create", "tetm_batch_step", "tetm_batch_sync", "tetm_batch_info",
           "tetm_batch_destroy", "tetm_set_bunch_static", "tetm_measure_fma_rate",
           "tetm_rz_create", "tetm_rz_set_bunch", "tetm_rz_step", "tetm_rz_sync", "tetm_rz_wake",
           "tetm_rz_energy", "tetm_rz_get_fields", "tetm_rz_set_fields", "tetm_rz_set_tiling",
           "tetm_rz_set_stream", "tetm_rz_get_info", "tetm_rz_bytes_needed", "tetm_rz_destroy",
           "tetm_rz_set_kernel", "tetm_rz_set_observer", "tetm_rz_transverse_wake",
           "tetm_rz_set_bunch_static", "tetm_rz_set_bunch_scattered", "tetm_rz_selftest_wait",
           "tetm_rz_check_guards", "tetm_rz_charge_residual", "tetm_rz_set_balance_every",
           "tetm_rz_balance_history", "tetm_rz_save", "tetm_rz_load",
           "tetm_create_slab", "tetm_plane_bytes", "tetm_export_plane", "tetm_import_plane",
           "tetm_create_on_stream", "tetm_pool_reserve", "tetm_batch_create_slots", "tetm_batch_add",
           "tetm_batch_remove", "tetm_batch_wait")
TETM_PLANES_UP = 0
TETM_PLANES_DOWN = 1
TETM_RZ_KERNEL_ASYNC = 0
TETM_RZ_KERNEL_REGISTER = 1
TETM_RZ_KERNEL_BULK = 2
TETM_RZ_KERNEL_BULK2 = 3
RZ_COMPONENTS = ("er", "ephi", "ez", "hr", "hphi", "hz")
TETM_RZ_MAX_MODES = 64


class tetm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dz", ctypes.c_double), ("cdt", ctypes.c_double)]


class tetm_info(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("active_cells", ctypes.c_int64), ("processed_cells", ctypes.c_int64),
                ("kernel", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32), ("chunk_z", ctypes.c_int32),
                ("work_items", ctypes.c_int32), ("wake_len", ctypes.c_int32),
                ("uniform_material", ctypes.c_int32)]


class tetm_rz_grid(ctypes.Structure):
    _fields_ = [("nr", ctypes.c_int32), ("nz", ctypes.c_int32), ("m_lo", ctypes.c_int32),
                ("m_hi", ctypes.c_int32), ("precision", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("dr", ctypes.c_double), ("dz", ctypes.c_double), ("cdt", ctypes.c_double)]


class tetm_rz_info(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("processed_cells", ctypes.c_int64), ("n_modes", ctypes.c_int32),
                ("chunk_z", ctypes.c_int32), ("work_items", ctypes.c_int32),
                ("wake_len", ctypes.c_int32), ("resident_warps", ctypes.c_int32),
                ("kernel", ctypes.c_int32)]


def _load():
    path = library_path()
    if not os.path.exists(path):
        raise ImportError("libtetm.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    vp, i32, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "tetm_create": (ctypes.c_int, [ctypes.POINTER(tetm_grid), vp, vp, vp, pp]),
        "tetm_set_bunch": (ctypes.c_int, [vp, dbl, dbl, i32, i32]),
        "tetm_set_bunch_static": (ctypes.c_int, [vp, dbl, dbl, i32, i32, i32]),
        "tetm_measure_fma_rate": (ctypes.c_int, [i32, ctypes.POINTER(dbl), vp]),
        "tetm_step": (ctypes.c_int, [vp, i32]),
        "tetm_sync": (ctypes.c_int, [vp]),
        "tetm_wake": (ctypes.c_int, [vp, vp, i32, ctypes.POINTER(i32), ctypes.POINTER(dbl),
                                     ctypes.POINTER(dbl)]),
        "tetm_set_observer": (ctypes.c_int, [vp, i32, i32]),
        "tetm_transverse_wake": (ctypes.c_int, [vp, vp, vp, i32, vp, vp, vp]),
        "tetm_destroy": (None, [vp]),
        "tetm_energy": (ctypes.c_int, [vp, ctypes.POINTER(dbl)]),
        "tetm_charge_residual": (ctypes.c_int, [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                                ctypes.POINTER(dbl)]),
        "tetm_get_fields": (ctypes.c_int, [vp, i32, vp]),
        "tetm_set_fields": (ctypes.c_int, [vp, i32, vp]),
        "tetm_set_stream": (ctypes.c_int, [vp, vp]),
        "tetm_set_kernel": (ctypes.c_int, [vp, i32]),
        "tetm_set_tiling": (ctypes.c_int, [vp, i32, i32, i32]),
        "tetm_set_scheme": (ctypes.c_int, [vp, i32]),
        "tetm_check_guards": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "tetm_rz_check_guards": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int64)]),
        "tetm_get_info": (ctypes.c_int, [vp, ctypes.POINTER(tetm_info)]),
        "tetm_bytes_needed": (ctypes.c_int64, [ctypes.POINTER(tetm_grid)]),
        "tetm_save": (ctypes.c_int, [vp, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
        "tetm_load": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
        "tetm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "tetm_set_balance_every": (ctypes.c_int, [vp, i32]),
        "tetm_balance_history": (ctypes.c_int, [vp, vp, i32, ctypes.POINTER(i32)]),
        "tetm_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), vp, i32, i32,
                                             ctypes.POINTER(ctypes.c_void_p)]),
        "tetm_batch_step": (ctypes.c_int, [vp, i32]),
        "tetm_batch_sync": (ctypes.c_int, [vp]),
        "tetm_batch_info": (ctypes.c_int, [vp, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                           ctypes.POINTER(i32)]),
        "tetm_batch_destroy": (None, [vp]),
        "tetm_create_on_stream": (ctypes.c_int, [ctypes.POINTER(tetm_grid), vp, vp, vp, vp, pp]),
        "tetm_pool_reserve": (ctypes.c_int, [ctypes.c_uint64]),
        "tetm_batch_create_slots": (ctypes.c_int, [i32, i32, i32, i32, i32, ctypes.POINTER(ctypes.c_void_p)]),
        "tetm_batch_add": (ctypes.c_int, [vp, vp, ctypes.c_int64, ctypes.POINTER(i32)]),
        "tetm_batch_remove": (ctypes.c_int, [vp, vp]),
        "tetm_batch_wait": (ctypes.c_int, [vp, i32, ctypes.POINTER(dbl)]),
        "tetm_energy_noalloc": (ctypes.c_int, [ctypes.POINTER(tetm_grid),
                                               ctypes.POINTER(ctypes.c_void_p), vp, vp, vp]),
        "tetm_rz_create": (ctypes.c_int, [ctypes.POINTER(tetm_rz_grid), vp, vp, vp, pp]),
        "tetm_rz_set_bunch": (ctypes.c_int, [vp, dbl, dbl, i32]),
        "tetm_rz_step": (ctypes.c_int, [vp, ctypes.c_int64]),
        "tetm_rz_sync": (ctypes.c_int, [vp]),
        "tetm_rz_wake": (ctypes.c_int, [vp, i32, vp, i32, ctypes.POINTER(i32),
                                        ctypes.POINTER(dbl), ctypes.POINTER(dbl)]),
        "tetm_rz_energy": (ctypes.c_int, [vp, i32, ctypes.POINTER(dbl)]),
        "tetm_rz_get_fields": (ctypes.c_int, [vp, i32, i32, vp]),
        "tetm_rz_set_fields": (ctypes.c_int, [vp, i32, i32, vp]),
        "tetm_rz_set_tiling": (ctypes.c_int, [vp, i32]),
        "tetm_rz_set_stream": (ctypes.c_int, [vp, vp]),
        "tetm_rz_set_kernel": (ctypes.c_int, [vp, i32]),
        "tetm_rz_set_observer": (ctypes.c_int, [vp, i32]),
        "tetm_rz_set_bunch_static": (ctypes.c_int, [vp, dbl, dbl, i32, i32]),
        "tetm_rz_set_bunch_scattered": (ctypes.c_int, [vp, dbl, dbl, i32, i32]),
        "tetm_rz_selftest_wait": (ctypes.c_int, [i32]),
        "tetm_rz_transverse_wake": (ctypes.c_int, [vp, i32, vp, i32, ctypes.POINTER(i32),
                                                   ctypes.POINTER(dbl), ctypes.POINTER(dbl)]),
        "tetm_rz_get_info": (ctypes.c_int, [vp, ctypes.POINTER(tetm_rz_info)]),
        "tetm_rz_bytes_needed": (ctypes.c_int64, [ctypes.POINTER(tetm_rz_grid)]),
        "tetm_rz_destroy": (ctypes.c_int, [vp]),
        "tetm_rz_charge_residual": (ctypes.c_int, [vp, i32, ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                                   ctypes.POINTER(dbl)]),
        "tetm_rz_set_balance_every": (ctypes.c_int, [vp, i32]),
        "tetm_rz_balance_history": (ctypes.c_int, [vp, vp, i32, ctypes.POINTER(i32)]),
        "tetm_rz_save": (ctypes.c_int, [vp, vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
        "tetm_rz_load": (ctypes.c_int, [vp, vp, ctypes.c_size_t]),
        "tetm_create_slab": (ctypes.c_int, [ctypes.POINTER(tetm_grid), i32, i32, vp, vp, vp, pp]),
        "tetm_plane_bytes": (ctypes.c_int64, [vp, i32]),
        "tetm_export_plane": (ctypes.c_int, [vp, i32, vp]),
        "tetm_import_plane": (ctypes.c_int, [vp, i32, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


class TetmError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, lib.tetm_strerror(code).decode(), code))


def _check(rc, where):
    if rc != TETM_OK:
        raise TetmError(rc, where)
    return rc


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _buf_ptr(b):
    """Address of a numpy array or of a tensor (host or device)."""
    return ctypes.c_void_p(b.data_ptr() if hasattr(b, "data_ptr") else b.ctypes.data)


def make_grid(nx, ny, nz, dx, dy, dz, cdt=0.0, precision="fp32"):
    p = {"fp64": TETM_FP64, "fp32": TETM_FP32}[precision] if isinstance(precision, str) else precision
    return tetm_grid(int(nx), int(ny), int(nz), int(p), float(dx), float(dy), float(dz), float(cdt))


def tetm_measure_fma_rate(precision="fp64", stream=0):
    """Measured FMA rate of the device in TFLOP/s (see include/tetm.h)."""
    p = {"fp64": TETM_FP64, "fp32": TETM_FP32}[precision] if isinstance(precision, str) else precision
    out = ctypes.c_double()
    _check(lib.tetm_measure_fma_rate(int(p), ctypes.byref(out), ctypes.c_void_p(int(stream) if stream else 0)),
           "tetm_measure_fma_rate")
    return out.value


def tetm_bytes_needed(grid):
    return int(lib.tetm_bytes_needed(ctypes.byref(grid)))


def tetm_pool_reserve(nbytes):
    """Released device memory the library's pool keeps for reuse."""
    _check(lib.tetm_pool_reserve(int(nbytes)), "tetm_pool_reserve")


def tetm_energy_noalloc(grid, field_ptrs, mask_ptr, w_ptr, stream=0):
    """Energy of a state held in caller-owned device arrays, without any
    device allocation (see include/tetm.h). All pointers are device
    addresses (ints); returns the TETM_* code."""
    arr = (ctypes.c_void_p * 6)(*[ctypes.c_void_p(int(p)) for p in field_ptrs])
    return int(lib.tetm_energy_noalloc(ctypes.byref(grid), arr,
                                       ctypes.c_void_p(int(mask_ptr) if mask_ptr else 0),
                                       ctypes.c_void_p(int(w_ptr)), ctypes.c_void_p(int(stream or 0))))


def tetm_strerror(code):
    return lib.tetm_strerror(int(code)).decode()


class Solver:
    """One solve; a thin object around a ``tetm_solver*`` handle.

    ``eps_r``/``mu_r``: float64 per cell (nz, ny, nx) or None; ``pec``: uint8
    per cell or None. Fields are exchanged in the canonical FIT layout
    (nz+1, ny+1, nx+1) as float64.
    """

    def __init__(self, nx, ny, nz, dx, dy, dz, cdt=0.0, precision="fp32", eps_r=None, mu_r=None,
                 pec=None, k_range=None, stream=None):
        """k_range=(k_lo, k_hi): the z-slab of planes [k_lo, k_hi) of this grid
        (tetm_create_slab); the cell arrays still cover the whole grid.
        stream: a cudaStream_t (int) that the solve's work, its creation
        included, is queued on (tetm_create_on_stream); None = the default
        stream."""
        self.grid = make_grid(nx, ny, nz, dx, dy, dz, cdt, precision)
        cell = (int(nz), int(ny), int(nx))
        arrs = []
        for a, dt in ((eps_r, np.float64), (mu_r, np.float64), (pec, np.uint8)):
            arrs.append(None if a is None else np.ascontiguousarray(a, dtype=dt).reshape(cell))
        h = ctypes.c_void_p()
        self.h = None
        if stream is not None:
            if k_range is not None:
                raise ValueError("a z-slab is created on the default stream")
            _check(lib.tetm_create_on_stream(ctypes.byref(self.grid), *[_ptr(a) for a in arrs],
                                             ctypes.c_void_p(int(stream)), ctypes.byref(h)),
                   "tetm_create_on_stream")
            nzl = int(nz)
        elif k_range is None:
            _check(lib.tetm_create(ctypes.byref(self.grid), *[_ptr(a) for a in arrs], ctypes.byref(h)),
                   "tetm_create")
            nzl = int(nz)
        else:
            k_lo, k_hi = int(k_range[0]), int(k_range[1])
            _check(lib.tetm_create_slab(ctypes.byref(self.grid), k_lo, k_hi, *[_ptr(a) for a in arrs],
                                        ctypes.byref(h)), "tetm_create_slab")
            nzl = k_hi - k_lo
        self.h = h
        self.k_range = None if k_range is None else (int(k_range[0]), int(k_range[1]))
        self.shape = (nzl + 1, int(ny) + 1, int(nx) + 1)

    @classmethod
    def from_workload(cls, w, precision=None):
        s = cls(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, precision or w.precision, pec=w.pec)
        s.set_bunch(w.sigma, w.charge, w.i0, w.j0)
        return s

    def close(self):
        if self.h is not None:
            lib.tetm_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_bunch(self, sigma, charge, i0, j0):
        _check(lib.tetm_set_bunch(self.h, float(sigma), float(charge), int(i0), int(j0)),
               "tetm_set_bunch")

    def set_bunch_static(self, sigma, charge, i0, j0, k_head):
        _check(lib.tetm_set_bunch_static(self.h, float(sigma), float(charge), int(i0), int(j0),
                                         int(k_head)), "tetm_set_bunch_static")

    def step(self, n=1):
        _check(lib.tetm_step(self.h, int(n)), "tetm_step")

    def sync(self):
        _check(lib.tetm_sync(self.h), "tetm_sync")

    def wake(self):
        n = ctypes.c_int32()
        s0, ds = ctypes.c_double(), ctypes.c_double()
        _check(lib.tetm_wake(self.h, None, 0, ctypes.byref(n), ctypes.byref(s0), ctypes.byref(ds)),
               "tetm_wake")
        out = np.empty(n.value, dtype=np.float64)
        _check(lib.tetm_wake(self.h, _ptr(out), n.value, None, None, None), "tetm_wake")
        return out, s0.value, ds.value

    def set_observer(self, i, j):
        """Observer line of the transverse wake (before the first step)."""
        _check(lib.tetm_set_observer(self.h, int(i), int(j)), "tetm_set_observer")

    def transverse_wake(self):
        """(W_x on the x-edge line (i+1/2, j), W_y on the y-edge line (i, j+1/2)) [V/C]."""
        n = ctypes.c_int32()
        _check(lib.tetm_transverse_wake(self.h, None, None, 0, ctypes.byref(n), None, None),
               "tetm_transverse_wake")
        wx = np.empty(n.value, dtype=np.float64)
        wy = np.empty(n.value, dtype=np.float64)
        _check(lib.tetm_transverse_wake(self.h, _ptr(wx), _ptr(wy), n.value, None, None, None),
               "tetm_transverse_wake")
        return wx, wy

    def energy(self):
        w = ctypes.c_double()
        _check(lib.tetm_energy(self.h, ctypes.byref(w)), "tetm_energy")
        return w.value

    def charge_residual(self):
        e, h, q = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib.tetm_charge_residual(self.h, ctypes.byref(e), ctypes.byref(h), ctypes.byref(q)),
               "tetm_charge_residual")
        return e.value, h.value, q.value

    def set_balance_every(self, every):
        _check(lib.tetm_set_balance_every(self.h, int(every)), "tetm_set_balance_every")

    def balance_history(self):
        """Array (n, 5): step, energy, max_e, max_h, q_scale per record."""
        n = ctypes.c_int32()
        _check(lib.tetm_balance_history(self.h, None, 0, ctypes.byref(n)), "tetm_balance_history")
        out = np.zeros((n.value, 5), dtype=np.float64)
        if n.value:
            _check(lib.tetm_balance_history(self.h, _ptr(out), n.value, ctypes.byref(n)),
                   "tetm_balance_history")
        return out

    def get(self, comp):
        out = np.empty(self.shape, dtype=np.float64)
        _check(lib.tetm_get_fields(self.h, _comp(comp), _ptr(out)), "tetm_get_fields")
        return out

    def set(self, comp, arr):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.shape)
        _check(lib.tetm_set_fields(self.h, _comp(comp), _ptr(a)), "tetm_set_fields")

    def fields(self):
        return {c: self.get(c) for c in COMPONENTS}

    def set_stream(self, stream):
        """stream: an int/pointer cudaStream_t (e.g. torch's ``stream.cuda_stream``) or None."""
        _check(lib.tetm_set_stream(self.h, ctypes.c_void_p(stream or 0)), "tetm_set_stream")

    def set_kernel(self, kernel):
        k = {"fused": TETM_KERNEL_FUSED, "reference": TETM_KERNEL_REFERENCE,
             "twostep": TETM_KERNEL_TWOSTEP}.get(kernel, kernel)
        _check(lib.tetm_set_kernel(self.h, int(k)), "tetm_set_kernel")

    def set_tiling(self, tile_x=0, tile_y=0, chunk_z=0):
        _check(lib.tetm_set_tiling(self.h, int(tile_x), int(tile_y), int(chunk_z)), "tetm_set_tiling")

    def set_scheme(self, scheme):
        """'tetm' (Eq. (23), the default) or 'yee' (Yee's E/M leapfrog, Eq. (7),
        field-only: e is read as e^{n-1/2}, h as h^n), before the first step."""
        k = {"tetm": TETM_SCHEME_TETM, "yee": TETM_SCHEME_YEE}.get(scheme, scheme)
        _check(lib.tetm_set_scheme(self.h, int(k)), "tetm_set_scheme")

    def check_guards(self):
        """Entries that hold a value although they carry no field (0 in a correct run)."""
        v = ctypes.c_int64()
        _check(lib.tetm_check_guards(self.h, ctypes.byref(v)), "tetm_check_guards")
        return int(v.value)

    def info(self):
        i = tetm_info()
        _check(lib.tetm_get_info(self.h, ctypes.byref(i)), "tetm_get_info")
        return {f: getattr(i, f) for f, _ in tetm_info._fields_}

    def save(self):
        used = ctypes.c_size_t()
        _check(lib.tetm_save(self.h, None, 0, ctypes.byref(used)), "tetm_save")
        buf = np.empty(used.value, dtype=np.uint8)
        _check(lib.tetm_save(self.h, _ptr(buf), used.value, ctypes.byref(used)), "tetm_save")
        return buf

    def load(self, buf):
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(lib.tetm_load(self.h, _ptr(b), b.size), "tetm_load")

    # --- z-slabs: ghost-plane messages (host numpy arrays or device tensors) ---
    def plane_bytes(self, direction):
        return int(lib.tetm_plane_bytes(self.h, int(direction)))

    def export_plane(self, direction, buf):
        """Queue the message for `direction` (TETM_PLANES_UP / _DOWN) into buf:
        a numpy array or a tensor with a data_ptr() of plane_bytes bytes."""
        _check(lib.tetm_export_plane(self.h, int(direction), _buf_ptr(buf)), "tetm_export_plane")

    def import_plane(self, direction, buf):
        _check(lib.tetm_import_plane(self.h, int(direction), _buf_ptr(buf)), "tetm_import_plane")


def _comp(c):
    return COMPONENTS.index(c) if isinstance(c, str) else int(c)


class Batch:
    """Solves advancing together (tetm_batch_*): one launch per step for all
    members, optionally replayed from a captured CUDA graph."""

    def __init__(self, solvers, step_limits=None, graph_steps=0):
        if solvers is None:   # an empty slot table (Batch.slots)
            self.h = None
            self.solvers = []
            return
        self.solvers = list(solvers)
        n = len(self.solvers)
        hs = (ctypes.c_void_p * n)(*[s.h for s in self.solvers])
        lim = None
        if step_limits is not None:
            self._lim = np.ascontiguousarray([int(x) for x in step_limits], dtype=np.int64)
            lim = _ptr(self._lim)
        h = ctypes.c_void_p()
        self.h = None
        _check(lib.tetm_batch_create(hs, lim, n, int(graph_steps), ctypes.byref(h)),
               "tetm_batch_create")
        self.h = h

    @classmethod
    def slots(cls, capacity, precision="fp32", tile=(56, 28), graph_steps=0):
        """An empty batch of `capacity` slots (tetm_batch_create_slots):
        members join (add) and leave (remove) between steps without
        rebuilding the batch or re-capturing its graph."""
        b = cls(None)
        p = {"fp64": TETM_FP64, "fp32": TETM_FP32}[precision]
        h = ctypes.c_void_p()
        _check(lib.tetm_batch_create_slots(int(capacity), p, int(tile[0]), int(tile[1]), int(graph_steps),
                                           ctypes.byref(h)), "tetm_batch_create_slots")
        b.h = h
        return b

    def add(self, solver, step_limit=-1):
        """Join: the solve takes a free slot; returns the slot index."""
        slot = ctypes.c_int32(-1)
        _check(lib.tetm_batch_add(self.h, solver.h, int(step_limit), ctypes.byref(slot)), "tetm_batch_add")
        self.solvers.append(solver)
        return slot.value

    def remove(self, solver):
        """Leave after the steps queued so far (no host wait)."""
        _check(lib.tetm_batch_remove(self.h, solver.h), "tetm_batch_remove")
        self.solvers = [s for s in self.solvers if s is not solver]

    def step(self, n):
        _check(lib.tetm_batch_step(self.h, int(n)), "tetm_batch_step")

    def wait(self, max_pending=0):
        """Blocks until at most max_pending step calls are unfinished on the
        device; returns the device seconds of the finished calls so far."""
        busy = ctypes.c_double(0.0)
        _check(lib.tetm_batch_wait(self.h, int(max_pending), ctypes.byref(busy)), "tetm_batch_wait")
        return busy.value

    def sync(self):
        _check(lib.tetm_batch_sync(self.h), "tetm_batch_sync")

    def info(self):
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib.tetm_batch_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "tetm_batch_info")
        return {"members": a.value, "active": b.value, "work_items": c.value}

    def close(self):
        if self.h is not None:
            lib.tetm_batch_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---------------------------------------------------------------------------
# Rotationally symmetric solver (include/tetm_rz.h)
# ---------------------------------------------------------------------------

def make_rz_grid(nr, nz, m_lo, m_hi, dr, dz, cdt=0.0, precision="fp32"):
    p = {"fp64": TETM_FP64, "fp32": TETM_FP32}[precision] if isinstance(precision, str) else precision
    return tetm_rz_grid(int(nr), int(nz), int(m_lo), int(m_hi), int(p), 0, float(dr), float(dz),
                        float(cdt))


def tetm_rz_bytes_needed(grid):
    return int(lib.tetm_rz_bytes_needed(ctypes.byref(grid)))


class RzSolver:
    """Modes m_lo..m_hi of the scheme (24) on one (r, z) grid; fields in the
    canonical (nz+1, nr+1) layout, r fastest, per radian."""

    def __init__(self, nr, nz, m_lo, m_hi, dr, dz, cdt=0.0, precision="fp32", pec=None, eps_r=None,
                 mu_r=None):
        """eps_r, mu_r: float64 per cell (nz, nr) or None (vacuum); pec: uint8
        per cell or None."""
        self.grid = make_rz_grid(nr, nz, m_lo, m_hi, dr, dz, cdt, precision)
        self.nr, self.nz = int(nr), int(nz)
        self.m_lo, self.m_hi = int(m_lo), int(m_hi)
        self.shape = (self.nz + 1, self.nr + 1)
        self.precision = precision
        cell = (self.nz, self.nr)
        arrs = []
        for a, dt in ((eps_r, np.float64), (mu_r, np.float64), (pec, np.uint8)):
            arrs.append(None if a is None else np.ascontiguousarray(a, dtype=dt).reshape(cell))
        h = ctypes.c_void_p()
        self.h = ctypes.c_void_p()
        _check(lib.tetm_rz_create(ctypes.byref(self.grid), *[_ptr(a) for a in arrs], ctypes.byref(h)),
               "tetm_rz_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib.tetm_rz_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _mode(self, m):
        if not self.m_lo <= m <= self.m_hi:
            raise ValueError("mode %d outside %d..%d" % (m, self.m_lo, self.m_hi))
        return m - self.m_lo

    def set_bunch(self, sigma, charge, i0):
        _check(lib.tetm_rz_set_bunch(self.h, float(sigma), float(charge), int(i0)),
               "tetm_rz_set_bunch")

    def step(self, n=1):
        _check(lib.tetm_rz_step(self.h, int(n)), "tetm_rz_step")

    def sync(self):
        _check(lib.tetm_rz_sync(self.h), "tetm_rz_sync")

    def set_tiling(self, chunk_z):
        _check(lib.tetm_rz_set_tiling(self.h, int(chunk_z)), "tetm_rz_set_tiling")

    def set_kernel(self, kernel):
        k = {"async": TETM_RZ_KERNEL_ASYNC, "register": TETM_RZ_KERNEL_REGISTER,
             "bulk": TETM_RZ_KERNEL_BULK, "bulk2": TETM_RZ_KERNEL_BULK2}[kernel] \
            if isinstance(kernel, str) else int(kernel)
        _check(lib.tetm_rz_set_kernel(self.h, k), "tetm_rz_set_kernel")

    def set_stream(self, stream):
        _check(lib.tetm_rz_set_stream(self.h, ctypes.c_void_p(int(stream) if stream else 0)),
               "tetm_rz_set_stream")

    def check_guards(self):
        """Entries that hold a value although they carry no field (0 in a correct run)."""
        v = ctypes.c_int64()
        _check(lib.tetm_rz_check_guards(self.h, ctypes.byref(v)), "tetm_rz_check_guards")
        return int(v.value)

    def info(self):
        inf = tetm_rz_info()
        _check(lib.tetm_rz_get_info(self.h, ctypes.byref(inf)), "tetm_rz_get_info")
        return {f[0]: getattr(inf, f[0]) for f in tetm_rz_info._fields_}

    def wake(self, m):
        n = ctypes.c_int32()
        s0 = ctypes.c_double()
        ds = ctypes.c_double()
        mi = self._mode(m)
        _check(lib.tetm_rz_wake(self.h, mi, None, 0, ctypes.byref(n), ctypes.byref(s0),
                                ctypes.byref(ds)), "tetm_rz_wake")
        out = np.empty(n.value, dtype=np.float64)
        _check(lib.tetm_rz_wake(self.h, mi, _ptr(out), n.value, None, None, None), "tetm_rz_wake")
        return out, s0.value, ds.value

    def set_observer(self, obs):
        _check(lib.tetm_rz_set_observer(self.h, int(obs)), "tetm_rz_set_observer")

    def set_bunch_static(self, sigma, charge, i0, k_head):
        _check(lib.tetm_rz_set_bunch_static(self.h, float(sigma), float(charge), int(i0), int(k_head)),
               "tetm_rz_set_bunch_static")

    def set_bunch_scattered(self, sigma, charge, i0, k_head):
        """The static start kept as scattered field: the stored field is the
        total minus the moving TEM field of the entry section."""
        _check(lib.tetm_rz_set_bunch_scattered(self.h, float(sigma), float(charge), int(i0),
                                               int(k_head)), "tetm_rz_set_bunch_scattered")

    def transverse_wake(self, m):
        n = ctypes.c_int32()
        mi = self._mode(m)
        _check(lib.tetm_rz_transverse_wake(self.h, mi, None, 0, ctypes.byref(n), None, None),
               "tetm_rz_transverse_wake")
        out = np.empty(n.value, dtype=np.float64)
        _check(lib.tetm_rz_transverse_wake(self.h, mi, _ptr(out), n.value, None, None, None),
               "tetm_rz_transverse_wake")
        return out

    def energy(self, m):
        w = ctypes.c_double()
        _check(lib.tetm_rz_energy(self.h, self._mode(m), ctypes.byref(w)), "tetm_rz_energy")
        return w.value

    def charge_residual(self, m):
        """(max |qe - qbunch|, max |qh|, bunch charge scale) of mode m."""
        e, h, q = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(lib.tetm_rz_charge_residual(self.h, self._mode(m), ctypes.byref(e), ctypes.byref(h),
                                           ctypes.byref(q)), "tetm_rz_charge_residual")
        return e.value, h.value, q.value

    def set_balance_every(self, every):
        _check(lib.tetm_rz_set_balance_every(self.h, int(every)), "tetm_rz_set_balance_every")

    def balance_history(self):
        """Array (rows, 6): step, m, energy, max_e, max_h, q_scale per mode and record."""
        n = ctypes.c_int32()
        _check(lib.tetm_rz_balance_history(self.h, None, 0, ctypes.byref(n)), "tetm_rz_balance_history")
        out = np.zeros((n.value, 6), dtype=np.float64)
        if n.value:
            _check(lib.tetm_rz_balance_history(self.h, _ptr(out), n.value, ctypes.byref(n)),
                   "tetm_rz_balance_history")
        return out

    def save(self):
        used = ctypes.c_size_t()
        _check(lib.tetm_rz_save(self.h, None, 0, ctypes.byref(used)), "tetm_rz_save")
        buf = (ctypes.c_char * used.value)()
        _check(lib.tetm_rz_save(self.h, buf, used.value, ctypes.byref(used)), "tetm_rz_save")
        return bytes(buf)

    def load(self, data):
        buf = ctypes.create_string_buffer(data, len(data))
        _check(lib.tetm_rz_load(self.h, buf, len(data)), "tetm_rz_load")

    def get(self, m, comp):
        c = RZ_COMPONENTS.index(comp) if isinstance(comp, str) else int(comp)
        out = np.empty(self.shape, dtype=np.float64)
        _check(lib.tetm_rz_get_fields(self.h, self._mode(m), c, _ptr(out)), "tetm_rz_get_fields")
        return out

    def set(self, m, comp, arr):
        c = RZ_COMPONENTS.index(comp) if isinstance(comp, str) else int(comp)
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.shape)
        _check(lib.tetm_rz_set_fields(self.h, self._mode(m), c, _ptr(a)), "tetm_rz_set_fields")

    def fields(self, m):
        return {c: self.get(m, c) for c in RZ_COMPONENTS}

    def wave_fitted_chunk(self, lo=24, hi=256):
        """Planes per work item whose item count fills whole waves of the
        resident warps best (ties go to the longer chunk); leaves that tiling
        set."""
        best = None
        for c in range(lo, hi + 1, 4):
            self.set_tiling(c)
            inf = self.info()
            n, slots = inf["work_items"], max(1, inf["resident_warps"])
            if n == 0:
                continue
            eff = n / (slots * -(-n // slots))
            if best is None or eff >= best[0] - 1e-9:
                best = (eff, c)
        c = best[1] if best else 32
        self.set_tiling(c)
        return c


def rz_selftest_wait(polls):
    """Bounded-wait self-test (tetm_rz_selftest_wait): returns the status code,
    TETM_E_TIMEOUT when the wait gave up as designed."""
    return int(lib.tetm_rz_selftest_wait(int(polls)))
