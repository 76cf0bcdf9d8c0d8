"""CPU-side checks of the C ABI: the library loads, exports every function
the headers in include/ declare, and its host-only paths (argument validation, the
stability bound of Eq. (25), sizes, error strings) answer without a GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    inc = os.path.join(ROOT, "include")
    txt = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc))
                  if f.endswith(".h"))
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tetm_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def tetm():
    from paper_0901_1053_gb300 import build as b
    if not os.path.exists(b.library_path()):
        b.build()
    from paper_0901_1053_gb300 import tetm as t
    return t


def test_library_exports_every_declared_function(tetm):
    declared = _header_functions()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(tetm.lib, name), name
    assert sorted(tetm.EXPORTS) == declared


def test_error_strings(tetm):
    assert tetm.tetm_strerror(0) == "ok"
    assert "Eq. (25)" in tetm.tetm_strerror(tetm.TETM_E_UNSTABLE)
    assert tetm.tetm_strerror(-1234) == "unknown error"


def test_create_rejects_bad_and_unstable_grids_before_touching_the_gpu(tetm):
    import ctypes
    h = ctypes.c_void_p(123)
    bad = tetm.make_grid(1, 8, 8, 1e-3, 1e-3, 1e-3)
    assert tetm.lib.tetm_create(ctypes.byref(bad), None, None, None, ctypes.byref(h)) == tetm.TETM_E_ARG
    assert not h.value
    cubic = tetm.make_grid(8, 8, 8, 1e-3, 1e-3, 1e-3, 0.0)   # dx=dy=dz, c*dt=dz: outside Eq. (25)
    assert tetm.lib.tetm_create(ctypes.byref(cubic), None, None, None, ctypes.byref(h)) == \
        tetm.TETM_E_UNSTABLE
    longstep = tetm.make_grid(8, 8, 8, 2e-3, 2e-3, 1e-3, 1.01e-3)  # c*dt > dz
    assert tetm.lib.tetm_create(ctypes.byref(longstep), None, None, None, ctypes.byref(h)) == \
        tetm.TETM_E_UNSTABLE


def test_bytes_needed(tetm):
    g32 = tetm.make_grid(256, 256, 2048, 1.414e-3, 1.414e-3, 1e-3, precision="fp32")
    g64 = tetm.make_grid(256, 256, 2048, 1.414e-3, 1.414e-3, 1e-3, precision="fp64")
    b32, b64 = tetm.tetm_bytes_needed(g32), tetm.tetm_bytes_needed(g64)
    cells = 256 * 256 * 2048
    assert 49 * cells < b32 < 60 * cells          # two field sets of six float32 + mask
    assert 97 * cells < b64 < 115 * cells
    assert tetm.tetm_bytes_needed(tetm.make_grid(0, 2, 2, 1, 1, 1)) == 0


def test_rz_create_rejects_bad_grids_and_materials_before_touching_the_gpu(tetm):
    import ctypes
    h = ctypes.c_void_p(123)
    bad = tetm.make_rz_grid(1, 8, 0, 0, 1e-3, 1e-3)
    assert tetm.lib.tetm_rz_create(ctypes.byref(bad), None, None, None, ctypes.byref(h)) == tetm.TETM_E_ARG
    assert not h.value
    modes = tetm.make_rz_grid(8, 8, 3, 2, 1e-3, 1e-3)
    assert tetm.lib.tetm_rz_create(ctypes.byref(modes), None, None, None, ctypes.byref(h)) == tetm.TETM_E_ARG
    too_long = tetm.make_rz_grid(8, 8, 0, 4, 0.9e-3, 1e-3, 1e-3)      # c*dt > dr (Sec. 4.4)
    assert tetm.lib.tetm_rz_create(ctypes.byref(too_long), None, None, None, ctypes.byref(h)) == \
        tetm.TETM_E_UNSTABLE
    import numpy as np
    ok = tetm.make_rz_grid(8, 8, 0, 0, 1e-3, 1e-3)
    for bad_value in (0.5, np.nan, np.inf):        # material arrays: physical and finite
        eps = np.ones(64)
        eps[17] = bad_value
        assert tetm.lib.tetm_rz_create(ctypes.byref(ok), ctypes.c_void_p(eps.ctypes.data), None, None,
                                       ctypes.byref(h)) == tetm.TETM_E_ARG
        assert tetm.lib.tetm_rz_create(ctypes.byref(ok), None, ctypes.c_void_p(eps.ctypes.data), None,
                                       ctypes.byref(h)) == tetm.TETM_E_ARG


def test_rz_bytes_needed(tetm):
    g32 = tetm.make_rz_grid(512, 16384, 0, 4, 1e-3, 1e-3, precision="fp32")
    g64 = tetm.make_rz_grid(512, 16384, 0, 4, 1e-3, 1e-3, precision="fp64")
    cells = 5 * 513 * 16385
    b32, b64 = tetm.tetm_rz_bytes_needed(g32), tetm.tetm_rz_bytes_needed(g64)
    assert 48 * cells < b32 < 57 * cells          # two sets of six float32 per mode + mask
    assert 96 * cells < b64 < 112 * cells         # row pitch padded to whole windows
    assert tetm.tetm_rz_bytes_needed(tetm.make_rz_grid(0, 8, 0, 0, 1e-3, 1e-3)) == 0


def test_every_handle_call_rejects_a_null_handle_without_a_gpu(tetm):
    """A NULL handle is an argument error (destroy calls are no-ops), answered
    before any device work, so it needs no GPU."""
    import ctypes
    L = tetm.lib
    E = tetm.TETM_E_ARG
    d = ctypes.c_double()
    i = ctypes.c_int32()
    calls = {
        "tetm_set_stream": lambda: L.tetm_set_stream(None, None),
        "tetm_set_kernel": lambda: L.tetm_set_kernel(None, 0),
        "tetm_set_tiling": lambda: L.tetm_set_tiling(None, 0, 0, 0),
        "tetm_set_scheme": lambda: L.tetm_set_scheme(None, 1),
        "tetm_check_guards": lambda: L.tetm_check_guards(None, None),
        "tetm_set_bunch": lambda: L.tetm_set_bunch(None, 1e-3, 1e-9, 1, 1),
        "tetm_set_bunch_static": lambda: L.tetm_set_bunch_static(None, 1e-3, 1e-9, 1, 1, 10),
        "tetm_step": lambda: L.tetm_step(None, 1),
        "tetm_sync": lambda: L.tetm_sync(None),
        "tetm_wake": lambda: L.tetm_wake(None, None, 0, None, None, None),
        "tetm_set_observer": lambda: L.tetm_set_observer(None, 1, 1),
        "tetm_transverse_wake": lambda: L.tetm_transverse_wake(None, None, None, 0, None, None, None),
        "tetm_energy": lambda: L.tetm_energy(None, ctypes.byref(d)),
        "tetm_charge_residual": lambda: L.tetm_charge_residual(None, None, None, None),
        "tetm_set_balance_every": lambda: L.tetm_set_balance_every(None, 1),
        "tetm_balance_history": lambda: L.tetm_balance_history(None, None, 0, None),
        "tetm_get_fields": lambda: L.tetm_get_fields(None, 0, None),
        "tetm_set_fields": lambda: L.tetm_set_fields(None, 0, None),
        "tetm_get_info": lambda: L.tetm_get_info(None, None),
        "tetm_save": lambda: L.tetm_save(None, None, 0, None),
        "tetm_load": lambda: L.tetm_load(None, None, 0),
        "tetm_batch_step": lambda: L.tetm_batch_step(None, 1),
        "tetm_batch_sync": lambda: L.tetm_batch_sync(None),
        "tetm_batch_info": lambda: L.tetm_batch_info(None, None, None, None),
        "tetm_rz_set_bunch": lambda: L.tetm_rz_set_bunch(None, 1e-3, 1e-9, 0),
        "tetm_rz_step": lambda: L.tetm_rz_step(None, 1),
        "tetm_rz_sync": lambda: L.tetm_rz_sync(None),
        "tetm_rz_wake": lambda: L.tetm_rz_wake(None, 0, None, 0, None, None, None),
        "tetm_rz_energy": lambda: L.tetm_rz_energy(None, 0, ctypes.byref(d)),
        "tetm_rz_get_fields": lambda: L.tetm_rz_get_fields(None, 0, 0, None),
        "tetm_rz_set_fields": lambda: L.tetm_rz_set_fields(None, 0, 0, None),
        "tetm_rz_set_tiling": lambda: L.tetm_rz_set_tiling(None, 16),
        "tetm_rz_set_kernel": lambda: L.tetm_rz_set_kernel(None, 0),
        "tetm_rz_set_stream": lambda: L.tetm_rz_set_stream(None, None),
        "tetm_rz_get_info": lambda: L.tetm_rz_get_info(None, None),
        "tetm_rz_set_observer": lambda: L.tetm_rz_set_observer(None, 1),
        "tetm_rz_transverse_wake": lambda: L.tetm_rz_transverse_wake(None, 0, None, 0, None, None, None),
        "tetm_rz_set_bunch_static": lambda: L.tetm_rz_set_bunch_static(None, 1e-3, 1e-9, 0, 10),
        "tetm_rz_set_bunch_scattered": lambda: L.tetm_rz_set_bunch_scattered(None, 1e-3, 1e-9, 0, 10),
        "tetm_rz_check_guards": lambda: L.tetm_rz_check_guards(None, None),
        "tetm_rz_charge_residual": lambda: L.tetm_rz_charge_residual(None, 0, None, None, None),
        "tetm_rz_set_balance_every": lambda: L.tetm_rz_set_balance_every(None, 1),
        "tetm_rz_balance_history": lambda: L.tetm_rz_balance_history(None, None, 0, None),
        "tetm_rz_save": lambda: L.tetm_rz_save(None, None, 0, None),
        "tetm_rz_load": lambda: L.tetm_rz_load(None, None, 0),
        "tetm_export_plane": lambda: L.tetm_export_plane(None, 0, None),
        "tetm_import_plane": lambda: L.tetm_import_plane(None, 0, None),
        "tetm_batch_add": lambda: L.tetm_batch_add(None, None, 0, None),
        "tetm_batch_remove": lambda: L.tetm_batch_remove(None, None),
        "tetm_batch_wait": lambda: L.tetm_batch_wait(None, 0, None),
    }
    for name, call in calls.items():
        assert call() == E, name
    L.tetm_destroy(None)
    L.tetm_batch_destroy(None)
    assert L.tetm_rz_destroy(None) == tetm.TETM_OK
    assert L.tetm_batch_create(None, None, 0, 0, None) == E
    assert L.tetm_batch_create_slots(4, tetm.TETM_FP32, 56, 28, 0, None) == E   # no output pointer
    out = ctypes.c_void_p()
    for args in ((0, tetm.TETM_FP32, 56, 28, 0), (4, 7, 56, 28, 0), (4, tetm.TETM_FP32, 30, 20, 0),
                 (4, tetm.TETM_FP64, 56, 28, 0), (4, tetm.TETM_FP32, 56, 28, -1)):
        assert L.tetm_batch_create_slots(*args, ctypes.byref(out)) == E, args   # rejected before any device call
    assert L.tetm_create_on_stream(None, None, None, None, None, None) == E
    assert L.tetm_create_slab(None, 0, 2, None, None, None, None) == E
    assert L.tetm_plane_bytes(None, 0) == 0
    handle_calls = [n for n in tetm.EXPORTS if n not in ("tetm_create", "tetm_rz_create", "tetm_destroy",
                    "tetm_create_slab", "tetm_plane_bytes", "tetm_create_on_stream", "tetm_pool_reserve",
                    "tetm_batch_create_slots",
                    "tetm_rz_destroy", "tetm_batch_destroy", "tetm_batch_create", "tetm_bytes_needed",
                    "tetm_rz_bytes_needed", "tetm_strerror", "tetm_energy_noalloc", "tetm_measure_fma_rate",
                    "tetm_rz_selftest_wait")]
    assert sorted(handle_calls) == sorted(calls), set(handle_calls) ^ set(calls)
