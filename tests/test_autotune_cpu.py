"""Host logic of the work-shape autotuner (no GPU): which shapes it offers for
each kind of solve, and its cache. The timing and the wave-fitted shapes need
a device, so they are replaced by stand-ins that record what they are asked."""
import types

import numpy as np

from paper_0901_1053_gb300 import autotune


def workload(nx=64, ny=48, nz=40):
    pec = np.zeros((nz, ny, nx), np.uint8)
    pec[:, :4, :] = 1
    return types.SimpleNamespace(nx=nx, ny=ny, nz=nz, pec=pec, precision="fp32")


class Recorder(autotune.Autotuner):
    """measure() and wave_fitted() without a device: each shape's time is its
    tile area over its chunk length (any fixed order will do), and every call
    is kept."""

    def __init__(self, path):
        super().__init__(cache_path=str(path))
        self.measured = []
        self.fitted_eps = []

    def measure(self, w, precision, shapes, eps_r=None):
        self.measured.append((precision, list(shapes), eps_r is not None))
        return {tuple(s): s[0] * s[1] / float(s[2]) for s in shapes}

    def wave_fitted(self, w, precision, tile_ys=(12, 20, 28), max_extra=6, eps_r=None):
        self.fitted_eps.append(eps_r is not None)
        out = [(28, 20, 24)]
        if precision == "fp32":
            out.append((56, 12, 21) if eps_r is not None else (56, 28, 45))
        return out


def test_material_solves_get_the_56x12_slab_tiles_and_no_56x28(tmp_path):
    t = Recorder(tmp_path / "cache.json")
    w = workload()
    eps = np.full((w.nz, w.ny, w.nx), 2.0)
    best = t.tune(w, "fp32", eps_r=eps)
    (prec, shapes, had_eps), = t.measured
    assert prec == "fp32" and had_eps and t.fitted_eps == [True]
    assert (56, 12, 21) in shapes and (56, 12, 32) in shapes
    assert all(s[0] == 28 or (s[0], s[1]) == (56, 12) for s in shapes)
    assert best in [tuple(s) for s in shapes]


def test_one_material_solves_never_get_56x12(tmp_path):
    t = Recorder(tmp_path / "cache.json")
    t.tune(workload(), "fp32")
    (_, shapes, had_eps), = t.measured
    assert not had_eps
    assert (56, 28, 45) in shapes and (56, 28, 32) in shapes
    assert not any((s[0], s[1]) == (56, 12) for s in shapes)


def test_batches_run_the_56x28_slab_or_the_warp_sweep(tmp_path):
    t = Recorder(tmp_path / "cache.json")
    t.tune(workload(), "fp32", batch=True)
    (_, shapes, _), = t.measured
    assert shapes and all(s[0] == 28 or (s[0], s[1]) == (56, 28) for s in shapes)


def test_float64_candidates_are_warp_tiled(tmp_path):
    t = Recorder(tmp_path / "cache.json")
    t.tune(workload(), "fp64")
    (_, shapes, _), = t.measured
    assert not any(s[0] == 56 for s in shapes)


def test_cache_keys_separate_materials_and_are_reused(tmp_path):
    path = tmp_path / "cache.json"
    t = Recorder(path)
    w = workload()
    eps_a = np.full((w.nz, w.ny, w.nx), 2.0)
    eps_b = np.full((w.nz, w.ny, w.nx), 3.0)
    plain = t.tune(w, "fp32")
    ma = t.tune(w, "fp32", eps_r=eps_a)
    mb = t.tune(w, "fp32", eps_r=eps_b)
    assert len(t.measured) == 3          # three keys: one material, and each eps array
    assert (plain[0], plain[1]) != (56, 12) and (ma[0], ma[1]) != (56, 28)
    # a second tuner on the same file answers from the cache without measuring
    u = Recorder(path)
    assert u.tune(w, "fp32") == plain
    assert u.tune(w, "fp32", eps_r=eps_a) == ma
    assert u.tune(w, "fp32", eps_r=eps_b) == mb
    assert u.measured == []
