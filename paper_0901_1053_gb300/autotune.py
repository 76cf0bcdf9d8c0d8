"""Work-shape autotuner for the fused step kernels.

For a grid and geometry it times candidate (tile_x, tile_y, chunk_z) shapes
on a scratch solve with the same geometry (the cost of a step does not depend
on the bunch or on the field values), keeps the fastest and caches it in a
JSON file keyed by GPU name, precision, grid size and a digest of the PEC
mask. Tuning runs solves through the C ABI only; nothing here computes fields.
"""
from __future__ import annotations

import hashlib
import json
import os
import time
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

Shape = Tuple[int, int, int]

CANDIDATES_FP32: List[Shape] = [(56, 28, 32), (56, 28, 16), (56, 28, 64), (56, 12, 32), (56, 12, 16),
                                (28, 20, 32), (28, 20, 16), (28, 12, 32), (28, 12, 16),
                                (28, 28, 32), (28, 8, 32), (28, 4, 32), (32, 8, 64)]
CANDIDATES_FP64: List[Shape] = [(28, 20, 32), (28, 20, 16), (28, 12, 32), (28, 28, 32),
                                (28, 4, 32), (32, 8, 64)]


def default_cache_path() -> str:
    return os.environ.get("TETM_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "tetm", "autotune.json"))


def _gpu_name() -> str:
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.get_device_name(0)
    except Exception:
        pass
    return "unknown-gpu"


def geometry_digest(pec) -> str:
    if pec is None:
        return "box"
    return hashlib.sha1(memoryview(pec).tobytes()).hexdigest()[:16]


class Autotuner:
    def __init__(self, cache_path: Optional[str] = None, steps: int = 20, warmup: int = 3, repeats: int = 2):
        self.path = cache_path or default_cache_path()
        self.steps = steps
        self.warmup = warmup
        self.repeats = repeats
        self.cache: Dict[str, list] = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.cache = json.load(f)
            except (OSError, ValueError):
                self.cache = {}

    def key(self, w, precision: str) -> str:
        return "|".join([_gpu_name(), precision, "%dx%dx%d" % (w.nx, w.ny, w.nz),
                         geometry_digest(w.pec)])

    def _save(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            tmp = self.path + ".tmp%d" % os.getpid()
            with open(tmp, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        except OSError:
            pass

    def measure(self, w, precision: str, shapes: Sequence[Shape], eps_r=None) -> Dict[Shape, float]:
        """Seconds per step of each shape on a scratch solve of w's geometry
        (and material array eps_r, which selects the coefficient-array kernels)."""
        from . import tetm
        s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, precision, eps_r=eps_r, pec=w.pec)
        out = {}
        try:
            for shape in shapes:
                try:
                    s.set_tiling(*shape)
                except tetm.TetmError:
                    continue
                s.step(self.warmup)
                s.sync()
                best = None
                for _ in range(self.repeats):  # the fastest of a few runs: less noise from the host
                    t0 = time.perf_counter()
                    s.step(self.steps)
                    s.sync()
                    dt = (time.perf_counter() - t0) / self.steps
                    best = dt if best is None else min(best, dt)
                out[tuple(shape)] = best
        finally:
            s.close()
        return out

    def wave_fitted(self, w, precision: str, tile_ys=(12, 20, 28), max_extra: int = 6, eps_r=None):
        """Shapes (28, ty, cz) whose work-item count fills whole waves of the
        resident warps (16 per SM): for each tile height, the chunk lengths
        around the one that gives one or two full waves; in float32 also slab
        shapes whose items split evenly over its CTAs (4 to 8 items each):
        (56, 28, cz), one CTA per SM, or with the material array eps_r
        (56, 12, cz), two CTAs per SM."""
        from . import tetm
        try:
            import torch
            sms = torch.cuda.get_device_properties(0).multi_processor_count
        except Exception:
            sms = 152
        slots = 16 * sms
        s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, precision, eps_r=eps_r, pec=w.pec)
        out = []
        try:
            for ty in tile_ys:
                s.set_tiling(28, ty, 32)
                items32 = s.info()["work_items"]
                for waves in (1, 2):
                    cz = max(4, int(round(32 * items32 / (waves * slots))))
                    best = None
                    for c in range(max(4, cz - max_extra), cz + max_extra + 1):
                        s.set_tiling(28, ty, c)
                        n = s.info()["work_items"]
                        eff = n / (slots * -(-n // slots))
                        if best is None or eff > best[0] + 1e-9:
                            best = (eff, c)
                    out.append((28, ty, best[1]))
            if precision == "fp32":
                ty, ctas = (28, sms) if eps_r is None else (12, 2 * sms)
                s.set_tiling(56, ty, 32)
                items32 = s.info()["work_items"]
                for rounds in range(4, 9):
                    cz = max(4, int(round(32 * items32 / (rounds * ctas))))
                    best = None
                    for c in range(max(4, cz - 4), cz + 5):
                        s.set_tiling(56, ty, c)
                        n = s.info()["work_items"]
                        eff = n / (ctas * -(-n // ctas))
                        if best is None or eff > best[0] + 1e-9:
                            best = (eff, c)
                    out.append((56, ty, best[1]))
        finally:
            s.close()
        return sorted(set(out))

    def tune(self, w, precision: Optional[str] = None,
             candidates: Optional[Sequence[Shape]] = None, materials: bool = False, eps_r=None,
             batch: bool = False) -> Shape:
        """materials: the solve has eps/mu arrays (per-entry coefficients run on
        the warp-tiled kernel, tile_x = 28, and the float32 slab kernel, 56 x 12);
        batch: the shape is for a batch of solves (batched launches run the
        warp-tiled kernel, tile_x = 28, and in float32 the slab kernel)."""
        precision = precision or w.precision
        materials = materials or eps_r is not None
        k = self.key(w, precision) + ("|materials56x12" if materials else "") + ("|batch" if batch else "")
        if eps_r is not None:
            k += "|" + hashlib.sha1(memoryview(np.ascontiguousarray(eps_r)).tobytes()).hexdigest()[:16]
        if k in self.cache:
            return tuple(self.cache[k])
        cands = list(candidates or (CANDIDATES_FP32 if precision == "fp32" else CANDIDATES_FP64))
        if candidates is None:
            cands += [c for c in self.wave_fitted(w, precision, eps_r=eps_r) if c not in cands]
        if materials:
            cands = [c for c in cands if c[0] == 28 or (c[0], c[1]) == (56, 12)]
        else:
            cands = [c for c in cands if (c[0], c[1]) != (56, 12)]
        if batch:
            cands = [c for c in cands if c[0] == 28 or (precision == "fp32" and (c[0], c[1]) == (56, 28))]
        times = self.measure(w, precision, cands, eps_r=eps_r)
        best = min(times, key=times.get)
        self.cache[k] = list(best)
        self._save()
        return best


# ---------------------------------------------------------------------------
# Rotationally symmetric solver: step kernel and planes per work item
# ---------------------------------------------------------------------------

def tune_rz(w, precision: Optional[str] = None, steps: int = 8, warmup: int = 3,
            extra_chunks: Sequence[int] = (16, 24, 32, 64, 128)):
    """(kernel, chunk_z) with the shortest step on a scratch solve of w's
    geometry: each step kernel with its wave-fitted chunk and a few fixed
    ones (the two-steps-per-pass kernel timed over pairs of steps). Returns
    ("bulk2" | "bulk" | "register" | "async", chunk_z)."""
    from . import tetm
    precision = precision or w.precision
    s = tetm.RzSolver(w.nr, w.nz, w.m_lo, w.m_hi, w.dr, w.dz, w.cdt, precision, pec=w.pec)
    best = None
    try:
        for kern in ("bulk2", "bulk", "register", "async"):
            s.set_kernel(kern)
            chunks = [s.wave_fitted_chunk()] + [c for c in extra_chunks]
            for c in dict.fromkeys(chunks):
                s.set_tiling(c)
                s.step(2 * warmup)
                s.sync()
                t0 = time.perf_counter()
                s.step(2 * steps)
                s.sync()
                dt = (time.perf_counter() - t0) / (2 * steps)
                if best is None or dt < best[0]:
                    best = (dt, kern, c)
    finally:
        s.close()
    return best[1], best[2]
