"""Running a list of independent solves as one batch (tetm_batch_*)."""
from __future__ import annotations

import time
from typing import List, Optional, Tuple


def run_batch(workloads, precision: str = "fp32", tiling: Optional[Tuple[int, int, int]] = None,
              graph_steps: int = 32, round_steps: Optional[int] = None, stats: Optional[dict] = None):
    """Create every solve, advance them together until each reached its own
    step count, and return (wakes, seconds of stepping, seconds total).
    stats (a dict), if given, receives the active cell-steps (cells that
    carry a field, times each solve's steps)."""
    from . import tetm
    t_start = time.perf_counter()
    solvers = []
    for w in workloads:
        s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, precision, pec=w.pec)
        s.set_bunch(w.sigma, w.charge, w.i0, w.j0)
        if tiling:
            s.set_tiling(*tiling)
        solvers.append(s)
    limits = [w.steps for w in workloads]
    if stats is not None:
        stats["active_cell_steps"] = sum(s.info()["active_cells"] * n for s, n in zip(solvers, limits))
    b = tetm.Batch(solvers, limits, graph_steps=graph_steps)
    b.sync()
    t0 = time.perf_counter()
    b.step(max(limits))
    b.sync()
    t1 = time.perf_counter()
    wakes = [s.wake()[0] for s in solvers]
    b.close()
    for s in solvers:
        s.close()
    return wakes, t1 - t0, time.perf_counter() - t_start


def run_sequential(workloads, precision: str = "fp64", tiling=None, kernel: str = "fused"):
    """Each solve alone, one after the other (the single-solve path)."""
    from . import tetm
    wakes = []
    t0 = time.perf_counter()
    for w in workloads:
        s = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, precision, pec=w.pec)
        s.set_bunch(w.sigma, w.charge, w.i0, w.j0)
        s.set_kernel(kernel)
        if tiling and kernel == "fused":
            s.set_tiling(*tiling)
        s.step(w.steps)
        wakes.append(s.wake()[0])
        s.close()
    return wakes, time.perf_counter() - t0
