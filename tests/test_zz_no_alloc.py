"""The no-allocation energy entry point, for callers that may not allocate
device memory (their device buffers come from an arena or a host framework,
or they run in a loop where cudaMalloc is not allowed): it must give the same
discrete energy as tetm_energy, call after call, while the caller passes
every input and output buffer itself.

Kept in a file of its own that sorts last, so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_0901_1053_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tetm():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0901_1053_gb300 import tetm as t
    return t


def _active_mask(tetm, w):
    """Activity bits per canonical entry, read back through the public API:
    tetm_set_fields keeps only entries that carry a field."""
    probe = tetm.Solver(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, "fp64", pec=w.pec)
    mask = np.zeros(probe.shape, np.uint8)
    ones = np.ones(probe.shape)
    for c in range(6):
        probe.set(c, ones)
        mask |= (probe.get(c) != 0).astype(np.uint8) << c
    probe.close()
    return mask


@pytest.mark.parametrize("precision,geometry", [("fp64", "collimator"), ("fp32", "collimator"),
                                                ("fp64", "box")])
def test_noalloc_energy_matches_tetm_energy_twice(tetm, precision, geometry):
    import torch
    if geometry == "box":
        w = wl.plain_pipe(nz=64, n=20, steps=90, precision=precision)
    else:
        w = wl.scaled_collimator(40, 96, sigma_cells=3.0, precision=precision)
        w.steps = 90
    s = tetm.Solver.from_workload(w)
    s.step(w.steps)
    w_ref = s.energy()
    host = [s.get(c) for c in range(6)]
    s.close()
    dt = torch.float64 if precision == "fp64" else torch.float32
    dev = torch.device("cuda", 0)
    fields = [torch.from_numpy(h).to(dev, dt).contiguous() for h in host]
    mask = None if geometry == "box" else torch.from_numpy(_active_mask(tetm, w)).to(dev)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
    grid = tetm.make_grid(w.nx, w.ny, w.nz, w.dx, w.dy, w.dz, w.cdt, precision)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        rc = tetm.tetm_energy_noalloc(grid, [f.data_ptr() for f in fields],
                                      0 if mask is None else mask.data_ptr(),
                                      out[call:].data_ptr(), stream)
        assert rc == tetm.TETM_OK, tetm.tetm_strerror(rc)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert w_ref > 0
    for v in got:
        assert v == pytest.approx(w_ref, rel=1e-12)


def test_noalloc_rejects_grids_beyond_its_scratch(tetm):
    grid = tetm.make_grid(256, 256, 600, 1e-3, 1e-3, 1e-3, 0.7e-3, "fp32")
    rc = tetm.tetm_energy_noalloc(grid, [1] * 6, 0, 1, 0)
    assert rc == tetm.TETM_E_TOO_LARGE
    assert "scratch" in tetm.tetm_strerror(rc)
