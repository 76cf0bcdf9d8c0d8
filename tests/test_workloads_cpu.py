"""The seeded input generators (paper_0901_1053_gb300/workloads.py): shapes,
seeds and the geometric facts the measurements rely on. They hold none of the
method's arithmetic; these tests check the inputs themselves."""
import math

import numpy as np

from paper_0901_1053_gb300 import workloads as wl


def test_step_collimator_geometry():
    w = wl.step_collimator(nz=64)
    assert (w.nx, w.ny, w.nz) == (256, 256, 64) and w.pec.shape == (64, 256, 256)
    assert w.precision == "fp32" and w.cdt == w.dz and abs(w.dx - math.sqrt(2.0) * w.dz) < 1e-15
    # a cell is PEC when its centre lies outside radius 96 (in transverse cells) about (128, 128)
    assert w.pec[0, 128, 128] == 0 and w.pec[0, 128, 128 + 95] == 0 and w.pec[0, 128, 128 + 96] == 1
    assert w.sigma == 6 * w.dz and (w.i0, w.j0) == (128, 128)


def test_seeded_streams_repeat_and_differ():
    a = wl.batch_solves(count=8)
    b = wl.batch_solves(count=8)
    assert [(x.nx, x.nz, x.sigma) for x in a] == [(x.nx, x.nz, x.sigma) for x in b]
    assert all(x.nz == 4 * x.nx for x in a)
    r1 = wl.request_stream(count=50)
    r2 = wl.request_stream(count=50, seed=1)
    t = [r.arrival for r in r1]
    assert t == sorted(t) and t != [r.arrival for r in r2]
    assert all(48 <= r.n <= 256 and 3.0 <= r.sigma_cells <= 10.0 for r in r1)


def test_coaxial_tem_profile_solves_the_discrete_laplace_equation():
    nx, ny = 12, 10
    dx, dy = 1.3e-3, 1.1e-3
    rod = (5, 7, 4, 6)
    ex, ey = wl.coax_tem_e(nx, ny, dx, dy, rod)
    # rebuild phi from the edge voltages along the first row and up the columns
    phi = np.zeros((ny + 1, nx + 1))
    phi[0, 1:] = -np.cumsum(ex[0, :-1])
    phi[1:, :] = phi[0, :] - np.cumsum(ey[:-1, :], axis=0)
    # the box wall is at 0, the rod's nodes at 1
    assert np.max(np.abs(phi[[0, -1], :])) < 1e-12 and np.max(np.abs(phi[:, [0, -1]])) < 1e-12
    assert np.max(np.abs(phi[4:7, 5:8] - 1.0)) < 1e-12
    # curl-free: the voltage around every cell sums to zero
    circ = ex[:-1, :-1] + ey[:-1, 1:] - ex[1:, :-1] - ey[:-1, :-1]
    assert np.max(np.abs(circ)) < 1e-12
    # discrete Laplace equation at every free node
    lap = ((phi[1:-1, 2:] - 2 * phi[1:-1, 1:-1] + phi[1:-1, :-2]) / dx ** 2
           + (phi[2:, 1:-1] - 2 * phi[1:-1, 1:-1] + phi[:-2, 1:-1]) / dy ** 2)
    fixed = np.zeros((ny + 1, nx + 1), dtype=bool)
    fixed[4:7, 5:8] = True
    free = ~fixed[1:-1, 1:-1]
    assert np.max(np.abs(lap[free])) < 1e-9 * np.max(np.abs(lap[~free]))
    # the rod is the only source: phi lies strictly between the conductors' values
    inner = phi[1:-1, 1:-1][free]
    assert np.all((inner > 0.0) & (inner < 1.0))


def test_coax_pec_is_a_rod_through_every_plane():
    pec = wl.coax_pec(10, 8, 5, (4, 6, 3, 5))
    assert pec.shape == (5, 8, 10) and int(pec.sum()) == 5 * 4
    assert np.all(pec[:, 3:5, 4:6] == 1)
