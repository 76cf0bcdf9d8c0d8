"""Seeded synthetic workloads: grids, staircase PEC geometries and bunches.

This module holds input generation only — no part of the TE/TM arithmetic —
so that both the CUDA path and the CPU oracle can be fed the same inputs.

The paper's own structures (a transverse deflecting cavity and 20 TESLA cells,
Sec. 5) are not available as data; pipes, step collimators and pillbox
cavities with the paper's resolutions stand in for them: sigma/dz between 2.5
and 10 (Sec. 5), transverse steps larger than dz, vacuum, staircase PEC, bunch
on the axis.

Mesh. Every workload uses dz = 1 mm and dx = dy = sqrt(2) mm with c*dt = dz,
the mesh the paper quotes for its cost comparison (Sec. 4.2). A cubic mesh
with c*dt = dz violates the transverse bound of Eq. (25) and is only offered
as the negative case ``plain_pipe_cubic``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np

MM = 1e-3
DZ = 1.0 * MM
DXY = math.sqrt(2.0) * MM


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    cdt: float
    pec: Optional[np.ndarray]      # uint8 (nz, ny, nx), 1 = PEC, or None
    sigma: float                   # RMS bunch length [m]
    charge: float                  # [C]
    i0: int                        # node indices of the bunch line
    j0: int
    steps: int
    precision: str = "fp32"        # field storage: "fp64" | "fp32"
    kind: str = "pipe"

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def cell_steps(self) -> int:
        return self.cells * self.steps


def steps_for_window(nz: int, sigma: float, dz: float = DZ) -> int:
    """Steps for the bunch to enter (its head starts 5 sigma behind the
    entrance), cross nz cells and leave a 15 sigma wake window behind."""
    return nz + int(math.ceil(5.0 * sigma / dz - 1e-12)) + int(math.ceil(15.0 * sigma / dz - 1e-12)) + 1


def radius_mask(nx: int, ny: int, nz: int, radius_of_k: Callable[[np.ndarray], np.ndarray],
                cx: Optional[float] = None, cy: Optional[float] = None) -> np.ndarray:
    """Staircase round pipe: cell (ci, cj, ck) is PEC when the distance of its
    centre from the axis (cx, cy) in cell units exceeds radius_of_k(ck)."""
    cx = nx / 2.0 if cx is None else cx
    cy = ny / 2.0 if cy is None else cy
    ci = np.arange(nx) + 0.5 - cx
    cj = np.arange(ny) + 0.5 - cy
    r = np.sqrt(ci[None, :] ** 2 + cj[:, None] ** 2)             # (ny, nx)
    rk = np.asarray(radius_of_k(np.arange(nz)), dtype=np.float64)  # (nz,)
    radii, which = np.unique(rk, return_inverse=True)
    planes = np.stack([(r > rad).astype(np.uint8) for rad in radii])  # one mask per radius
    return planes[which.reshape(-1)]


def collimator_radius(nz: int, r_out: float, r_in: float, k1: int, k2: int):
    return lambda k: np.where((k >= k1) & (k < k2), r_in, r_out)


# ---------------------------------------------------------------------------
# The named configurations
# ---------------------------------------------------------------------------

def plain_pipe(nz: int = 96, n: int = 24, steps: int = 400, precision: str = "fp64") -> Workload:
    """3D rectangular PEC pipe n x n x nz (the box is the pipe), vacuum,
    sigma = 4 dz, 1 nC, bunch on the axis node (n/2, n/2), wake over 20 sigma."""
    return Workload("plain_pipe_%dx%dx%d" % (n, n, nz), n, n, nz, DXY, DXY, DZ, DZ, None,
                    4 * DZ, 1e-9, n // 2, n // 2, steps, precision, "box")


def plain_pipe_cubic(nz: int = 96, n: int = 24, steps: int = 400) -> Workload:
    """The same pipe on a cubic 1 mm mesh with c*dt = dz: outside Eq. (25)."""
    w = plain_pipe(nz, n, steps)
    w.name += "_cubic"
    w.dx = w.dy = DZ
    return w


def step_collimator(n: int = 256, nz: int = 2048, steps: int = 6000, precision: str = "fp32",
                    r_out: float = 96.0, r_in: float = 32.0) -> Workload:
    """Staircase step collimator: a round pipe about node (n/2, n/2) whose
    radius (in transverse cells) is r_out, then r_in over the middle half of
    the length, then r_out again. sigma = 6 dz, 1 nC, on axis."""
    k1, k2 = nz // 4, (3 * nz) // 4
    pec = radius_mask(n, n, nz, collimator_radius(nz, r_out, r_in, k1, k2))
    return Workload("step_collimator_%dx%dx%d" % (n, n, nz), n, n, nz, DXY, DXY, DZ, DZ, pec,
                    6 * DZ, 1e-9, n // 2, n // 2, steps, precision, "collimator")


def scaled_collimator(n: int, nz: int, sigma_cells: float = 6.0, steps: Optional[int] = None,
                      precision: str = "fp32") -> Workload:
    """The step collimator scaled to an n x n x nz grid (radii 3n/8 and n/8)."""
    w = step_collimator(n, nz, 0, precision, r_out=0.375 * n, r_in=0.125 * n)
    w.sigma = sigma_cells * DZ
    w.steps = steps if steps is not None else steps_for_window(nz, w.sigma)
    w.name = "collimator_%dx%dx%d" % (n, n, nz)
    return w


def dielectric_collimator(n: int = 256, nz: int = 1024, sigma_cells: float = 6.0,
                          precision: str = "fp32", eps_liner: float = 3.0):
    """The scaled step collimator with a dielectric liner: cells within 4
    transverse cells inside the narrow section's wall have eps_r = eps_liner.
    Returns (workload, eps_r per cell)."""
    w = scaled_collimator(n, nz, sigma_cells=sigma_cells, precision=precision)
    r_in = 0.125 * n
    k1, k2 = nz // 4, (3 * nz) // 4
    liner = radius_mask(n, n, nz, collimator_radius(nz, 1e9, r_in - 4.0, k1, k2))
    eps = np.ones((nz, n, n))
    eps[(liner == 1) & (w.pec == 0)] = eps_liner
    w.name = "dielectric_collimator_%dx%dx%d" % (n, n, nz)
    w.kind = "dielectric"
    return w, eps


def _solve_geometry(n: int, kind: str, rng: np.random.Generator):
    nz = 4 * n
    if kind == "pipe":
        r = rng.uniform(0.25, 0.45) * n
        return nz, (lambda k, r=r: np.full(k.shape, r))
    if kind == "cavity":
        # pipe of radius 0.2 N with one pillbox cell of radius 0.45 N in the middle
        return nz, collimator_radius(nz, 0.2 * n, 0.45 * n, int(1.5 * n), int(2.5 * n))
    if kind == "collimator":
        r1 = rng.uniform(0.3, 0.45) * n
        r2 = rng.uniform(0.08, 0.2) * n
        return nz, collimator_radius(nz, r1, r2, nz // 4, (3 * nz) // 4)
    raise ValueError(kind)


def make_solve(name: str, n: int, kind: str, sigma_cells: float, rng: np.random.Generator,
               precision: str = "fp32") -> Workload:
    nz, rad = _solve_geometry(n, kind, rng)
    pec = radius_mask(n, n, nz, rad)
    sigma = sigma_cells * DZ
    return Workload(name, n, n, nz, DXY, DXY, DZ, DZ, pec, sigma, 1e-9, n // 2, n // 2,
                    steps_for_window(nz, sigma), precision, kind)


def batch_solves(count: int = 64, seed: int = 9011053, n_lo: int = 32, n_hi: int = 192,
                 precision: str = "fp32") -> List[Workload]:
    """Uneven batch of pipe/cavity solves: N ~ U{n_lo..n_hi}, grid N x N x 4N,
    sigma ~ U[3, 10] dz. Draw order per solve: N, kind, shape, sigma."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        n -= n % 2
        kind = ("pipe", "cavity")[int(rng.integers(0, 2))]
        nz, rad = _solve_geometry(n, kind, rng)
        sigma = float(rng.uniform(3.0, 10.0)) * DZ
        pec = radius_mask(n, n, nz, rad)
        out.append(Workload("batch%02d_%s_%d" % (s, kind, n), n, n, nz, DXY, DXY, DZ, DZ, pec,
                            sigma, 1e-9, n // 2, n // 2, steps_for_window(nz, sigma),
                            precision, kind))
    return out


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                 # seconds since the start of the stream
    n: int
    kind: str
    sigma_cells: float
    seed: int

    def spec(self, precision: str = "fp32") -> "RequestSpec":
        """The request's sizes without its geometry (cheap); .build() makes
        the Workload, so a server can build it off its scheduling thread."""
        nz = 4 * self.n
        sigma = self.sigma_cells * DZ
        return RequestSpec(self, precision, self.n, self.n, nz, DXY, DXY, DZ, DZ,
                           steps_for_window(nz, sigma))

    def workload(self, precision: str = "fp32") -> Workload:
        rng = np.random.default_rng(self.seed)
        nz, rad = _solve_geometry(self.n, self.kind, rng)
        sigma = self.sigma_cells * DZ
        pec = radius_mask(self.n, self.n, nz, rad)
        return Workload("req%04d_%s_%d" % (self.rid, self.kind, self.n), self.n, self.n, nz,
                        DXY, DXY, DZ, DZ, pec, sigma, 1e-9, self.n // 2, self.n // 2,
                        steps_for_window(nz, sigma), precision, self.kind)


@dataclasses.dataclass
class RequestSpec:
    request: "Request"
    precision: str
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    cdt: float
    steps: int

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def build(self) -> Workload:
        return self.request.workload(self.precision)


def request_stream(count: int = 2000, rate: float = 40.0, seed: int = 9011054, n_lo: int = 48,
                   n_hi: int = 256) -> List[Request]:
    """Poisson stream of solve requests: exponential gaps of mean 1/rate,
    N ~ U{n_lo..n_hi}, kind in {pipe, cavity, collimator}, sigma ~ U[3,10] dz."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(count):
        t += float(rng.exponential(1.0 / rate))
        n = int(rng.integers(n_lo, n_hi + 1))
        n -= n % 2
        kind = ("pipe", "cavity", "collimator")[int(rng.integers(0, 3))]
        sig = float(rng.uniform(3.0, 10.0))
        out.append(Request(r, t, n, kind, sig, int(rng.integers(0, 2**31 - 1))))
    return out


def coax_pec(nx: int, ny: int, nz: int, rod) -> np.ndarray:
    """Coaxial line along z: the PEC rod cells [i_lo, i_hi) x [j_lo, j_hi) in every
    plane; the PEC box is the outer conductor."""
    i_lo, i_hi, j_lo, j_hi = rod
    pec = np.zeros((nz, ny, nx), dtype=np.uint8)
    pec[:, j_lo:j_hi, i_lo:i_hi] = 1
    return pec


def coax_tem_e(nx: int, ny: int, dx: float, dy: float, rod):
    """Transverse shape of the coaxial line's TEM field, an input profile: the
    node potential phi = 1 on the rod's nodes, 0 on the box wall, and
    (phi(i+1) - 2 phi(i) + phi(i-1)) / dx^2 + (phi(j+1) - 2 phi(j) + phi(j-1)) / dy^2 = 0
    at every other node; returns the edge voltages e_x = -(phi(i+1,j) - phi(i,j)) and
    e_y = -(phi(i,j+1) - phi(i,j)) as (ny+1, nx+1) arrays."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    i_lo, i_hi, j_lo, j_hi = rod
    mx, my = nx + 1, ny + 1
    fixed = np.zeros((my, mx), dtype=bool)
    phi = np.zeros((my, mx))
    fixed[0, :] = fixed[-1, :] = fixed[:, 0] = fixed[:, -1] = True
    fixed[j_lo:j_hi + 1, i_lo:i_hi + 1] = True
    phi[j_lo:j_hi + 1, i_lo:i_hi + 1] = 1.0
    free = np.flatnonzero(~fixed.ravel())
    pos = -np.ones(mx * my, dtype=np.int64)
    pos[free] = np.arange(free.size)
    wx, wy = 1.0 / dx ** 2, 1.0 / dy ** 2
    rows, cols, vals = [], [], []
    rhs = np.zeros(free.size)
    for q, node in enumerate(free):
        j, i = divmod(int(node), mx)
        rows.append(q)
        cols.append(q)
        vals.append(-2.0 * (wx + wy))
        for (jj, ii), w in (((j, i - 1), wx), ((j, i + 1), wx), ((j - 1, i), wy), ((j + 1, i), wy)):
            nb = jj * mx + ii
            if fixed[jj, ii]:
                rhs[q] -= w * phi[jj, ii]
            else:
                rows.append(q)
                cols.append(int(pos[nb]))
                vals.append(w)
    a = sp.csr_matrix((vals, (rows, cols)), shape=(free.size, free.size))
    phi.ravel()[free] = spl.spsolve(a.tocsc(), rhs)
    ex = np.zeros((my, mx))
    ey = np.zeros((my, mx))
    ex[:, :-1] = -(phi[:, 1:] - phi[:, :-1])
    ey[:-1, :] = -(phi[1:, :] - phi[:-1, :])
    return ex, ey


def random_fields(shape, seed: int, scale: float = 1.0):
    """Six seeded standard-normal arrays (ex, ey, ez, hx, hy, hz)."""
    rng = np.random.default_rng(seed)
    return [scale * rng.standard_normal(shape) for _ in range(6)]


def random_materials(nx: int, ny: int, nz: int, seed: int):
    """Seeded per-cell eps_r, mu_r in [1, 4) and a sparse random PEC mask."""
    rng = np.random.default_rng(seed)
    eps = rng.uniform(1.0, 4.0, (nz, ny, nx))
    mu = rng.uniform(1.0, 4.0, (nz, ny, nx))
    pec = (rng.uniform(size=(nz, ny, nx)) < 0.1).astype(np.uint8)
    return eps, mu, pec


# ---------------------------------------------------------------------------
# Rotationally symmetric workloads (Sec. 4.3): (r, z) grids, modes m_lo..m_hi
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class RzWorkload:
    name: str
    nr: int
    nz: int
    m_lo: int
    m_hi: int
    dr: float
    dz: float
    cdt: float
    pec: Optional[np.ndarray]      # uint8 (nz, nr), 1 = PEC, or None
    sigma: float
    charge: float
    i0: int                        # ring r = i0 * dr of the bunch (0: the axis, m = 0 only)
    steps: int
    precision: str = "fp32"

    @property
    def n_modes(self) -> int:
        return self.m_hi - self.m_lo + 1

    @property
    def cells(self) -> int:
        """Cells of all modes: one (r, z) grid per mode."""
        return self.n_modes * self.nr * self.nz


def rz_radius_mask(nr: int, nz: int, radius_of_k: Callable[[np.ndarray], np.ndarray]) -> np.ndarray:
    """Staircase body of revolution: cell (ci, ck) is PEC when its centre
    radius (ci + 1/2) exceeds radius_of_k(ck) (in cells)."""
    rk = np.asarray(radius_of_k(np.arange(nz)), dtype=np.float64)
    ci = np.arange(nr) + 0.5
    return (ci[None, :] > rk[:, None]).astype(np.uint8)


def cavity_chain_radius(nz: int, n_cells: int, r_cav: float, r_iris: float, period: int,
                        gap: int):
    """Radius per plane of a chain of n_cells pillbox cells (radius r_cav,
    length gap) separated by irises (radius r_iris, length period - gap),
    centred in nz planes with beam pipes of radius r_iris on both sides."""
    start = (nz - n_cells * period) // 2

    def rad(k):
        k = np.asarray(k)
        rel = k - start - (period - gap) // 2
        inside = (rel >= 0) & (rel < n_cells * period) & ((rel % period) < gap)
        return np.where(inside, r_cav, r_iris)
    return rad


def cavity_chain_rz(nr: int = 512, nz: int = 16384, m_lo: int = 0, m_hi: int = 4,
                    sigma_cells: float = 8.0, precision: str = "fp32", steps: Optional[int] = None,
                    n_cells: int = 9, i0: Optional[int] = None) -> RzWorkload:
    """Chain of 9 pillbox cells on an (r, z) grid (stand-in for the paper's
    multi-cell structures): cavity radius 400/512 of nr, iris and pipe radius
    160/512 of nr, period 3/32 of nz with 3/4 of it cavity gap; dr = dz =
    0.25 mm, c*dt = dz; Gaussian bunch sigma = 8 dz, 1 nC, on the ring
    i0 = nr/64 (the axis when only m = 0 is solved)."""
    r_cav, r_iris = 400.0 * nr / 512.0, 160.0 * nr / 512.0
    period = max(4, (3 * nz) // 32)
    gap = (3 * period) // 4
    pec = rz_radius_mask(nr, nz, cavity_chain_radius(nz, n_cells, r_cav, r_iris, period, gap))
    dz = 0.25 * MM
    sigma = sigma_cells * dz
    if i0 is None:
        i0 = 0 if m_hi == 0 else max(1, nr // 64)
    st = steps if steps is not None else steps_for_window(nz, sigma, dz)
    return RzWorkload("cavity_chain_rz_%dx%d_m%d-%d" % (nr, nz, m_lo, m_hi), nr, nz, m_lo, m_hi,
                      dz, dz, dz, pec, sigma, 1e-9, i0, st, precision)
