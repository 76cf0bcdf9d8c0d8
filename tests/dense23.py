"""Dense-matrix form of the explicit TE/TM scheme, built from the paper's
operator definitions, for brute-force checks on tiny grids.

This is a second, independent route to the same step as the oracle's ten
detailed updates (Sec. 4.2): the normalised skew system (5), its TE/TM
regrouping (15) into u = (hx, hy, ez), v = (ex, ey, hz), the factors
L_{T_i}, U_{T_i}, L_L of Sec. 4.2 and the two-level form (23)

    B^e (y^{n+1} - y^n)/dtau + A y^n = f^n,   B^e = L_L + L_T U_T,
    A = [[-T_0, -L], [L^T, -T_1]],  y^n = (u^{n-1/2}, v^n),
    f^n = (j_u^n, j_v^{n+1/2}),  j_u = (0, 0, -j_z),  j_v = (-j_x, -j_y, 0).

Only the grid sizes and the diagonal material matrices are taken from the
caller; the curl is assembled here from dense P_x, P_y, P_z.
"""
from __future__ import annotations

import numpy as np

C_LIGHT = 299792458.0


def shift_matrix(n, s):
    """Dense P with (P v)[i] = v[i+s] - v[i], v = 0 outside [0, n)."""
    p = -np.eye(n)
    for i in range(n - s):
        p[i, i + s] = 1.0
    return p


class Dense23:
    """coef: list of six canonical diagonals (M_eps^-1 for ex, ey, ez and
    M_mu^-1 for hx, hy, hz), flattened; dims (nx, ny, nz); cdt = c*dt."""

    def __init__(self, nx, ny, nz, coef, cdt):
        mx, my, mz = nx + 1, ny + 1, nz + 1
        n = mx * my * mz
        self.n = n
        px, py, pz = shift_matrix(n, 1), shift_matrix(n, mx), shift_matrix(n, mx * my)
        z = np.zeros((n, n))
        # curl of Sec. 2 acting on (ex, ey, ez) and giving face fluxes (bx, by, bz)
        curl = np.block([[z, -pz, py], [pz, z, -px], [-py, px, z]])
        me = np.concatenate([np.ravel(c) for c in coef[:3]])
        mh = np.concatenate([np.ravel(c) for c in coef[3:]])
        self.ae = np.nonzero(me > 0)[0]          # active e entries (0..3n)
        self.ah = np.nonzero(mh > 0)[0]          # active h entries (0..3n)
        self.de = np.sqrt(me[self.ae])
        self.dh = np.sqrt(mh[self.ah])
        c0 = (self.dh[:, None] * curl[np.ix_(self.ah, self.ae)] * self.de[None, :]) / C_LIGHT
        ne, nh = len(self.ae), len(self.ah)
        # full normalised skew operator on x = (e, h): de/dtau = C0^T h - j, dh/dtau = -C0 e
        k = np.zeros((ne + nh, ne + nh))
        k[:ne, ne:] = c0.T
        k[ne:, :ne] = -c0
        # component of every active entry: 0..2 e components, 3..5 h components
        comp = np.concatenate([self.ae // n, 3 + self.ah // n])
        u_sel = [np.nonzero(comp == c)[0] for c in (3, 4, 2)]   # hx, hy, ez
        v_sel = [np.nonzero(comp == c)[0] for c in (0, 1, 5)]   # ex, ey, hz
        self.u_idx = np.concatenate(u_sel)
        self.v_idx = np.concatenate(v_sel)
        perm = np.concatenate([self.u_idx, self.v_idx])
        self.perm = perm
        kk = k[np.ix_(perm, perm)]
        nu = len(self.u_idx)
        self.nu = nu
        t0, l_, t1, lt_neg = kk[:nu, :nu], kk[:nu, nu:], kk[nu:, nu:], kk[nu:, :nu]
        self.t0, self.l, self.t1 = t0, l_, t1
        self.skew_ok = np.max(np.abs(lt_neg + l_.T)) if l_.size else 0.0
        self.alpha = 0.5 * cdt
        self.dtau = cdt
        a = self.alpha
        blocks_u = [len(s) for s in u_sel]
        blocks_v = [len(s) for s in v_sel]
        lt0, ut0 = self._lu(t0, blocks_u, a)
        lt1, ut1 = self._lu(t1, blocks_v, a)
        nv = len(self.v_idx)
        be = np.zeros((nu + nv, nu + nv))
        be[:nu, :nu] = lt0 @ ut0
        be[nu:, nu:] = lt1 @ ut1
        be[nu:, :nu] = 2.0 * a * l_.T                       # L_L
        amat = np.block([[-t0, -l_], [l_.T, -t1]])
        self.be, self.a = be, amat
        self.qe = be - a * amat
        self.comp = comp
        self.ne = ne

    @staticmethod
    def _lu(t, sizes, a):
        """L_{T_i}, U_{T_i} of Sec. 4.2 from T_i = [[0,0,-p],[0,0,q],[p*,-q*,0]]."""
        n1, n2, n3 = sizes
        o1, o2 = n1, n1 + n2
        p = -t[:o1, o2:]
        q = t[o1:o2, o2:]
        nt = t.shape[0]
        lt = np.eye(nt)
        ut = np.eye(nt)
        lt[o2:, :o1] = -a * p.T
        lt[o2:, o1:o2] = a * q.T
        ut[:o1, o2:] = a * p
        ut[o1:o2, o2:] = -a * q
        return lt, ut

    # --- conversions between FIT integral fields and the normalised y --------
    def y_from_fields(self, f):
        """f: dict or list of six canonical arrays -> y = (u, v) normalised."""
        f = [np.ravel(f[c]) for c in range(6)] if not isinstance(f, dict) else \
            [np.ravel(f[c]) for c in ("ex", "ey", "ez", "hx", "hy", "hz")]
        ev = np.concatenate(f[:3])[self.ae] / self.de
        hv = np.concatenate(f[3:])[self.ah] / self.dh
        x = np.concatenate([ev, hv])
        return x[self.perm]

    def fields_from_y(self, y):
        x = np.empty_like(y)
        x[self.perm] = y
        e = np.zeros(3 * self.n)
        h = np.zeros(3 * self.n)
        e[self.ae] = x[:self.ne] * self.de
        h[self.ah] = x[self.ne:] * self.dh
        return [e[c * self.n:(c + 1) * self.n] for c in range(3)] + \
               [h[c * self.n:(c + 1) * self.n] for c in range(3)]

    def f_vec(self, jz=None, jx=None, jy=None):
        """f^n = (j_u^n, j_v^{n+1/2}) from FIT currents jj (canonical ez/ex/ey
        layouts); normalised j = c^-1 M_eps^-1/2 jj, Eq. (5)."""
        jj = np.zeros(3 * self.n)
        for c, a in ((0, jx), (1, jy), (2, jz)):
            if a is not None:
                jj[c * self.n:(c + 1) * self.n] = np.ravel(a)
        jn = jj[self.ae] * self.de / C_LIGHT
        x = np.concatenate([-jn, np.zeros(len(self.ah))])     # source of de/dtau is -j
        return x[self.perm]

    def step(self, y, f=None):
        rhs = -self.a @ y
        if f is not None:
            rhs = rhs + f
        return y + self.dtau * np.linalg.solve(self.be, rhs)

    def energy(self, y):
        return 0.5 * y @ (self.qe @ y)

    def propagator(self):
        return np.eye(self.be.shape[0]) - self.dtau * np.linalg.solve(self.be, self.a)
