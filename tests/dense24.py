"""Dense-matrix form of the rotationally symmetric explicit scheme (Sec. 4.3,
Eq. (24)) for one azimuthal mode m, built from operator definitions, for
brute-force checks on tiny (r, z) grids.

A second route to the same step as the oracle's ten detailed updates: the
per-mode curl (the azimuthal derivative of a mode is a multiplication by m),
the normalised skew system, its TE/TM regrouping into
u = (h_phi, h_r, e_z), v = (e_phi, e_r, h_z), the factors L_{T_i}, U_{T_i},
L_L of Sec. 4.2 with the transverse differences (P_r, m), and the two-level
form (24)

    B^{e,r} (y^{n+1} - y^n)/dtau + A y^n = f^n,
    B^{e,r} = B - alpha^2 R^r = L_L + L_T U_T + alpha^2 R^m,

where R^r holds P_r^* P_r and R^m the m^2 part of the splitting operator.
Nothing here writes the implicit diagonal factor of the detailed updates:
``step`` solves with B^{e,r} directly.

Component order of the coefficient list: e_r, e_phi, e_z, h_r, h_phi, h_z,
each flattened from the canonical (nz+1, nr+1) layout (r fastest).
"""
from __future__ import annotations

import numpy as np

from dense23 import Dense23, shift_matrix, C_LIGHT


def mode_curl(nr, nz, m):
    """Curl of a mode-m field acting on (e_r, e_phi, e_z) and giving the face
    fluxes of (h_r, h_phi, h_z), with P^* = P^T:
        h_r   <- -P_z e_phi + m e_z
        h_phi <-  P_z e_r   - P_r e_z
        h_z   <-  P_r e_phi - m e_r
    returned as C with M_mu dh/dt = -C e, M_eps de/dt = C^T h - j."""
    n = (nr + 1) * (nz + 1)
    pr, pz = shift_matrix(n, 1), shift_matrix(n, nr + 1)
    z = np.zeros((n, n))
    mi = m * np.eye(n)
    k = np.block([[z, -pz, mi], [pz, z, -pr], [-mi, pr, z]])
    return -k


class Dense24(Dense23):
    def __init__(self, nr, nz, m, coef, cdt):
        n = (nr + 1) * (nz + 1)
        self.n = n
        curl = mode_curl(nr, nz, m)
        me = np.concatenate([np.ravel(c) for c in coef[:3]])
        mh = np.concatenate([np.ravel(c) for c in coef[3:]])
        self.ae = np.nonzero(me > 0)[0]
        self.ah = np.nonzero(mh > 0)[0]
        self.de = np.sqrt(me[self.ae])
        self.dh = np.sqrt(mh[self.ah])
        c0 = (self.dh[:, None] * curl[np.ix_(self.ah, self.ae)] * self.de[None, :]) / C_LIGHT
        ne, nh = len(self.ae), len(self.ah)
        k = np.zeros((ne + nh, ne + nh))
        k[:ne, ne:] = c0.T
        k[ne:, :ne] = -c0
        comp = np.concatenate([self.ae // n, 3 + self.ah // n])
        u_sel = [np.nonzero(comp == c)[0] for c in (4, 3, 2)]   # h_phi, h_r, e_z
        v_sel = [np.nonzero(comp == c)[0] for c in (1, 0, 5)]   # e_phi, e_r, h_z
        self.u_idx = np.concatenate(u_sel)
        self.v_idx = np.concatenate(v_sel)
        perm = np.concatenate([self.u_idx, self.v_idx])
        self.perm = perm
        kk = k[np.ix_(perm, perm)]
        nu = len(self.u_idx)
        nv = len(self.v_idx)
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
        rm0 = self._r_m(t0, blocks_u)
        rm1 = self._r_m(t1, blocks_v)
        be = np.zeros((nu + nv, nu + nv))
        be[:nu, :nu] = lt0 @ ut0 + a * a * rm0
        be[nu:, nu:] = lt1 @ ut1 + a * a * rm1
        be[nu:, :nu] = 2.0 * a * l_.T
        amat = np.block([[-t0, -l_], [l_.T, -t1]])
        self.be, self.a = be, amat
        self.qe = be - a * amat
        self.comp = comp
        self.ne = ne

    @staticmethod
    def _r_m(t, sizes):
        """R^m_i: q^* q in the third diagonal block, q the m-coupling of T_i."""
        n1, n2, n3 = sizes
        o1, o2 = n1, n1 + n2
        q = t[o1:o2, o2:]
        r = np.zeros_like(t)
        r[o2:, o2:] = q.T @ q
        return r

    def y_from_fields(self, f):
        names = ("er", "ephi", "ez", "hr", "hphi", "hz")
        f = [np.ravel(f[c]) for c in names] if isinstance(f, dict) else \
            [np.ravel(f[c]) for c in range(6)]
        ev = np.concatenate(f[:3])[self.ae] / self.de
        hv = np.concatenate(f[3:])[self.ah] / self.dh
        x = np.concatenate([ev, hv])
        return x[self.perm]

    def f_vec(self, jz=None):
        return super().f_vec(jz=jz)
