/*
 * Plain FP64 CPU oracle of the explicit TE/TM scheme for rotationally
 * symmetric structures (Sec. 4.3, Eq. (24)), one azimuthal mode m at a time.
 *
 * TEST INFRASTRUCTURE. Like tetm_oracle.c this is the slow reference the CUDA
 * path is checked against; only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it, and it shares no code with the
 * product library.
 *
 * Fields of mode m (cos/sin pairing): E_r, E_z, H_phi ~ cos(m phi) and
 * E_phi, H_r, H_z ~ sin(m phi). Grid: primary cells nr x nz in (r, z),
 * nodes r_i = i dr (i = 0 .. nr, the axis is i = 0, the PEC wall i = nr),
 * z_k = k dz. One vector per component over the canonical index
 * n = i + (nr+1) k (r fastest), integral quantities per radian of azimuth:
 *   er   (r_{i+1/2}, z_k)        edge along r          [V]
 *   ephi (r_i, z_k)              edge along phi, length r_i
 *   ez   (r_i, z_{k+1/2})        edge along z          [V]
 *   hphi (r_{i+1/2}, z_{k+1/2})  dual edge along phi, face = the r-z cell
 *   hr   (r_i, z_{k+1/2})        face normal to r at r_i (area r_i dz)
 *   hz   (r_{i+1/2}, z_k)        face normal to z (area r_{i+1/2} dr)
 * In these variables the azimuthal derivative of a mode is a multiplication
 * by m, so the scheme is the 3D one of Sec. 4.2 with the x-differences
 * replaced by m: the TM stage updates (hphi, hr, ez), the TE stage (ephi, er,
 * hz). Keeping the m-part of the splitting operator in B^{e,r} (Sec. 4.3)
 * puts a diagonal factor (I + alpha^2 m^2 M M)^-1 on the ez and hz updates;
 * it pairs each ez edge with the hr face of the same index and each hz face
 * with the er edge of the same index (these are the entries the m-terms
 * couple).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define RZ_C0 299792458.0
#define RZ_EPS0 8.8541878128e-12
#define RZ_MU0 (1.0 / (RZ_EPS0 * RZ_C0 * RZ_C0))
#define RZ_PI 3.14159265358979323846

enum { ER = 0, EPHI, EZ, HR, HPHI, HZ };  /* (r, phi, z) order for both families */

typedef struct rz_oracle {
  int nr, nz, m;
  long mr, n;        /* mr = nr + 1, n = (nr+1)(nz+1) */
  double dr, dz, dt, at;
  double *f[6], *c[6];  /* fields; M^-1 diagonals (0 = inactive) */
  int has_bunch, i0, c0, m_min, m_max;
  double sigma, q, weight;
  double *qcell, *wake, *jz;
  /* transverse wake at r_{obs+1/2} and longitudinal wakes at rings obs, obs+1 */
  int obs;
  double *twake, *wake_o0, *wake_o1;
  long kshift;   /* bunch head at plane step + kshift (0: cold start at the wall) */
  int vacuum;    /* no material arrays were given */
  long step;
} rz_oracle_t;

static double Pz(const rz_oracle_t *o, const double *v, long n) {
  return (n + o->mr < o->n ? v[n + o->mr] : 0.0) - v[n];
}
static double PzT(const rz_oracle_t *o, const double *v, long n) {
  return (n - o->mr >= 0 ? v[n - o->mr] : 0.0) - v[n];
}
static double Pr(const rz_oracle_t *o, const double *v, long n) {
  return (n + 1 < o->n ? v[n + 1] : 0.0) - v[n];
}
static double PrT(const double *v, long n) { return (n - 1 >= 0 ? v[n - 1] : 0.0) - v[n]; }

/* cell (ci, ck) is PEC when outside the grid (ci >= nr, ck < 0, ck >= nz) or
 * marked; ci < 0 is the mirror image through the axis (same cell as ci = 0
 * is never needed: the axis is not a wall) */
static int rz_pec(const rz_oracle_t *o, const uint8_t *pec, long ci, long ck) {
  if (ci >= o->nr || ck < 0 || ck >= o->nz) return 1;
  if (ci < 0) ci = -ci - 1;
  return pec ? pec[ci + (long)o->nr * ck] != 0 : 0;
}

/* Per-radian cylindrical FIT metric (staircase: an edge is PEC if a cell
 * sharing it is; a face is active only if both cells sharing it are not):
 *   er   L = dr,       dual area r_{i+1/2} dz
 *   ephi L = r_i,      dual area dr dz
 *   ez   L = dz,       dual area r_i dr (dr^2/4 on the axis, see below)
 *   hphi area dr dz,   dual L = r_{i+1/2}
 *   hr   area r_i dz,  dual L = dr (inactive on the axis: zero area)
 *   hz   area r_{i+1/2} dr, dual L = dz
 * eps_r, mu_r per cell or NULL (vacuum); averaging as in the 3D oracle. On
 * the axis the ez edge exists for m = 0 only (E_z ~ cos(m phi) must vanish
 * on r = 0 for m >= 1). Its dual area is taken as dr^2/4 per radian: with
 * the disc r < dr/2 (dr^2/8) the radial operator P_r^* P_r has spectral
 * radius 1.21 * 4/dr^2 and the scheme would need c*dt <= 0.909 dr, while
 * Sec. 4.4 states c*dt <= min(dr, dz) for every m; dr^2/4 keeps the radius
 * below 4/dr^2 and the scheme second-order accurate.
 * cdt = c*dt (0 -> min(dr, dz), the bound of Sec. 4.4). */
rz_oracle_t *rz_oracle_new(int nr, int nz, int m, double dr, double dz, double cdt,
                           const double *eps_r, const double *mu_r, const uint8_t *pec) {
  if (nr < 2 || nz < 2 || m < 0 || !(dr > 0) || !(dz > 0) || cdt < 0) return NULL;
  rz_oracle_t *o = (rz_oracle_t *)calloc(1, sizeof(rz_oracle_t));
  o->nr = nr; o->nz = nz; o->m = m;
  o->mr = nr + 1;
  o->n = (long)(nr + 1) * (nz + 1);
  o->dr = dr; o->dz = dz;
  o->dt = (cdt > 0 ? cdt : (dr < dz ? dr : dz)) / RZ_C0;
  o->vacuum = (eps_r == NULL && mu_r == NULL);
  o->at = 0.5 * o->dt;
  for (int q = 0; q < 6; ++q) {
    o->f[q] = (double *)calloc((size_t)o->n, sizeof(double));
    o->c[q] = (double *)calloc((size_t)o->n, sizeof(double));
  }
  o->jz = (double *)calloc((size_t)o->n, sizeof(double));
#define EPS(ci, ck) (eps_r ? eps_r[(ci) + (long)nr * (ck)] : 1.0)
#define MU(ci, ck) (mu_r ? mu_r[(ci) + (long)nr * (ck)] : 1.0)
  for (long k = 0; k <= nz; ++k)
    for (long i = 0; i <= nr; ++i) {
      const long n = i + o->mr * k;
      const double ri = i * dr, rh = (i + 0.5) * dr;
      if (i < nr) { /* er: cells (i, k-1), (i, k) */
        if (!rz_pec(o, pec, i, k - 1) && !rz_pec(o, pec, i, k)) {
          const double e = 0.5 * (EPS(i, k - 1) + EPS(i, k));
          o->c[ER][n] = dr / (RZ_EPS0 * e * rh * dz);
        }
      }
      if (i > 0) { /* ephi: cells (i-1..i, k-1..k) */
        int bad = 0;
        double e = 0.0;
        for (int a = -1; a <= 0; ++a)
          for (int b = -1; b <= 0; ++b) {
            if (rz_pec(o, pec, i + a, k + b)) bad = 1;
            else e += EPS(i + a, k + b);
          }
        if (!bad) o->c[EPHI][n] = ri / (RZ_EPS0 * (e / 4.0) * dr * dz);
      }
      if (k < nz) { /* ez: cells (i-1, k), (i, k); axis: the disc */
        if (i == 0) {
          if (m == 0 && !rz_pec(o, pec, 0, k))
            o->c[EZ][n] = dz / (RZ_EPS0 * EPS(0, k) * dr * dr / 4.0);
        } else if (!rz_pec(o, pec, i - 1, k) && !rz_pec(o, pec, i, k)) {
          const double e = 0.5 * (EPS(i - 1, k) + EPS(i, k));
          o->c[EZ][n] = dz / (RZ_EPS0 * e * ri * dr);
        }
      }
      if (i < nr && k < nz && !rz_pec(o, pec, i, k)) /* hphi: the cell itself */
        o->c[HPHI][n] = rh / (RZ_MU0 * MU(i, k) * dr * dz);
      if (i > 0 && k < nz && !rz_pec(o, pec, i - 1, k) && !rz_pec(o, pec, i, k)) { /* hr */
        const double ir = 0.5 * (1.0 / MU(i - 1, k) + 1.0 / MU(i, k));
        o->c[HR][n] = dr * ir / (RZ_MU0 * ri * dz);
      }
      if (i < nr && !rz_pec(o, pec, i, k - 1) && !rz_pec(o, pec, i, k)) { /* hz */
        const double ir = 0.5 * (1.0 / MU(i, k - 1) + 1.0 / MU(i, k));
        o->c[HZ][n] = dz * ir / (RZ_MU0 * rh * dr);
      }
    }
#undef EPS
#undef MU
  return o;
}

void rz_oracle_free(rz_oracle_t *o) {
  if (!o) return;
  for (int q = 0; q < 6; ++q) { free(o->f[q]); free(o->c[q]); }
  free(o->jz); free(o->qcell); free(o->wake);
  free(o->twake); free(o->wake_o0); free(o->wake_o1);
  free(o);
}

static double Phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* Gaussian bunch as in the 3D oracle (truncated at +-5 sigma, head at z = 0
 * at t = 0), on the ring r = i0 dr (the axis for i0 = 0). A point charge at
 * azimuth 0 has the mode-m share (2 - delta_m0)/(2 pi) per radian. */
int rz_oracle_set_bunch(rz_oracle_t *o, double sigma, double q, int i0) {
  if (!(sigma > 0) || q == 0 || i0 < 0 || i0 >= o->nr) return -1;
  if (i0 == 0 && o->m != 0) return -1;  /* only m = 0 lives on the axis */
  o->has_bunch = 1;
  o->sigma = sigma; o->q = q; o->i0 = i0;
  o->weight = (o->m == 0 ? 1.0 : 2.0) / (2.0 * RZ_PI);
  o->c0 = (int)ceil(5.0 * sigma / o->dz - 1e-12);
  o->m_min = -o->c0 - 1;
  o->m_max = (int)ceil(15.0 * sigma / o->dz - 1e-12);
  free(o->qcell); free(o->wake); free(o->twake); free(o->wake_o0); free(o->wake_o1);
  o->qcell = (double *)calloc((size_t)(2 * o->c0), sizeof(double));
  o->wake = (double *)calloc((size_t)(o->m_max - o->m_min + 1), sizeof(double));
  o->twake = (double *)calloc((size_t)(o->m_max - o->m_min + 1), sizeof(double));
  o->wake_o0 = (double *)calloc((size_t)(o->m_max - o->m_min + 1), sizeof(double));
  o->wake_o1 = (double *)calloc((size_t)(o->m_max - o->m_min + 1), sizeof(double));
  o->obs = i0;
  for (int d = -o->c0; d < o->c0; ++d) {
    double a = d * o->dz, b = (d + 1) * o->dz;
    if (a < -5.0 * sigma) a = -5.0 * sigma;
    if (b > 5.0 * sigma) b = 5.0 * sigma;
    o->qcell[d + o->c0] = (b > a) ? q * (Phi(b / sigma) - Phi(a / sigma)) : 0.0;
  }
  return 0;
}

void rz_oracle_current(const rz_oracle_t *o, long n, double *jz) {
  memset(jz, 0, sizeof(double) * (size_t)o->n);
  if (!o->has_bunch) return;
  for (long k = 0; k < o->nz; ++k) {
    const long d = k - (n + o->kshift) + o->c0;
    if (d < -o->c0 || d >= o->c0) continue;
    jz[o->i0 + o->mr * k] = o->weight * RZ_C0 * o->qcell[d + o->c0] / o->dz;
  }
}

/* One step of Eq. (24) in the paper's order. */
void rz_oracle_step_j(rz_oracle_t *o, const double *jz) {
  double *er = o->f[ER], *ep = o->f[EPHI], *ez = o->f[EZ];
  double *hp = o->f[HPHI], *hr = o->f[HR], *hz = o->f[HZ];
  const double *cer = o->c[ER], *cep = o->c[EPHI], *cez = o->c[EZ];
  const double *chp = o->c[HPHI], *chr = o->c[HR], *chz = o->c[HZ];
  const double a = o->at, m = (double)o->m;
  const long N = o->n;
  /* TM stage */
  for (long n = 0; n < N; ++n) hp[n] += a * chp[n] * (Pz(o, er, n) - Pr(o, ez, n));
  for (long n = 0; n < N; ++n) hr[n] += a * chr[n] * (-Pz(o, ep, n) + m * ez[n]);
  for (long n = 0; n < N; ++n)
    ez[n] += 2.0 * a * cez[n] * (PrT(hp, n) - m * hr[n] - (jz ? jz[n] : 0.0)) /
             (1.0 + a * a * m * m * cez[n] * chr[n]);
  for (long n = 0; n < N; ++n) hp[n] += a * chp[n] * (Pz(o, er, n) - Pr(o, ez, n));
  for (long n = 0; n < N; ++n) hr[n] += a * chr[n] * (-Pz(o, ep, n) + m * ez[n]);
  /* TE stage */
  for (long n = 0; n < N; ++n) ep[n] += a * cep[n] * (PzT(o, hr, n) - PrT(hz, n));
  for (long n = 0; n < N; ++n) er[n] += a * cer[n] * (-PzT(o, hp, n) + m * hz[n]);
  for (long n = 0; n < N; ++n)
    hz[n] += 2.0 * a * chz[n] * (Pr(o, ep, n) - m * er[n]) / (1.0 + a * a * m * m * chz[n] * cer[n]);
  for (long n = 0; n < N; ++n) ep[n] += a * cep[n] * (PzT(o, hr, n) - PrT(hz, n));
  for (long n = 0; n < N; ++n) er[n] += a * cer[n] * (-PzT(o, hp, n) + m * hz[n]);
}

/* Wakes (Sec. 5) along the path s = m*dz behind the bunch centre: with
 * c*dt = dz the path meets e_z(k+1/2) at time n+1/2, e_r(k) at time n and
 * h_phi(k+1/2) at time n+1/2 for the same n = k + m + c0.
 * Longitudinal: W(s) = -(1/Q) sum e_z at the bunch ring (and at rings obs,
 * obs+1). Transverse, radial component at r = r_{obs+1/2}, phi = 0 (the
 * paper's dipole wake, Sec. 5): W_r(s) = (1/Q) sum (E_r - c mu0 H_phi) dz,
 * with E_r = e_r/dr and, per radian, h_phi = -r H_phi (the sign with which
 * the m-terms of (24) are written), so E_r - c mu0 H_phi =
 * e_r/dr + eta0 h_phi/r_{obs+1/2}. er_n: e_r before the step. */
static void rz_wake_gather(rz_oracle_t *o, long n, const double *er_n) {
  const double eta0 = RZ_MU0 * RZ_C0;
  const double rh = (o->obs + 0.5) * o->dr;
  for (int mm = o->m_min; mm <= o->m_max; ++mm) {
    const long k = (n + o->kshift) - mm - o->c0;
    if (k < 0 || k >= o->nz) continue;
    const int w = mm - o->m_min;
    o->wake[w] -= o->f[EZ][o->i0 + o->mr * k] / o->q;
    o->wake_o0[w] -= o->f[EZ][o->obs + o->mr * k] / o->q;
    o->wake_o1[w] -= o->f[EZ][o->obs + 1 + o->mr * k] / o->q;
    o->twake[w] += (er_n[o->obs + o->mr * k] / o->dr + eta0 * o->f[HPHI][o->obs + o->mr * k] / rh) *
                   o->dz / o->q;
  }
}

static void rz_step_gather(rz_oracle_t *o, const double *jz) {
  double *er_n = NULL;
  if (o->has_bunch) {
    er_n = (double *)malloc(sizeof(double) * (size_t)o->n);
    memcpy(er_n, o->f[ER], sizeof(double) * (size_t)o->n);
  }
  rz_oracle_step_j(o, jz);
  if (o->has_bunch) rz_wake_gather(o, o->step, er_n);
  free(er_n);
  o->step += 1;
}

void rz_oracle_step(rz_oracle_t *o, int nsteps) {
  for (int s = 0; s < nsteps; ++s) {
    if (o->has_bunch) rz_oracle_current(o, o->step, o->jz);
    rz_step_gather(o, o->has_bunch ? o->jz : NULL);
  }
}

void rz_oracle_step_custom(rz_oracle_t *o, const double *jz) { rz_step_gather(o, jz); }

/* Observation radius of the transverse wake: r_{obs+1/2}, 0 <= obs < nr - 1
 * (before the first step; the bunch ring by default). */
int rz_oracle_set_observer(rz_oracle_t *o, int obs) {
  if (!o->has_bunch || o->step != 0 || obs < 0 || obs >= o->nr - 1) return -1;
  o->obs = obs;
  return 0;
}

/* which: 0 the transverse wake at r_{obs+1/2}, 1 / 2 the longitudinal wakes
 * at rings obs / obs+1 (same window as rz_oracle_wake) */
int rz_oracle_wake_extra(const rz_oracle_t *o, int which, double *out, int cap) {
  if (!o->has_bunch || which < 0 || which > 2) return -1;
  const int nw = o->m_max - o->m_min + 1;
  if (cap < nw) return -1;
  const double *src = which == 0 ? o->twake : (which == 1 ? o->wake_o0 : o->wake_o1);
  memcpy(out, src, sizeof(double) * (size_t)nw);
  return 0;
}

int rz_oracle_wake(const rz_oracle_t *o, double *out, int cap, int *n_out, double *s0, double *ds) {
  if (!o->has_bunch) return -1;
  const int nw = o->m_max - o->m_min + 1;
  if (n_out) *n_out = nw;
  if (s0) *s0 = o->m_min * o->dz;
  if (ds) *ds = o->dz;
  if (out) {
    if (cap < nw) return -1;
    memcpy(out, o->wake, sizeof(double) * (size_t)nw);
  }
  return 0;
}

/* Discrete energy 1/2 <Q^{e,r} y, y>, Q^{e,r} = B^{e,r} - alpha A (Sec. 4.3,
 * 4.4): as in 3D, with only the r-part of the splitting operator subtracted
 * (the m-part stays in B^{e,r}). */
double rz_oracle_energy(const rz_oracle_t *o) {
  const double a = o->at;
  double w = 0.0, r = 0.0, l = 0.0;
  for (int q = 0; q < 6; ++q)
    for (long n = 0; n < o->n; ++n)
      if (o->c[q][n] != 0.0) w += 0.5 * o->f[q][n] * o->f[q][n] / o->c[q][n];
  for (long n = 0; n < o->n; ++n) {
    double t;
    t = Pr(o, o->f[EZ], n); r += o->c[HPHI][n] * t * t;
    t = PrT(o->f[HZ], n); r += o->c[EPHI][n] * t * t;
    l += o->f[HPHI][n] * Pz(o, o->f[ER], n) - o->f[HR][n] * Pz(o, o->f[EPHI], n);
  }
  return w - 0.5 * a * a * r + a * l;
}

/* Second-order charges of mode m (Sec. 4.5, the analogue of Eqs. (35) and
 * (34) for the scheme of Eq. (24)). The discrete divergence of the mode
 * annihilates the curl operators of (24): with the x-differences replaced by
 * m it is -P_r^T d_r - m d_phi - P_z^T d_z at a node (electric) and
 * m b_phi + P_r b_r + P_z b_z at a cell (magnetic), per radian. The split
 * scheme conserves it with the transverse fluxes averaged over the two time
 * levels and the z-fluxes corrected by the radial part of the splitting
 * operator only (the m-part stays in B^{e,r}, Sec. 4.3):
 *   qe = -P_r^T dr - m dphi - P_z^T dz~,  dr = M_er (er1 + er0)/2,
 *        dphi = M_ephi (ephi1 + ephi0)/2,
 *        dz~ = M_ez ez - alpha^2 P_r^T M_hphi^-1 P_r ez  (on non-PEC ez edges);
 *   qh = m bphi + P_r br + P_z bz~,  bphi = M_hphi (hphi1 + hphi0)/2,
 *        br = M_hr (hr1 + hr0)/2,
 *        bz~ = M_hz hz - alpha^2 P_r M_ephi^-1 P_r^T hz  (on non-PEC hz faces).
 * er1/ephi1 at time n+1 and er0/ephi0 at n with ez at n+1/2 (qe at
 * n+1/2); hphi1/hr1 at n+1/2 and hphi0/hr0 at n-1/2 with hz at n (qh at n).
 * q per node (electric) or per cell by its lower node (magnetic), canonical
 * r-fastest layout. */
static double PrT2(const rz_oracle_t *o, const double *v, long n) {
  return (n % o->mr > 0 ? v[n - 1] : 0.0) - v[n];
}
static double Pr2(const rz_oracle_t *o, const double *v, long n) {
  return (n % o->mr < o->nr ? v[n + 1] : 0.0) - v[n];
}
void rz_oracle_qbar_e(const rz_oracle_t *o, const double *er1, const double *er0, const double *ep1,
                      const double *ep0, const double *ez, double *q) {
  const long N = o->n;
  const double a2 = o->at * o->at, m = (double)o->m;
  double *dr = (double *)calloc((size_t)N, sizeof(double));
  double *dp = (double *)calloc((size_t)N, sizeof(double));
  double *dz = (double *)calloc((size_t)N, sizeof(double));
  double *t = (double *)calloc((size_t)N, sizeof(double));
  for (long n = 0; n < N; ++n) {
    if (o->c[ER][n] != 0.0) dr[n] = 0.5 * (er1[n] + er0[n]) / o->c[ER][n];
    if (o->c[EPHI][n] != 0.0) dp[n] = 0.5 * (ep1[n] + ep0[n]) / o->c[EPHI][n];
    t[n] = o->c[HPHI][n] * Pr2(o, ez, n);
  }
  for (long n = 0; n < N; ++n)
    if (o->c[EZ][n] != 0.0) dz[n] = ez[n] / o->c[EZ][n] - a2 * PrT2(o, t, n);
  for (long n = 0; n < N; ++n) q[n] = -PrT2(o, dr, n) - m * dp[n] - PzT(o, dz, n);
  free(dr); free(dp); free(dz); free(t);
}
void rz_oracle_qbar_h(const rz_oracle_t *o, const double *hp1, const double *hp0, const double *hr1,
                      const double *hr0, const double *hz, double *q) {
  const long N = o->n;
  const double a2 = o->at * o->at, m = (double)o->m;
  double *bp = (double *)calloc((size_t)N, sizeof(double));
  double *br = (double *)calloc((size_t)N, sizeof(double));
  double *bz = (double *)calloc((size_t)N, sizeof(double));
  double *t = (double *)calloc((size_t)N, sizeof(double));
  for (long n = 0; n < N; ++n) {
    if (o->c[HPHI][n] != 0.0) bp[n] = 0.5 * (hp1[n] + hp0[n]) / o->c[HPHI][n];
    if (o->c[HR][n] != 0.0) br[n] = 0.5 * (hr1[n] + hr0[n]) / o->c[HR][n];
    t[n] = o->c[EPHI][n] * PrT2(o, hz, n);
  }
  for (long n = 0; n < N; ++n)
    if (o->c[HZ][n] != 0.0) bz[n] = hz[n] / o->c[HZ][n] - a2 * Pr2(o, t, n);
  for (long n = 0; n < N; ++n) q[n] = m * bp[n] + Pr2(o, br, n) + Pz(o, bz, n);
  free(bp); free(br); free(bz); free(t);
}

void rz_oracle_get(const rz_oracle_t *o, int comp, double *out) {
  memcpy(out, o->f[comp], sizeof(double) * (size_t)o->n);
}
void rz_oracle_set(rz_oracle_t *o, int comp, const double *in) {
  for (long n = 0; n < o->n; ++n) o->f[comp][n] = (o->c[comp][n] != 0.0) ? in[n] : 0.0;
}
void rz_oracle_coef(const rz_oracle_t *o, int comp, double *out) {
  memcpy(out, o->c[comp], sizeof(double) * (size_t)o->n);
}
double rz_oracle_dt(const rz_oracle_t *o) { return o->dt; }
long rz_oracle_step_count(const rz_oracle_t *o) { return o->step; }

/* Stability bound of the rotationally symmetric scheme (Sec. 4.4): the time
 * step does not depend on the azimuthal mode number. */
int rz_oracle_stable(double dr, double dz, double cdt) {
  return cdt > 0 && cdt <= dz * (1.0 + 1e-12) && cdt <= dr * (1.0 + 1e-12);
}


/* Static start (the paper's structures sit between infinite ingoing and
 * outgoing pipes, Sec. 5): the bunch begins with its head at plane K inside a
 * uniform vacuum entry section carrying its discrete TEM field, which at
 * c*dt = dz moves one cell per step with the bunch (Sec. 4.5). It is the TEM
 * field of the Cartesian case with x -> phi, y -> r and P_x -> m:
 *   psi solves (P_r^T diag(r_{i+1/2}/dr) P_r + m^2 diag(dr/r_i)) psi = delta(i0)
 *   on the nodes whose e_z is not PEC (psi = 0 elsewhere),
 *   e_r = -P_r psi G(u), e_phi = -m psi G(u)                     (time n)
 *   h_phi = (r_{i+1/2}/(dr eta0)) P_r psi G(u+1),
 *   h_r = -(dr/(r_i eta0)) m psi G(u+1)                          (n - 1/2)
 * with u = k - n and G(u) + G(u+1) = 2 eta0 jj(u), jj the mode's line current,
 * G = 0 ahead of the head. */
int rz_oracle_set_bunch_static(rz_oracle_t *o, double sigma, double q, int i0, int k_head) {
  if (!o->vacuum || o->step != 0 || o->has_bunch) return -1;
  if (rz_oracle_set_bunch(o, sigma, q, i0) != 0) return -1;
  const int c0 = o->c0, K = k_head;
  const long mr = o->mr;
  if (K < 2 * c0 + 2 || K > o->nz) { o->has_bunch = 0; return -1; }
  for (int c = 0; c < 6; ++c)
    for (long k = 2; k <= K; ++k)
      for (long i = 0; i <= o->nr; ++i)
        if (o->c[c][i + mr * k] != o->c[c][i + mr]) { o->has_bunch = 0; return -1; }
  const int nn = o->nr + 1;
  const double dr = o->dr, m = (double)o->m;
  /* dense normal equations on the unknown nodes (a tridiagonal matrix,
   * solved by Gaussian elimination without pivoting: it is diagonally
   * dominant and symmetric positive definite) */
  int *unk = (int *)malloc(sizeof(int) * (size_t)nn);
  for (int i = 0; i < nn; ++i) unk[i] = o->c[EZ][i + mr] != 0.0;
  if (!unk[i0]) { free(unk); o->has_bunch = 0; return -1; }
  double *a = (double *)calloc((size_t)nn, sizeof(double));  /* sub-diagonal */
  double *b = (double *)calloc((size_t)nn, sizeof(double));  /* diagonal */
  double *cc = (double *)calloc((size_t)nn, sizeof(double)); /* super-diagonal */
  double *rhs = (double *)calloc((size_t)nn, sizeof(double));
  for (int i = 0; i < nn; ++i) {
    if (!unk[i]) { b[i] = 1.0; continue; }        /* psi = 0 */
    if (i + 1 < nn && o->c[ER][i + mr] != 0.0) {  /* e_r edge (i+1/2) */
      const double w = (i + 0.5) * dr / dr;
      b[i] += w;
      if (unk[i + 1]) cc[i] = -w;
    }
    if (i >= 1 && o->c[ER][i - 1 + mr] != 0.0) {  /* e_r edge (i-1/2) */
      const double w = (i - 0.5) * dr / dr;
      b[i] += w;
      if (unk[i - 1]) a[i] = -w;
    }
    if (i >= 1) b[i] += m * m * dr / (i * dr);
  }
  rhs[i0] = 1.0;
  for (int i = 1; i < nn; ++i) {                   /* forward elimination */
    const double f = a[i] / b[i - 1];
    b[i] -= f * cc[i - 1];
    rhs[i] -= f * rhs[i - 1];
  }
  double *psi = (double *)calloc((size_t)nn, sizeof(double));
  psi[nn - 1] = rhs[nn - 1] / b[nn - 1];
  for (int i = nn - 2; i >= 0; --i) psi[i] = (rhs[i] - cc[i] * psi[i + 1]) / b[i];
  for (int i = 0; i < nn; ++i) if (!unk[i]) psi[i] = 0.0;
  const double eta0 = RZ_MU0 * RZ_C0;
  double *G = (double *)calloc((size_t)(K + 3), sizeof(double));   /* G[u + 1] */
  for (long u = K - 1; u >= K - 2 * c0; --u) {
    const double jj = o->weight * RZ_C0 * o->qcell[u - K + 2 * c0] / o->dz;
    G[u + 1] = 2.0 * eta0 * jj - G[u + 2];
  }
  for (long k = 0; k <= o->nz; ++k)
    for (long i = 0; i <= o->nr; ++i) {
      const long n = i + mr * k;
      const double g0 = (k <= K) ? G[k + 1] : 0.0;
      const double g1 = (k + 1 <= K) ? G[k + 2] : 0.0;
      const double prp = (i < o->nr) ? psi[i + 1] - psi[i] : 0.0;
      const double rh = (i + 0.5) * dr, ri = i * dr;
      o->f[ER][n] = o->c[ER][n] != 0.0 ? -prp * g0 : 0.0;
      o->f[EPHI][n] = o->c[EPHI][n] != 0.0 ? -m * psi[i] * g0 : 0.0;
      o->f[EZ][n] = 0.0;
      o->f[HPHI][n] = o->c[HPHI][n] != 0.0 ? (rh / (dr * eta0)) * prp * g1 : 0.0;
      o->f[HR][n] = (o->c[HR][n] != 0.0 && i > 0) ? -(dr / (ri * eta0)) * m * psi[i] * g1 : 0.0;
      o->f[HZ][n] = 0.0;
    }
  o->kshift = K;
  free(unk); free(a); free(b); free(cc); free(rhs); free(psi); free(G);
  return 0;
}
