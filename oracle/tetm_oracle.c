/*
 * Plain FP64 CPU oracle of the explicit TE/TM scheme of Dohlus & Zagorodnov,
 * "Explicit TE/TM scheme for particle beam simulations" (Sec. 4.2, Eq. (23)).
 *
 * TEST INFRASTRUCTURE. This is the slow, obviously-correct reference the CUDA
 * path is checked against. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it; the product library never does, and
 * the two share no code, header, table or helper.
 *
 * Data model (Sec. 2, Eq. (4)): the FIT grid doublet on Nx x Ny x Nz primary
 * cells. Each field component is ONE vector over the canonical node index
 *     n = i + Mx*(j + My*k),   Mx = Nx+1, My = Ny+1, Mz = Nz+1,
 * x fastest, (Nx+1)(Ny+1)(Nz+1) entries. Entry n holds the integral quantity
 * of the grid object attached to node (i,j,k):
 *     ex (i+1/2, j, k)    ey (i, j+1/2, k)    ez (i, j, k+1/2)      [V]
 *     hx (i, j+1/2, k+1/2) hy (i+1/2, j, k+1/2) hz (i+1/2, j+1/2, k)  [A]
 * Objects outside the box ("phantom" entries) and PEC edges get a zero
 * material coefficient and stay zero.
 *
 * Topological operators (Sec. 2): (P_a v)[n] = v[n+s_a] - v[n] with
 * s_x = 1, s_y = Mx, s_z = Mx*My and v = 0 outside [0, N). P_a^T is the
 * matrix transpose: (P_a^T v)[n] = v[n-s_a] - v[n].
 *
 * Readings of the paper that this file fixes (each one also listed in the
 * design notes): the current enters every e-update with a minus sign (the
 * sign of Eq. (7), Eq. (15) and the energy law (19)); alpha = dt/2 in the
 * integral variables; staircase PEC and material averaging as described at
 * oracle_new(); Gaussian bunch truncated at +-5 sigma as described at
 * oracle_set_bunch().
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_C0 299792458.0
#define OR_EPS0 8.8541878128e-12
#define OR_MU0 (1.0 / (OR_EPS0 * OR_C0 * OR_C0))

typedef struct oracle {
  int nx, ny, nz;
  long mx, my, mz, n;   /* canonical extents and vector length */
  long sx, sy, sz;      /* index strides of P_x, P_y, P_z */
  double dx, dy, dz, dt, at; /* at = alpha = dt/2 */
  double *f[6];         /* ex ey ez hx hy hz */
  double *m[6];         /* diagonals of M_eps^-1 (ex,ey,ez) and M_mu^-1 (hx,hy,hz) */
  /* bunch (Sec. 5: rigid Gaussian, RMS sigma, moving along z at c) */
  int has_bunch, i0, j0, c0, m_min, m_max;
  double sigma, q;
  double *qcell;        /* Q_cell(d), d = -c0 .. c0-1 */
  double *wake;         /* W(s_m), m = m_min .. m_max */
  double *jz;           /* work array for the current of one step */
  long step;            /* n of the state y^n = (u^{n-1/2}, v^n) */
  long kshift;          /* bunch head at plane step + kshift (0: cold start at the wall) */
  int vacuum;           /* no material arrays were given */
  /* transverse wake on the observer line (io, jo): W_x on the x-edge line
   * (io+1/2, jo), W_y on the y-edge line (io, jo+1/2); longitudinal wakes on
   * the node lines (io, jo), (io+1, jo), (io, jo+1) */
  int io, jo;
  double *twx, *twy, *w00, *w10, *w01;
  double *exo, *eyo;    /* e_x, e_y of the observer column before a step */
} oracle_t;

enum { EX = 0, EY, EZ, HX, HY, HZ };

static long idx(const oracle_t *o, long i, long j, long k) { return i + o->mx * (j + o->my * k); }

/* (P_a v)[n] = v[n+s] - v[n] */
static double P(const oracle_t *o, const double *v, long n, long s) {
  return (n + s < o->n ? v[n + s] : 0.0) - v[n];
}
/* (P_a^T v)[n] = v[n-s] - v[n] */
static double PT(const double *v, long n, long s) { return (n - s >= 0 ? v[n - s] : 0.0) - v[n]; }

static int cell_pec(const oracle_t *o, const uint8_t *pec, long ci, long cj, long ck) {
  if (ci < 0 || cj < 0 || ck < 0 || ci >= o->nx || cj >= o->ny || ck >= o->nz) return 1;
  return pec ? pec[ci + o->nx * (cj + o->ny * ck)] != 0 : 0;
}
static double cell_val(const oracle_t *o, const double *a, long ci, long cj, long ck) {
  return a ? a[ci + o->nx * (cj + o->ny * ck)] : 1.0;
}

/* Edge coefficient M_eps^-1 = L_edge / (eps0 * mean(eps_r) * A_dual) over the
 * (up to) four cells sharing the edge; zero if any of them is PEC or outside
 * the box (staircase reading; the paper cites FIT [11] for this step). */
static double edge_coef(const oracle_t *o, const double *eps, const uint8_t *pec, long ca[4][3],
                        double len, double area) {
  double s = 0.0;
  for (int c = 0; c < 4; ++c) {
    if (cell_pec(o, pec, ca[c][0], ca[c][1], ca[c][2])) return 0.0;
    s += cell_val(o, eps, ca[c][0], ca[c][1], ca[c][2]);
  }
  return len / (OR_EPS0 * (s / 4.0) * area);
}
/* Face coefficient M_mu^-1 = L_dual / (mu0 * mu_bar * A_face), 1/mu_bar the
 * mean of 1/mu_r over the two cells sharing the face; zero unless both cells
 * are inside the box and not PEC. */
static double face_coef(const oracle_t *o, const double *mu, const uint8_t *pec, long ca[2][3],
                        double len, double area) {
  double s = 0.0;
  for (int c = 0; c < 2; ++c) {
    if (cell_pec(o, pec, ca[c][0], ca[c][1], ca[c][2])) return 0.0;
    s += 1.0 / cell_val(o, mu, ca[c][0], ca[c][1], ca[c][2]);
  }
  return len * (s / 2.0) / (OR_MU0 * area);
}

/* Build the grid, the diagonal material matrices (Sec. 2, Eq. (4)) and zero
 * fields. eps_r, mu_r, pec are per primary cell, index ci + nx*(cj + ny*ck);
 * NULL means vacuum / no interior PEC. cdt = c*dt in metres (0 -> dz). */
oracle_t *oracle_new(int nx, int ny, int nz, double dx, double dy, double dz, double cdt,
                     const double *eps_r, const double *mu_r, const uint8_t *pec) {
  if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0) || !(dz > 0) || cdt < 0) return NULL;
  oracle_t *o = (oracle_t *)calloc(1, sizeof(oracle_t));
  o->nx = nx; o->ny = ny; o->nz = nz;
  o->mx = nx + 1; o->my = ny + 1; o->mz = nz + 1;
  o->n = o->mx * o->my * o->mz;
  o->sx = 1; o->sy = o->mx; o->sz = o->mx * o->my;
  o->vacuum = (eps_r == NULL && mu_r == NULL);
  o->dx = dx; o->dy = dy; o->dz = dz;
  o->dt = (cdt > 0 ? cdt : dz) / OR_C0;
  o->at = 0.5 * o->dt;
  for (int c = 0; c < 6; ++c) {
    o->f[c] = (double *)calloc((size_t)o->n, sizeof(double));
    o->m[c] = (double *)calloc((size_t)o->n, sizeof(double));
  }
  o->jz = (double *)calloc((size_t)o->n, sizeof(double));
  for (long k = 0; k <= nz; ++k)
    for (long j = 0; j <= ny; ++j)
      for (long i = 0; i <= nx; ++i) {
        long n = idx(o, i, j, k);
        if (i < nx) { /* ex edge (i+1/2, j, k): cells (i, j-1..j, k-1..k) */
          long ca[4][3] = {{i, j - 1, k - 1}, {i, j, k - 1}, {i, j - 1, k}, {i, j, k}};
          o->m[EX][n] = edge_coef(o, eps_r, pec, ca, dx, dy * dz);
        }
        if (j < ny) { /* ey edge (i, j+1/2, k): cells (i-1..i, j, k-1..k) */
          long ca[4][3] = {{i - 1, j, k - 1}, {i, j, k - 1}, {i - 1, j, k}, {i, j, k}};
          o->m[EY][n] = edge_coef(o, eps_r, pec, ca, dy, dx * dz);
        }
        if (k < nz) { /* ez edge (i, j, k+1/2): cells (i-1..i, j-1..j, k) */
          long ca[4][3] = {{i - 1, j - 1, k}, {i, j - 1, k}, {i - 1, j, k}, {i, j, k}};
          o->m[EZ][n] = edge_coef(o, eps_r, pec, ca, dz, dx * dy);
        }
        if (j < ny && k < nz) { /* hx face x=i: cells (i-1..i, j, k) */
          long ca[2][3] = {{i - 1, j, k}, {i, j, k}};
          o->m[HX][n] = face_coef(o, mu_r, pec, ca, dx, dy * dz);
        }
        if (i < nx && k < nz) { /* hy face y=j: cells (i, j-1..j, k) */
          long ca[2][3] = {{i, j - 1, k}, {i, j, k}};
          o->m[HY][n] = face_coef(o, mu_r, pec, ca, dy, dx * dz);
        }
        if (i < nx && j < ny) { /* hz face z=k: cells (i, j, k-1..k) */
          long ca[2][3] = {{i, j, k - 1}, {i, j, k}};
          o->m[HZ][n] = face_coef(o, mu_r, pec, ca, dz, dx * dy);
        }
      }
  return o;
}

void oracle_free(oracle_t *o) {
  if (!o) return;
  for (int c = 0; c < 6; ++c) { free(o->f[c]); free(o->m[c]); }
  free(o->jz); free(o->qcell); free(o->wake);
  free(o->twx); free(o->twy); free(o->w00); free(o->w10); free(o->w01); free(o->exo); free(o->eyo);
  free(o);
}

/* Necessary and sufficient step bound of the explicit scheme in vacuum with a
 * staircase boundary, Eq. (25): c*dt <= dz and c*dt <= (dx^-2 + dy^-2)^-1/2. */
int oracle_stable(double dx, double dy, double dz, double cdt) {
  double lim_t = 1.0 / sqrt(1.0 / (dx * dx) + 1.0 / (dy * dy));
  return cdt <= dz * (1.0 + 1e-12) && cdt <= lim_t * (1.0 + 1e-12);
}

static double Phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

/* Rigid Gaussian bunch (Sec. 3 and Sec. 5): RMS length sigma, charge q, on the
 * z-line through node (i0, j0), moving at c. The line density is truncated to
 * |zeta| <= 5 sigma (not renormalised). At t = 0 its centre is at
 * z = -c0*dz, c0 = ceil(5 sigma/dz), so the head just touches the wall z = 0.
 * Q_cell(d) is the charge inside [d*dz, (d+1)*dz] of the bunch frame. */
int oracle_set_bunch(oracle_t *o, double sigma, double q, int i0, int j0) {
  if (!(sigma > 0) || q == 0 || i0 < 0 || j0 < 0 || i0 > o->nx || j0 > o->ny) return -1;
  o->has_bunch = 1;
  o->sigma = sigma; o->q = q; o->i0 = i0; o->j0 = j0;
  o->c0 = (int)ceil(5.0 * sigma / o->dz - 1e-12);
  o->m_min = -o->c0 - 1;
  o->m_max = (int)ceil(15.0 * sigma / o->dz - 1e-12);
  free(o->qcell); free(o->wake);
  o->qcell = (double *)calloc((size_t)(2 * o->c0), sizeof(double));
  const size_t nw = (size_t)(o->m_max - o->m_min + 1);
  o->wake = (double *)calloc(nw, sizeof(double));
  free(o->twx); free(o->twy); free(o->w00); free(o->w10); free(o->w01); free(o->exo); free(o->eyo);
  o->twx = (double *)calloc(nw, sizeof(double));
  o->twy = (double *)calloc(nw, sizeof(double));
  o->w00 = (double *)calloc(nw, sizeof(double));
  o->w10 = (double *)calloc(nw, sizeof(double));
  o->w01 = (double *)calloc(nw, sizeof(double));
  o->exo = (double *)calloc((size_t)o->mz, sizeof(double));
  o->eyo = (double *)calloc((size_t)o->mz, sizeof(double));
  o->io = i0 < o->nx ? i0 : o->nx - 1;
  o->jo = j0 < o->ny ? j0 : o->ny - 1;
  double lo = -5.0 * sigma, hi = 5.0 * sigma;
  for (int d = -o->c0; d < o->c0; ++d) {
    double a = d * o->dz, b = (d + 1) * o->dz;
    if (a < lo) a = lo;
    if (b > hi) b = hi;
    o->qcell[d + o->c0] = (b > a) ? q * (Phi(b / sigma) - Phi(a / sigma)) : 0.0;
  }
  return 0;
}

/* Line current of step n (integer time) on the ez edges (i0, j0, k+1/2):
 * jj_z = c * Q_cell(k - n + c0) / dz [A], the bunch charge of the edge's
 * length carried at c. Writes the full canonical ez-layout array. */
void oracle_current(const oracle_t *o, long n, double *jz) {
  memset(jz, 0, sizeof(double) * (size_t)o->n);
  if (!o->has_bunch) return;
  for (long k = 0; k < o->nz; ++k) {
    long d = k - (n + o->kshift) + o->c0;
    if (d < -o->c0 || d >= o->c0) continue;
    jz[idx(o, o->i0, o->j0, k)] = OR_C0 * o->qcell[d + o->c0] / o->dz;
  }
}

/* One step of the explicit scheme (23) in the detailed form of Sec. 4.2, in
 * the paper's order U1..U10; alpha = dt/2. jz is jj_z^n, jx and jy are
 * jj_{x,y}^{n+1/2}; each may be NULL (zero). The current is subtracted
 * (Ampere's law C^T h = dd/dt + j, Eq. (4)). */
void oracle_step_j(oracle_t *o, const double *jz, const double *jx, const double *jy) {
  double *ex = o->f[EX], *ey = o->f[EY], *ez = o->f[EZ];
  double *hx = o->f[HX], *hy = o->f[HY], *hz = o->f[HZ];
  const double *iex = o->m[EX], *iey = o->m[EY], *iez = o->m[EZ];
  const double *ihx = o->m[HX], *ihy = o->m[HY], *ihz = o->m[HZ];
  const double a = o->at;
  const long N = o->n, sx = o->sx, sy = o->sy, sz = o->sz;
  /* TM stage: u^{n-1/2} -> u^{n+1/2} */
  for (long n = 0; n < N; ++n) /* U1: auxiliary hx^n */
    hx[n] += a * ihx[n] * (P(o, ey, n, sz) - P(o, ez, n, sy));
  for (long n = 0; n < N; ++n) /* U2: auxiliary hy^n */
    hy[n] += a * ihy[n] * (-P(o, ex, n, sz) + P(o, ez, n, sx));
  for (long n = 0; n < N; ++n) /* U3: ez^{n+1/2} */
    ez[n] += 2.0 * a * iez[n] * (PT(hx, n, sy) - PT(hy, n, sx) - (jz ? jz[n] : 0.0));
  for (long n = 0; n < N; ++n) /* U4: hx^{n+1/2} */
    hx[n] += a * ihx[n] * (P(o, ey, n, sz) - P(o, ez, n, sy));
  for (long n = 0; n < N; ++n) /* U5: hy^{n+1/2} */
    hy[n] += a * ihy[n] * (-P(o, ex, n, sz) + P(o, ez, n, sx));
  /* TE stage: v^n -> v^{n+1} */
  for (long n = 0; n < N; ++n) /* U6: auxiliary ex^{n+1/2} */
    ex[n] += a * iex[n] * (PT(hy, n, sz) - PT(hz, n, sy) - (jx ? jx[n] : 0.0));
  for (long n = 0; n < N; ++n) /* U7: auxiliary ey^{n+1/2} */
    ey[n] += a * iey[n] * (-PT(hx, n, sz) + PT(hz, n, sx) - (jy ? jy[n] : 0.0));
  for (long n = 0; n < N; ++n) /* U8: hz^{n+1} */
    hz[n] += 2.0 * a * ihz[n] * (P(o, ex, n, sy) - P(o, ey, n, sx));
  for (long n = 0; n < N; ++n) /* U9: ex^{n+1} */
    ex[n] += a * iex[n] * (PT(hy, n, sz) - PT(hz, n, sy) - (jx ? jx[n] : 0.0));
  for (long n = 0; n < N; ++n) /* U10: ey^{n+1} */
    ey[n] += a * iey[n] * (-PT(hx, n, sz) + PT(hz, n, sx) - (jy ? jy[n] : 0.0));
}

/* Longitudinal wake (Sec. 5): W(s) = -(1/Q) * integral of E_z along the
 * path of a test charge a distance s behind the bunch centre. ez is already
 * the edge integral of E_z, and with c*dt = dz the path meets edge k+1/2
 * exactly at time n+1/2 with n = k + m + c0 (s = m*dz), so each step adds one
 * on-grid sample per window point. */
static void wake_gather(oracle_t *o, long n) {
  const double *ez = o->f[EZ];
  for (int m = o->m_min; m <= o->m_max; ++m) {
    long k = (n + o->kshift) - m - o->c0;
    if (k < 0 || k >= o->nz) continue;
    o->wake[m - o->m_min] -= ez[idx(o, o->i0, o->j0, k)] / o->q;
  }
}

/* Observer line of the transverse wake (before the first step). */
int oracle_set_observer(oracle_t *o, int io, int jo) {
  if (!o->has_bunch || o->step != 0 || io < 0 || jo < 0 || io >= o->nx || jo >= o->ny) return -1;
  o->io = io;
  o->jo = jo;
  return 0;
}

static void keep_observer_e(oracle_t *o) {
  for (long k = 0; k < o->mz; ++k) {
    o->exo[k] = o->f[EX][idx(o, o->io, o->jo, k)];
    o->eyo[k] = o->f[EY][idx(o, o->io, o->jo, k)];
  }
}

/* Transverse wake (Sec. 5): W_perp(s) = (1/Q) * integral of the Lorentz
 * force per charge (E + v x B)_perp on the test charge moving along +z at c,
 * i.e. E_x - c B_y and E_y + c B_x. On the x-edge line (io+1/2, jo) the path
 * meets e_x (edge length dx) at plane k at time n and h_y (dual edge length
 * dy) at k+1/2 at time n+1/2, with the same n = k + m + c0 as the
 * longitudinal wake; likewise e_y (dy) and h_x (dx) on the y-edge line
 * (io, jo+1/2). B = mu0 H. Also the longitudinal wakes of the three node
 * lines around the observer. e of time n was kept before the step. */
static void transverse_gather(oracle_t *o, long n) {
  const double eta0 = OR_MU0 * OR_C0;
  for (int m = o->m_min; m <= o->m_max; ++m) {
    long k = (n + o->kshift) - m - o->c0;
    if (k < 0 || k >= o->nz) continue;
    const long id = idx(o, o->io, o->jo, k);
    o->twx[m - o->m_min] += o->dz / o->q * (o->exo[k] / o->dx - eta0 * o->f[HY][id] / o->dy);
    o->twy[m - o->m_min] += o->dz / o->q * (o->eyo[k] / o->dy + eta0 * o->f[HX][id] / o->dx);
    o->w00[m - o->m_min] -= o->f[EZ][id] / o->q;
    o->w10[m - o->m_min] -= o->f[EZ][idx(o, o->io + 1, o->jo, k)] / o->q;
    o->w01[m - o->m_min] -= o->f[EZ][idx(o, o->io, o->jo + 1, k)] / o->q;
  }
}

/* Advance nsteps steps with the bunch current (if a bunch is set) and
 * accumulate the wakes. */
void oracle_step(oracle_t *o, int nsteps) {
  for (int s = 0; s < nsteps; ++s) {
    if (o->has_bunch) {
      oracle_current(o, o->step, o->jz);
      keep_observer_e(o);
    }
    oracle_step_j(o, o->has_bunch ? o->jz : NULL, NULL, NULL);
    if (o->has_bunch) {
      wake_gather(o, o->step);
      transverse_gather(o, o->step);
    }
    o->step += 1;
  }
}

/* Same as oracle_step_j but also counts the step and gathers the wakes. */
void oracle_step_custom(oracle_t *o, const double *jz, const double *jx, const double *jy) {
  if (o->has_bunch) keep_observer_e(o);
  oracle_step_j(o, jz, jx, jy);
  if (o->has_bunch) {
    wake_gather(o, o->step);
    transverse_gather(o, o->step);
  }
  o->step += 1;
}

/* which: 0 W_x, 1 W_y, 2..4 the longitudinal wakes at (io, jo), (io+1, jo),
 * (io, jo+1); same window as oracle_wake. */
int oracle_wake_extra(const oracle_t *o, int which, double *out, int cap) {
  if (!o->has_bunch || which < 0 || which > 4) return -1;
  int nw = o->m_max - o->m_min + 1;
  if (cap < nw) return -1;
  const double *src[5] = {o->twx, o->twy, o->w00, o->w10, o->w01};
  memcpy(out, src[which], sizeof(double) * (size_t)nw);
  return 0;
}

int oracle_wake(const oracle_t *o, double *out, int cap, int *n_out, double *s0, double *ds) {
  if (!o->has_bunch) return -1;
  int nw = o->m_max - o->m_min + 1;
  if (n_out) *n_out = nw;
  if (s0) *s0 = o->m_min * o->dz;
  if (ds) *ds = o->dz;
  if (out) {
    if (cap < nw) return -1;
    memcpy(out, o->wake, sizeof(double) * (size_t)nw);
  }
  return 0;
}

/* Discrete energy of the explicit scheme, Sec. 4.4: W^{n,e} = 1/2 <Q^e y, y>
 * with Q^e = B^e - alpha*A = [[I - alpha^2 R_0, alpha L], [alpha L^T,
 * I - alpha^2 R_1]] and y^n = (u^{n-1/2}, v^n), written out in the integral
 * variables (M_eps = 1/M_eps^-1 on non-PEC objects):
 *   1/2 sum M_eps e^2 + 1/2 sum M_mu h^2
 *   - alpha^2/2 [ sum M_mux^-1 (P_y ez)^2 + sum M_muy^-1 (P_x ez)^2
 *               + sum M_epsx^-1 (P_y^T hz)^2 + sum M_epsy^-1 (P_x^T hz)^2 ]
 *   + alpha [ hx . P_z ey - hy . P_z ex ]. */
double oracle_energy(const oracle_t *o) {
  const double a = o->at;
  double w = 0.0;
  for (int c = 0; c < 6; ++c)
    for (long n = 0; n < o->n; ++n)
      if (o->m[c][n] != 0.0) w += 0.5 * o->f[c][n] * o->f[c][n] / o->m[c][n];
  double r = 0.0, l = 0.0;
  for (long n = 0; n < o->n; ++n) {
    double t;
    t = P(o, o->f[EZ], n, o->sy); r += o->m[HX][n] * t * t;
    t = P(o, o->f[EZ], n, o->sx); r += o->m[HY][n] * t * t;
    t = PT(o->f[HZ], n, o->sy); r += o->m[EX][n] * t * t;
    t = PT(o->f[HZ], n, o->sx); r += o->m[EY][n] * t * t;
    l += o->f[HX][n] * P(o, o->f[EY], n, o->sz) - o->f[HY][n] * P(o, o->f[EX], n, o->sz);
  }
  return w - 0.5 * a * a * r + a * l;
}

/* Second-order electric node charge of Eq. (35), in the integral variables:
 *   qe = -P_x^T dx - P_y^T dy - P_z^T dz~,
 *   dx = M_epsx (ex1 + ex0)/2,  dy = M_epsy (ey1 + ey0)/2,
 *   dz~ = M_epsz ez - alpha^2 (P_y^T M_mux^-1 P_y + P_x^T M_muy^-1 P_x) ez
 * on non-PEC ez edges (zero elsewhere): the (I - alpha^2 r_0) factor acts on
 * the ez vector before the z-divergence. ex1/ey1 at n+1, ex0/ey0 at n, ez at
 * n+1/2. q has the canonical node layout. */
void oracle_qbar_e(const oracle_t *o, const double *ex1, const double *ex0, const double *ey1,
                   const double *ey0, const double *ez, double *q) {
  const long N = o->n;
  const double a2 = o->at * o->at;
  double *dx = (double *)calloc((size_t)N, sizeof(double));
  double *dy = (double *)calloc((size_t)N, sizeof(double));
  double *dz = (double *)calloc((size_t)N, sizeof(double));
  double *t1 = (double *)calloc((size_t)N, sizeof(double));
  double *t2 = (double *)calloc((size_t)N, sizeof(double));
  for (long n = 0; n < N; ++n) {
    if (o->m[EX][n] != 0.0) dx[n] = 0.5 * (ex1[n] + ex0[n]) / o->m[EX][n];
    if (o->m[EY][n] != 0.0) dy[n] = 0.5 * (ey1[n] + ey0[n]) / o->m[EY][n];
    t1[n] = o->m[HX][n] * P(o, ez, n, o->sy);
    t2[n] = o->m[HY][n] * P(o, ez, n, o->sx);
  }
  for (long n = 0; n < N; ++n)
    if (o->m[EZ][n] != 0.0)
      dz[n] = ez[n] / o->m[EZ][n] - a2 * (PT(t1, n, o->sy) + PT(t2, n, o->sx));
  for (long n = 0; n < N; ++n)
    q[n] = -PT(dx, n, o->sx) - PT(dy, n, o->sy) - PT(dz, n, o->sz);
  free(dx); free(dy); free(dz); free(t1); free(t2);
}

/* Second-order magnetic cell charge of Eq. (34):
 *   qh = P_x bx + P_y by + P_z bz~,
 *   bx = M_mux (hx1 + hx0)/2,  by = M_muy (hy1 + hy0)/2,
 *   bz~ = M_muz hz - alpha^2 (P_y M_epsx^-1 P_y^T + P_x M_epsy^-1 P_x^T) hz
 * on non-PEC hz faces. hx1/hy1 at n+1/2, hx0/hy0 at n-1/2, hz at n. q is
 * indexed by the cell's lower node (canonical layout). */
void oracle_qbar_h(const oracle_t *o, const double *hx1, const double *hx0, const double *hy1,
                   const double *hy0, const double *hz, double *q) {
  const long N = o->n;
  const double a2 = o->at * o->at;
  double *bx = (double *)calloc((size_t)N, sizeof(double));
  double *by = (double *)calloc((size_t)N, sizeof(double));
  double *bz = (double *)calloc((size_t)N, sizeof(double));
  double *t1 = (double *)calloc((size_t)N, sizeof(double));
  double *t2 = (double *)calloc((size_t)N, sizeof(double));
  for (long n = 0; n < N; ++n) {
    if (o->m[HX][n] != 0.0) bx[n] = 0.5 * (hx1[n] + hx0[n]) / o->m[HX][n];
    if (o->m[HY][n] != 0.0) by[n] = 0.5 * (hy1[n] + hy0[n]) / o->m[HY][n];
    t1[n] = o->m[EX][n] * PT(hz, n, o->sy);
    t2[n] = o->m[EY][n] * PT(hz, n, o->sx);
  }
  for (long n = 0; n < N; ++n)
    if (o->m[HZ][n] != 0.0)
      bz[n] = hz[n] / o->m[HZ][n] - a2 * (P(o, t1, n, o->sy) + P(o, t2, n, o->sx));
  for (long n = 0; n < N; ++n)
    q[n] = P(o, bx, n, o->sx) + P(o, by, n, o->sy) + P(o, bz, n, o->sz);
  free(bx); free(by); free(bz); free(t1); free(t2);
}

/* Field / coefficient access. set() zeroes entries whose coefficient is zero
 * (PEC edges, faces next to PEC, phantom objects): they carry no field. */
void oracle_get(const oracle_t *o, int comp, double *out) {
  memcpy(out, o->f[comp], sizeof(double) * (size_t)o->n);
}
void oracle_set(oracle_t *o, int comp, const double *in) {
  for (long n = 0; n < o->n; ++n) o->f[comp][n] = (o->m[comp][n] != 0.0) ? in[n] : 0.0;
}
void oracle_coef(const oracle_t *o, int comp, double *out) {
  memcpy(out, o->m[comp], sizeof(double) * (size_t)o->n);
}
/* Yee's E/M leapfrog (Sec. 3, Eq. (7)) on the same grid doublet and material
 * matrices: the scheme the paper measures the TE/TM scheme against. The state
 * is (e^{n-1/2}, h^n) and one step is
 *     e^{n+1/2} = e^{n-1/2} + dt M_eps^-1 C~ h^n,
 *     h^{n+1}   = h^n - dt M_mu^-1 C e^{n+1/2},
 * C the curl of the primary grid, C~ = C^T that of the dual grid. Written in
 * components with the P operators above (the same difference terms as the TE/TM
 * updates, each with the full step dt). Source-free: it serves the field-only
 * comparison (dispersion (9), stability (8), cost per step), so it refuses a
 * solve that carries a bunch. */
int oracle_yee_step(oracle_t *o, int nsteps) {
  if (o->has_bunch) return -1;
  double *ex = o->f[EX], *ey = o->f[EY], *ez = o->f[EZ];
  double *hx = o->f[HX], *hy = o->f[HY], *hz = o->f[HZ];
  const double *iex = o->m[EX], *iey = o->m[EY], *iez = o->m[EZ];
  const double *ihx = o->m[HX], *ihy = o->m[HY], *ihz = o->m[HZ];
  const double dt = o->dt;
  const long N = o->n, sx = o->sx, sy = o->sy, sz = o->sz;
  for (int s = 0; s < nsteps; ++s) {
    /* electric half: e^{n-1/2} -> e^{n+1/2} from h^n */
    for (long n = 0; n < N; ++n) {
      ex[n] += dt * iex[n] * (PT(hy, n, sz) - PT(hz, n, sy));
      ey[n] += dt * iey[n] * (-PT(hx, n, sz) + PT(hz, n, sx));
      ez[n] += dt * iez[n] * (PT(hx, n, sy) - PT(hy, n, sx));
    }
    /* magnetic half: h^n -> h^{n+1} from e^{n+1/2} */
    for (long n = 0; n < N; ++n) {
      hx[n] += dt * ihx[n] * (P(o, ey, n, sz) - P(o, ez, n, sy));
      hy[n] += dt * ihy[n] * (-P(o, ex, n, sz) + P(o, ez, n, sx));
      hz[n] += dt * ihz[n] * (P(o, ex, n, sy) - P(o, ey, n, sx));
    }
    o->step += 1;
  }
  return 0;
}

/* Step bound of Yee's scheme in vacuum, Eq. (8):
 * c*dt <= (dx^-2 + dy^-2 + dz^-2)^-1/2. */
int oracle_yee_stable(double dx, double dy, double dz, double cdt) {
  return cdt <= (1.0 + 1e-12) / sqrt(1.0 / (dx * dx) + 1.0 / (dy * dy) + 1.0 / (dz * dz));
}

long oracle_step_count(const oracle_t *o) { return o->step; }
double oracle_dt(const oracle_t *o) { return o->dt; }
int oracle_bunch_info(const oracle_t *o, int *c0, int *m_min, int *m_max, double *qcell) {
  if (!o->has_bunch) return -1;
  *c0 = o->c0; *m_min = o->m_min; *m_max = o->m_max;
  if (qcell) memcpy(qcell, o->qcell, sizeof(double) * (size_t)(2 * o->c0));
  return 0;
}


/* ------------------------------------------------------------------------
 * Static start: the bunch begins inside a uniform entry pipe carrying its own
 * discrete TEM field, as if it had come from an infinite ingoing pipe (the
 * paper's examples, Sec. 5). At c*dt = dz such a field moves exactly one
 * cell per step with the bunch (zero z-dispersion, Sec. 4.5), so nothing is
 * radiated until the bunch meets a change of cross-section.
 *
 * Transverse part: the potential phi on the nodes of the entry cross-section
 * solves (dy/dx P_x^T P_x + dx/dy P_y^T P_y) phi = delta(i0, j0) over the
 * non-PEC edges, phi = 0 on every node that touches a PEC cell or the wall.
 * Longitudinal part: with the head at plane K at step 0, the line current of
 * step n on edge k is jj(u) = c Q_cell(u - K + c0)/dz with u = k - n; a TEM
 * field ex = -P_x phi G(u), ey = -P_y phi G(u) at time n and
 * hx = (dx/dy) P_y phi G(u+1)/eta0, hy = -(dy/dx) P_x phi G(u+1)/eta0 at
 * n - 1/2 carries the current (G(u) + G(u+1))/(2 eta0), so
 * G(u) + G(u+1) = 2 eta0 jj(u), G = 0 ahead of the head. (The alternating
 * remainder behind the tail is the alternating sum of the symmetric
 * Q_cell, which vanishes.)
 * ---------------------------------------------------------------------- */

/* plain conjugate gradients on the unknown nodes of one cross-section */
static void cg_solve(int n, const long *ex_a, const long *ex_b, const double *ex_w, long nex,
                     const long *node_of, const double *rhs, double *x) {
  double *r = (double *)calloc((size_t)n, sizeof(double));
  double *p = (double *)calloc((size_t)n, sizeof(double));
  double *ap = (double *)calloc((size_t)n, sizeof(double));
  (void)node_of;
  for (int q = 0; q < n; ++q) { x[q] = 0.0; r[q] = rhs[q]; p[q] = rhs[q]; }
  double rr = 0.0, bb = 0.0;
  for (int q = 0; q < n; ++q) { rr += r[q] * r[q]; bb += rhs[q] * rhs[q]; }
  for (int it = 0; it < 20 * n + 100 && rr > 1e-30 * bb; ++it) {
    for (int q = 0; q < n; ++q) ap[q] = 0.0;
    for (long e = 0; e < nex; ++e) {       /* each edge couples nodes a, b (-1: on the wall) */
      const long a = ex_a[e], b = ex_b[e];
      const double pa = a >= 0 ? p[a] : 0.0, pb = b >= 0 ? p[b] : 0.0;
      if (a >= 0) ap[a] += ex_w[e] * (pa - pb);
      if (b >= 0) ap[b] += ex_w[e] * (pb - pa);
    }
    double pap = 0.0;
    for (int q = 0; q < n; ++q) pap += p[q] * ap[q];
    const double alpha = rr / pap;
    double rr2 = 0.0;
    for (int q = 0; q < n; ++q) {
      x[q] += alpha * p[q];
      r[q] -= alpha * ap[q];
      rr2 += r[q] * r[q];
    }
    const double beta = rr2 / rr;
    for (int q = 0; q < n; ++q) p[q] = r[q] + beta * p[q];
    rr = rr2;
  }
  free(r); free(p); free(ap);
}

int oracle_set_bunch_static(oracle_t *o, double sigma, double q, int i0, int j0, int k_head) {
  if (!o->vacuum || o->step != 0 || o->has_bunch) return -1;
  if (oracle_set_bunch(o, sigma, q, i0, j0) != 0) return -1;
  const int c0 = o->c0, K = k_head;
  if (K < 2 * c0 + 2 || K > o->nz) { o->has_bunch = 0; return -1; }
  /* the entry section: planes 1..K carry the same objects as plane 1 */
  for (int c = 0; c < 6; ++c)
    for (long k = 2; k <= K; ++k)
      for (long j = 0; j <= o->ny; ++j)
        for (long i = 0; i <= o->nx; ++i)
          if (o->m[c][idx(o, i, j, k)] != o->m[c][idx(o, i, j, 1)]) { o->has_bunch = 0; return -1; }
  /* unknown nodes: those whose ez edge in plane 1 is non-PEC (all four cells) */
  const long nn = o->mx * o->my;
  long *node_of = (long *)malloc(sizeof(long) * (size_t)nn);
  int n_unk = 0;
  for (long j = 0; j <= o->ny; ++j)
    for (long i = 0; i <= o->nx; ++i)
      node_of[i + o->mx * j] = o->m[EZ][idx(o, i, j, 1)] != 0.0 ? n_unk++ : -1;
  if (node_of[i0 + o->mx * j0] < 0 || n_unk == 0) { free(node_of); o->has_bunch = 0; return -1; }
  /* non-PEC transverse edges of the section with their weights */
  long cap = 2 * nn, nex = 0;
  long *ea = (long *)malloc(sizeof(long) * (size_t)cap);
  long *eb = (long *)malloc(sizeof(long) * (size_t)cap);
  double *ew = (double *)malloc(sizeof(double) * (size_t)cap);
  for (long j = 0; j <= o->ny; ++j)
    for (long i = 0; i <= o->nx; ++i) {
      if (i < o->nx && o->m[EX][idx(o, i, j, 1)] != 0.0) {
        ea[nex] = node_of[i + o->mx * j]; eb[nex] = node_of[i + 1 + o->mx * j];
        ew[nex++] = o->dy / o->dx;
      }
      if (j < o->ny && o->m[EY][idx(o, i, j, 1)] != 0.0) {
        ea[nex] = node_of[i + o->mx * j]; eb[nex] = node_of[i + o->mx * (j + 1)];
        ew[nex++] = o->dx / o->dy;
      }
    }
  double *rhs = (double *)calloc((size_t)n_unk, sizeof(double));
  double *x = (double *)calloc((size_t)n_unk, sizeof(double));
  rhs[node_of[i0 + o->mx * j0]] = 1.0;
  cg_solve(n_unk, ea, eb, ew, nex, node_of, rhs, x);
  double *phi = (double *)calloc((size_t)nn, sizeof(double));
  for (long t = 0; t < nn; ++t) phi[t] = node_of[t] >= 0 ? x[node_of[t]] : 0.0;
  /* longitudinal profile G(u), u = -1 .. K (G = 0 elsewhere) */
  const double eta0 = OR_MU0 * OR_C0;
  double *G = (double *)calloc((size_t)(K + 3), sizeof(double));   /* G[u + 1] */
  for (long u = K - 1; u >= K - 2 * c0; --u) {
    const double jj = OR_C0 * o->qcell[u - K + 2 * c0] / o->dz;
    G[u + 1] = 2.0 * eta0 * jj - G[u + 2];
  }
  for (long k = 0; k <= o->nz; ++k)
    for (long j = 0; j <= o->ny; ++j)
      for (long i = 0; i <= o->nx; ++i) {
        const long n = idx(o, i, j, k);
        const double g0 = (k <= K) ? G[k + 1] : 0.0;
        const double g1 = (k + 1 <= K) ? G[k + 2] : 0.0;
        const double pxp = (i < o->nx) ? phi[i + 1 + o->mx * j] - phi[i + o->mx * j] : 0.0;
        const double pyp = (j < o->ny) ? phi[i + o->mx * (j + 1)] - phi[i + o->mx * j] : 0.0;
        o->f[EX][n] = o->m[EX][n] != 0.0 ? -pxp * g0 : 0.0;
        o->f[EY][n] = o->m[EY][n] != 0.0 ? -pyp * g0 : 0.0;
        o->f[EZ][n] = 0.0;
        o->f[HX][n] = o->m[HX][n] != 0.0 ? (o->dx / o->dy) * pyp * g1 / eta0 : 0.0;
        o->f[HY][n] = o->m[HY][n] != 0.0 ? -(o->dy / o->dx) * pxp * g1 / eta0 : 0.0;
        o->f[HZ][n] = 0.0;
      }
  o->kshift = K;
  free(node_of); free(ea); free(eb); free(ew); free(rhs); free(x); free(phi); free(G);
  return 0;
}

long oracle_kshift(const oracle_t *o) { return o->kshift; }
