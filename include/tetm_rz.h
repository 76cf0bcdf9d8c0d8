/*
 * tetm_rz.h — C ABI of the rotationally symmetric solver in libtetm.so: the
 * explicit TE/TM scheme for bodies of revolution (Sec. 4.3, Eq. (24)), one
 * set of azimuthal modes m_lo..m_hi advanced together on one (r, z) grid,
 * with a rigid relativistic Gaussian bunch on a ring and the longitudinal
 * wake potential of every mode gathered along the bunch path (Sec. 5).
 *
 * Conventions are those of tetm.h (return codes, ownership, streams); in
 * addition:
 *  - Grid: nr x nz primary cells in (r, z); nodes r_i = i*dr (i = 0..nr, the
 *    axis is i = 0), z_k = k*dz. Perfectly conducting wall at r = nr*dr and
 *    at both z ends; cold start. Cell (ci, ck) has the index ci + nr*ck.
 *  - Fields of mode m: e_r, e_z, h_phi ~ cos(m phi) and e_phi, h_r, h_z ~
 *    sin(m phi), integral quantities per radian of azimuth. Canonical layout:
 *    one float64 vector per component with (nr+1)*(nz+1) entries, entry
 *    i + (nr+1)*k attached to node (i, k):
 *      e_r (i+1/2, k)   e_phi (i, k)   e_z (i, k+1/2)
 *      h_r (i, k+1/2)   h_phi (i+1/2, k+1/2)   h_z (i+1/2, k)
 *    Entries on PEC edges, on faces next to PEC, e_phi and h_r on the axis
 *    and e_z on the axis for m >= 1 are zero.
 *  - Metric (per radian, staircase): the cylindrical FIT lengths and areas;
 *    the axis e_z (m = 0) has the dual area dr^2/4, which keeps the bound of
 *    Sec. 4.4 (c*dt <= min(dr, dz) for every m).
 *  - Time: the state after n steps is y^n = (u^{n-1/2}, v^n) with
 *    u = (h_phi, h_r, e_z), v = (e_phi, e_r, h_z).
 */
#ifndef TETM_RZ_H
#define TETM_RZ_H

#include "tetm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define TETM_RZ_ER 0
#define TETM_RZ_EPHI 1
#define TETM_RZ_EZ 2
#define TETM_RZ_HR 3
#define TETM_RZ_HPHI 4
#define TETM_RZ_HZ 5

#define TETM_RZ_MAX_MODES 64
/* Polls of an mbarrier after which the bulk-copy step kernels give up on a
 * copy, raise the error word and drain (tetm_rz_sync then reports
 * TETM_E_TIMEOUT); a poll suspends for a few microseconds, so the limit is
 * about one second. */
#define TETM_RZ_MAX_POLLS (1 << 18)

/* step kernels (same results bit for bit; they differ in how loads run ahead
 * and in how many steps one pass over the fields takes) */
#define TETM_RZ_KERNEL_ASYNC 0     /* asynchronous copies into a shared-memory ring (default) */
#define TETM_RZ_KERNEL_REGISTER 1  /* a register ring of planes                               */
#define TETM_RZ_KERNEL_BULK 2      /* one bulk (TMA) copy per plane and work item into a
                                      shared-memory ring, mbarrier completion               */
#define TETM_RZ_KERNEL_BULK2 3     /* the bulk-copy sweep advancing two time steps per pass
                                      (temporal blocking: y^n read and y^{n+2} written once;
                                      an odd remaining step runs one-step)                  */

typedef struct tetm_rz_grid {
  int32_t nr, nz;      /* primary cells, each >= 2                                 */
  int32_t m_lo, m_hi;  /* azimuthal modes m_lo..m_hi, 0 <= m_lo <= m_hi,
                          at most TETM_RZ_MAX_MODES of them                        */
  int32_t precision;   /* TETM_FP64 or TETM_FP32                                    */
  int32_t pad;
  double dr, dz;       /* cell sizes [m], > 0                                       */
  double cdt;          /* c*dt [m]; 0 selects min(dr, dz)                           */
} tetm_rz_grid;

typedef struct tetm_rz_info {
  int64_t step;             /* n of the current state                          */
  int64_t device_bytes;     /* device memory held by the solve                 */
  int64_t processed_cells;  /* entries one step updates, summed over the modes */
  int32_t n_modes;
  int32_t chunk_z;          /* planes per work item                            */
  int32_t work_items;       /* (mode, radial tile, z chunk) items per step      */
  int32_t wake_len;         /* samples of each mode's wake, 0 without a bunch  */
  int32_t resident_warps;   /* step-kernel warps resident on the device at once */
  int32_t kernel;           /* TETM_RZ_KERNEL_*                                 */
} tetm_rz_info;

typedef struct tetm_rz tetm_rz;

/* Creates a solve (Sec. 4.3). pec: uint8 per cell (1 = PEC), nr*nz entries
 * (cell ci + nr*ck), or NULL for the empty pipe of radius nr*dr. eps_r, mu_r:
 * float64 per cell (>= 1, finite, else TETM_E_ARG) or NULL (vacuum). With
 * material arrays the per-radian material matrices are the column's metric
 * over the staircase mean of eps_r of the cells an edge touches (e_r, e_z:
 * two, e_phi: four, the axis e_z: one) and times the mean of 1/mu_r of the
 * cells a face touches (h_phi: one, h_r, h_z: two); the coefficients are then
 * per entry and plane (about (8 esz + 48) bytes per entry and mode more
 * device memory than tetm_rz_bytes_needed counts), the step runs the
 * register kernel (tetm_rz_set_kernel of another: TETM_E_UNSUPPORTED) and
 * the static starts answer TETM_E_UNSUPPORTED (their entry section is
 * vacuum). Fails with TETM_E_UNSTABLE when c*dt > min(dr, dz) (Sec. 4.4).
 * Synchronizes. */
int tetm_rz_create(const tetm_rz_grid* g, const double* eps_r, const double* mu_r,
                   const uint8_t* pec, tetm_rz** out);

/* Rigid Gaussian bunch of RMS length sigma [m] and charge q [C] on the ring
 * r = i0*dr (Sec. 5), truncated at +-5 sigma, head at z = 0 at t = 0, moving
 * at c along +z. Mode m receives the share (2 - delta_m0)/(2 pi) per radian.
 * i0 = 0 (the axis) only when m_hi = 0. Requires c*dt == dz
 * (TETM_E_NOT_MAGIC) and step 0 (TETM_E_STATE). The wake window of every mode
 * is s = m*dz, m = -c0-1 .. ceil(15 sigma/dz), c0 = ceil(5 sigma/dz). */
int tetm_rz_set_bunch(tetm_rz* s, double sigma, double q, int32_t i0);

/* Static start (Sec. 5: the paper's structures sit between infinite
 * ingoing and outgoing pipes): the bunch of tetm_rz_set_bunch (same sigma,
 * q, i0, profile and wake window) begins with its head at plane k_head,
 * carrying the discrete TEM field of every mode, so it crosses the uniform
 * entry section without radiating (the field moves one cell per step at
 * c*dt = dz, Sec. 4.5). Per mode m the radial potential solves
 * (P_r^T diag(r_{i+1/2}/dr) P_r + m^2 diag(dr/r_i)) psi = delta(i0) on the
 * nodes whose e_z is not PEC. Current and wakes then refer to step + k_head.
 * Requires step 0 and no bunch (TETM_E_STATE), c*dt == dz
 * (TETM_E_NOT_MAGIC), 2*c0 + 2 <= k_head <= nz, planes 1..k_head carrying
 * the same objects, i0 as for tetm_rz_set_bunch (TETM_E_ARG). Writes planes
 * 0..k_head+1 of every mode. Synchronizes. */
int tetm_rz_set_bunch_static(tetm_rz* s, double sigma, double q, int32_t i0, int32_t k_head);

/* Scattered-field form of the static start: the same solve as
 * tetm_rz_set_bunch_static (same arguments, the same fields, wakes and energy
 * in exact arithmetic), but the field kept on the device is the total minus
 * the incident field, the static start's TEM field moving one plane per step
 * through a continuation of the entry section. Each step first evaluates, in
 * the field precision, the incident field's mismatch with the geometry (one
 * step of (24) applied to it, bunch current included, minus its next
 * position: an exact zero wherever the geometry is the entry section) on the
 * 2*c0 + 3 planes around the bunch and adds it to the new field; the step
 * kernels deposit no current. The stored field thus carries no near field of
 * the bunch, which keeps float32 wakes accurate for every mode.
 * tetm_rz_get_fields, tetm_rz_set_fields and tetm_rz_energy take and return
 * the total field. Extra requirement: every object of the entry section
 * (plane 1) is present on planes 1..nz-1 (TETM_E_ARG otherwise). Device
 * memory: eight source windows of 2*c0 + 3 planes of all modes (the sources
 * of eight steps are computed per launch). Synchronizes. */
int tetm_rz_set_bunch_scattered(tetm_rz* s, double sigma, double q, int32_t i0, int32_t k_head);

/* Failure-detection self-test (no solve needed): one warp waits, with the
 * bulk-copy kernels' bounded poll loop, on an mbarrier that nothing ever
 * completes; after polls polls (1 .. 2^26, else TETM_E_ARG) it raises a
 * device error word, which this call reads: TETM_E_TIMEOUT is the expected
 * result, and the context stays usable. Synchronizes (default stream). */
int tetm_rz_selftest_wait(int32_t polls);

/* Queues n steps of Eq. (24) for every mode (n >= 0). */
int tetm_rz_step(tetm_rz* s, int64_t n);

/* Waits for the solve's stream. Returns TETM_E_TIMEOUT when a bounded
 * device-side wait of the bulk-copy kernel gave up since the solve was
 * created (the state is then not advanced correctly). */
int tetm_rz_sync(tetm_rz* s);

/* Wake potential of mode m_lo + mode [V/C], W(s) = -(1/q) * sum of e_z at the
 * bunch ring over the passage, as float64 (cap entries at out). n_out, s0
 * (first sample's s [m]) and ds may be NULL. out == NULL returns the length
 * only. Synchronizes. */
int tetm_rz_wake(tetm_rz* s, int32_t mode, double* out, int32_t cap, int32_t* n_out,
                 double* s0, double* ds);

/* Radius of the transverse wake: r_{obs+1/2} = (obs + 1/2) dr, 0 <= obs <
 * nr - 1 (default: the bunch ring i0, or nr - 2 if i0 = nr - 1). After
 * tetm_rz_set_bunch, before the first step (TETM_E_STATE otherwise). */
int tetm_rz_set_observer(tetm_rz* s, int32_t obs);

/* Radial transverse wake of mode m_lo + mode at r_{obs+1/2}, phi = 0 [V/C]
 * (Sec. 5, the dipole wake for m = 1): W_r(s) = (1/q) * sum over the passage
 * of (E_r - c mu0 H_phi) dz along the path s behind the bunch centre, with
 * E_r from e_r at time n and H_phi from h_phi at time n+1/2 (the same path
 * point at c*dt = dz), float64, same samples as tetm_rz_wake. The scheme
 * satisfies the discrete Panofsky-Wenzel relation
 * W_r(m+1) - W_r(m) = dz/dr * mean over m, m+1 of (W_{obs+1} - W_obs)
 * with the longitudinal wakes at rings obs, obs+1. Synchronizes. */
int tetm_rz_transverse_wake(tetm_rz* s, int32_t mode, double* out, int32_t cap, int32_t* n_out,
                            double* s0, double* ds);

/* Discrete energy per radian of mode m_lo + mode, 0.5 <Q^{e,r} y, y>
 * (Sec. 4.4), reduced in float64 on the device. Synchronizes. */
int tetm_rz_energy(tetm_rz* s, int32_t mode, double* w);

/* Copy one component of one mode to / from a host float64 array in the
 * canonical layout ((nr+1)*(nz+1) entries). Writes zero inactive entries.
 * Synchronize. */
int tetm_rz_get_fields(tetm_rz* s, int32_t mode, int32_t comp, double* out);
int tetm_rz_set_fields(tetm_rz* s, int32_t mode, int32_t comp, const double* in);

/* Planes per work item (>= 4); rebuilds the work list. */
int tetm_rz_set_tiling(tetm_rz* s, int32_t chunk_z);

/* Selects the step kernel (TETM_RZ_KERNEL_*). */
int tetm_rz_set_kernel(tetm_rz* s, int32_t kernel);

/* Queue on this CUDA stream (NULL: the solve's own stream). */
int tetm_rz_set_stream(tetm_rz* s, void* cuda_stream);

int tetm_rz_get_info(tetm_rz* s, tetm_rz_info* info);

/* Canary of out-of-place writes: counts, over both field sets and every mode,
 * the entries that hold a non-zero value although their activity bit is clear
 * (the zero guard rows and columns, PEC objects). A correct run reports 0.
 * Synchronizes; TETM_E_ARG for NULL arguments. */
int tetm_rz_check_guards(tetm_rz* s, int64_t* violations);

/* Charges of mode m_lo + mode in the discrete charge laws of Sec. 4.5 for
 * scheme (24) (per radian; the x-differences of Eqs. (35), (34) become the
 * multiplication by m): the node charge -P_r^T d_r - m d_phi - P_z^T d_z~
 * with d_r, d_phi averaged over the last two states and d_z~ = M_ez e_z -
 * alpha^2 P_r^T M_hphi^-1 P_r e_z (the m-part of the splitting operator stays
 * in B^{e,r}, Sec. 4.3), against the bunch's share (2 - delta_m0)/(2 pi) of
 * its node charges on the bunch ring; the cell charge m b_phi + P_r b_r +
 * P_z b_z~ with b_z~ = M_hz h_z - alpha^2 P_r M_ephi^-1 P_r^T h_z of the
 * previous state. *max_e = max |qe - qbunch| over nodes whose every edge
 * carries a field, *max_h = max |qh| over such cells, *q_scale = the bunch
 * share's largest node charge (0 without bunch); float64 on the device, on
 * the total field in the scattered-field form. Needs the state one step
 * before the current one (TETM_E_STATE after tetm_rz_set_fields,
 * tetm_rz_load, before the first step, or after a two-step pass of
 * TETM_RZ_KERNEL_BULK2; a last single step makes it available).
 * Synchronizes. */
int tetm_rz_charge_residual(tetm_rz* s, int32_t mode, double* max_e, double* max_h, double* q_scale);

/* Periodic balances: after every step n with n % every == 0 the energy and
 * the charges of every mode are queued into a device history without host
 * synchronisation (every = 0 turns them off); the two-step kernel takes a
 * single step into each such n. tetm_rz_balance_history copies the last
 * records (up to 1024 steps) into out: rows of six doubles {n, m, energy,
 * max_e, max_h, q_scale}, one row per mode and step, oldest first;
 * *n_out = rows (out may be NULL to query it; cap counts rows). Synchronizes. */
int tetm_rz_set_balance_every(tetm_rz* s, int32_t every);
int tetm_rz_balance_history(tetm_rz* s, double* out, int32_t cap, int32_t* n_out);

/* Checkpoint: tetm_rz_save writes the solve's current state (every mode, the
 * device layout), step and wake accumulators into a caller buffer of cap
 * bytes; *used receives the size (buf may be NULL to query it). tetm_rz_load
 * restores it into a solve created with the same grid, modes and geometry and
 * given the same bunch call (tetm_rz_set_bunch, _static or _scattered with the
 * same arguments; TETM_E_ARG on any mismatch). A run continued from a
 * checkpoint is bitwise the run without the split. Both synchronize. */
int tetm_rz_save(tetm_rz* s, void* buf, size_t cap, size_t* used);
int tetm_rz_load(tetm_rz* s, const void* buf, size_t size);

/* Device bytes tetm_rz_create would allocate for g (0 for a bad grid). */
int64_t tetm_rz_bytes_needed(const tetm_rz_grid* g);

/* Frees every device and host resource of the solve. NULL is accepted. */
int tetm_rz_destroy(tetm_rz* s);

#ifdef __cplusplus
}
#endif

#endif
