/*
 * tetm.h — C ABI of libtetm.so, a GB300 (sm_103a) solver for the explicit
 * TE/TM scheme of M. Dohlus and I. Zagorodnov, "Explicit TE/TM scheme for
 * particle beam simulations": the two-level TE/TM-split leapfrog (Sec. 4.2,
 * Eq. (23)) of the FIT grid-doublet fields on a Cartesian grid, with a rigid
 * relativistic Gaussian bunch current injected each step and the longitudinal
 * wake potential (Sec. 5) gathered along the bunch path.
 *
 * Conventions shared by every call
 *  - Return value: TETM_OK (0) or a negative TETM_E_* code; no call aborts,
 *    traps or exits. tetm_strerror() names a code.
 *  - Handles are not thread-safe; distinct handles may be used from distinct
 *    host threads. All device memory of a solve is allocated by tetm_create
 *    and released by tetm_destroy (the handle owns it). Host arrays passed in
 *    are read during the call only; host arrays passed out are written
 *    during the call only; the caller owns both.
 *  - Device work is queued on the solver's CUDA stream (tetm_set_stream).
 *    Calls marked "synchronizes" wait for that stream before returning.
 *  - Geometry: a closed box of nx*ny*nz primary cells with perfectly
 *    conducting walls, n x E = 0 (Sec. 2, Eq. (1)). Cell (ci, cj, ck) has the
 *    C-order index ci + nx*(cj + ny*ck) (x fastest).
 *  - Field layout ("canonical FIT layout", Sec. 2): one float64 vector per
 *    component with (nx+1)*(ny+1)*(nz+1) entries, entry i + (nx+1)*(j +
 *    (ny+1)*k) attached to node (i,j,k):
 *      ex (i+1/2,j,k)  ey (i,j+1/2,k)  ez (i,j,k+1/2)       edge voltages [V]
 *      hx (i,j+1/2,k+1/2)  hy (i+1/2,j,k+1/2)  hz (i+1/2,j+1/2,k)  [A]
 *    Entries on PEC edges, on faces next to PEC and outside the box are zero.
 *  - Time: the state after n steps is y^n = (u^{n-1/2}, v^n) with
 *    u = (hx, hy, ez) and v = (ex, ey, hz) (Sec. 4.1, Eq. (17)).
 */
#ifndef TETM_H
#define TETM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define TETM_OK 0
#define TETM_E_ARG (-1)        /* bad argument (NULL, size, range)                 */
#define TETM_E_UNSTABLE (-2)   /* time step outside Eq. (25)                        */
#define TETM_E_NOT_MAGIC (-3)  /* bunch / wake need c*dt == dz (Sec. 4.5, Sec. 5)   */
#define TETM_E_NOMEM (-4)      /* device or host allocation failed                  */
#define TETM_E_CUDA (-5)       /* a CUDA runtime call failed                        */
#define TETM_E_STATE (-6)      /* call not valid in the solver's current state      */
#define TETM_E_TIMEOUT (-7)    /* a bounded device-side wait gave up                */
#define TETM_E_DIVERGED (-8)   /* non-finite energy: the run blew up               */
#define TETM_E_UNSUPPORTED (-9) /* combination of options the library does not offer */
#define TETM_E_TOO_LARGE (-10) /* problem exceeds the fixed scratch of tetm_energy_noalloc */

/* ---- field precision ---------------------------------------------------- */
#define TETM_FP64 0            /* fields stored and updated in float64            */
#define TETM_FP32 1            /* fields in float32; wake and balances in float64 */

/* ---- update kernels ------------------------------------------------------ */
#define TETM_KERNEL_FUSED 0     /* one z-marching launch per step (default)        */
#define TETM_KERNEL_REFERENCE 1 /* one launch per update equation: 10 per step     */
#define TETM_KERNEL_TWOSTEP 2   /* block-tiled sweep advancing two steps per pass   */

/* ---- time-stepping schemes ------------------------------------------------ */
#define TETM_SCHEME_TETM 0      /* the explicit TE/TM scheme, Eq. (23) (default)   */
#define TETM_SCHEME_YEE 1       /* Yee's E/M leapfrog, Eq. (7), field-only         */

/* ---- components ---------------------------------------------------------- */
#define TETM_EX 0
#define TETM_EY 1
#define TETM_EZ 2
#define TETM_HX 3
#define TETM_HY 4
#define TETM_HZ 5

typedef struct tetm_grid {
  int32_t nx, ny, nz;  /* primary cells, each >= 2                          */
  int32_t precision;   /* TETM_FP64 or TETM_FP32                             */
  double dx, dy, dz;   /* cell sizes [m], > 0                                */
  double cdt;          /* c*dt [m]; 0 selects dz, the step of Sec. 4.5       */
} tetm_grid;

typedef struct tetm_info {
  int64_t step;            /* n of the current state y^n                     */
  int64_t device_bytes;    /* device memory held by the solve                */
  int64_t active_cells;    /* cells that carry at least one non-PEC object   */
  int64_t processed_cells; /* cells the fused kernel reads and writes a step */
  int32_t kernel;          /* TETM_KERNEL_*                                  */
  int32_t precision;       /* TETM_FP64 / TETM_FP32                          */
  int32_t tile_x, tile_y, chunk_z; /* fused-kernel block shape               */
  int32_t work_items;      /* (tile, z-chunk) blocks launched per step       */
  int32_t wake_len;        /* wake samples (0 before tetm_set_bunch)         */
  int32_t uniform_material;/* 1 if every active coefficient of a component is equal */
} tetm_info;

typedef struct tetm_solver tetm_solver;

/* Create a solve (Sec. 2, Eq. (4) with the staircase reading of the
 * material matrices):
 *   - an edge is PEC (M_eps^-1 = 0) if any of the up to four cells sharing it
 *     is PEC or outside the box; otherwise M_eps^-1 = L / (eps0 eps_bar A~)
 *     with eps_bar the mean eps_r of those cells;
 *   - a face is active only if both cells sharing it are inside and not PEC;
 *     M_mu^-1 = L~ / (mu0 mu_bar A), 1/mu_bar the mean of 1/mu_r.
 * eps_r, mu_r: float64 per cell (>= 1), NULL = vacuum. pec: uint8 per cell,
 * nonzero = PEC, NULL = none. All three are read during the call only.
 * Checks Eq. (25): c*dt <= dz and c*dt <= (dx^-2 + dy^-2)^-1/2, else
 * TETM_E_UNSTABLE. The fields start at zero (cold start, y^0 = 0).
 * On failure *out is set to NULL. */
int tetm_create(const tetm_grid* g, const double* eps_r, const double* mu_r, const uint8_t* pec,
                tetm_solver** out);

/* tetm_create with the solve's work, its creation included, queued on
 * `stream` (a cudaStream_t; NULL = the legacy default stream, as
 * tetm_create). Creating on a non-blocking stream from another host thread
 * does not wait for, or hold up, work on other streams (a running batch).
 * Device memory of every solve comes from a stream-ordered pool of the
 * library (one per device): allocations and releases are queued on the
 * solve's stream and never wait for the whole device. */
int tetm_create_on_stream(const tetm_grid* g, const double* eps_r, const double* mu_r, const uint8_t* pec,
                          void* stream, tetm_solver** out);

/* Bytes of released device memory the library's pool keeps for reuse
 * instead of returning them to the device (default 0: everything is
 * returned at the next synchronization). A server that creates and
 * destroys solves continuously sets its device-memory budget here. */
int tetm_pool_reserve(uint64_t bytes);

/* Rigid ultra-relativistic Gaussian bunch (Sec. 3 and Sec. 5): RMS length
 * sigma_z [m] > 0, charge [C] != 0, moving at c along the z-line through
 * node (i0, j0), 1 <= i0 <= nx-1, 1 <= j0 <= ny-1. The line density is
 * truncated at +-5 sigma_z; at t = 0 the centre is c0 = ceil(5 sigma/dz)
 * cells behind the wall z = 0. Edge (i0, j0, k+1/2) carries
 * jj_z^n = c * Q_cell(k - n + c0) / dz, Q_cell(d) the charge in
 * [d dz, (d+1) dz] of the bunch frame. Needs c*dt == dz (TETM_E_NOT_MAGIC)
 * and must precede the first step (TETM_E_STATE). Defines the wake window
 * s_m = m dz, m = -c0-1 .. ceil(15 sigma/dz). */
int tetm_set_bunch(tetm_solver* s, double sigma_z, double charge, int32_t i0, int32_t j0);

/* Static start (Sec. 5: the paper's structures sit between infinite ingoing
 * and outgoing pipes): the bunch of tetm_set_bunch (same sigma_z, charge,
 * i0, j0, profile and wake window) begins with its head at plane k_head
 * instead of at the wall, carrying its own discrete TEM field, so it moves
 * through the uniform entry section without radiating (at c*dt = dz the field
 * shifts one cell per step, Sec. 4.5). The transverse potential solves the
 * discrete Poisson problem of the entry cross-section (non-PEC edges, zero on
 * nodes touching PEC); the longitudinal profile carries the bunch current.
 * Current and wake samples then refer to step + k_head. Requires: vacuum
 * (no eps_r/mu_r, else TETM_E_UNSUPPORTED); step 0 and no bunch yet
 * (TETM_E_STATE); c*dt == dz (TETM_E_NOT_MAGIC); 2*c0 + 2 <= k_head <= nz
 * with c0 = ceil(5 sigma_z/dz), planes 1..k_head of the grid carrying the
 * same objects, and (i0, j0) a node whose ez edge is not PEC (TETM_E_ARG).
 * Writes planes 0..k_head+1 of the state. Synchronizes. */
int tetm_set_bunch_static(tetm_solver* s, double sigma_z, double charge, int32_t i0, int32_t j0,
                          int32_t k_head);

/* Advance n >= 0 steps of Eq. (23): per step the ten updates of Sec. 4.2
 * (TM stage hx, hy, ez, hx, hy; TE stage ex, ey, hz, ex, ey), the bunch
 * current in the ez update and one wake sample per window point. Queued on
 * the solver's stream; returns once the launches are queued. */
int tetm_step(tetm_solver* s, int32_t n);

/* Wait for the solver's stream (synchronizes). */
int tetm_sync(tetm_solver* s);

/* Longitudinal wake W(s_m) [V/C], W(s) = -(1/Q) * integral of E_z along the
 * test-charge path t = (z + s)/c (Sec. 5), exact on the grid at c*dt = dz,
 * accumulated in float64. Copies n = window length values into out[cap]
 * (cap >= n, else TETM_E_ARG; out may be NULL to query n). *s0 = s of the
 * first sample, *ds = dz. Any output pointer may be NULL. Synchronizes. */
int tetm_wake(tetm_solver* s, double* out, int32_t cap, int32_t* n_out, double* s0, double* ds);

/* Turns on the transverse (dipole) wake W_perp = (1/Q) * integral of
 * (E + c z^ x B)_perp along the test-charge path (Sec. 5) on the observer
 * line through node (i, j), 0 <= i <= nx-1, 0 <= j <= ny-1 (pass i0, j0 for
 * the bunch line). Each step then adds one small gather launch (none without
 * an observer). Needs a bunch and step 0 (TETM_E_STATE). */
int tetm_set_observer(tetm_solver* s, int32_t i, int32_t j);

/* Transverse wake [V/C] on the window of tetm_wake, accumulated in float64:
 * wx = (1/Q) sum (E_x - c mu0 H_y) dz on the x-edge line (i + 1/2, j),
 * from e_x of time n at plane k and h_y of time n+1/2 at k+1/2 (both met by
 * the test charge at c*dt = dz); wy = (1/Q) sum (E_y + c mu0 H_x) dz on the
 * y-edge line (i, j + 1/2), from e_y and h_x. E = e / (edge length), H = h /
 * (dual edge length). Either output may be NULL; cap >= the window length
 * (TETM_E_ARG), TETM_E_STATE without a bunch or an observer. Synchronizes. */
int tetm_transverse_wake(tetm_solver* s, double* wx, double* wy, int32_t cap, int32_t* n_out,
                         double* s0, double* ds);

/* Release the solve and all its device memory. NULL-safe. */
void tetm_destroy(tetm_solver* s);

/* Discrete energy of the explicit scheme, W^{n,e} = 1/2 <Q^e y^n, y^n>
 * with Q^e = B^e - alpha A (Sec. 4.4), in J, summed in float64 on the
 * device in a fixed order. TETM_E_DIVERGED if not finite. Synchronizes. */
int tetm_energy(tetm_solver* s, double* w);

/* Charge balances of the last step (Sec. 4.5), float64 on the device, over
 * nodes (cells) whose six edges (faces) are all active:
 *   *max_e = max |qbar_e^{n+1/2} - q_bunch^{n+1/2}|, Eq. (35) summed from a
 *            cold start; q_bunch is the truncated Gaussian charge inside the
 *            node's dual cell on the bunch line, 0 elsewhere;
 *   *max_h = max |qbar_h^{n-1/2}|, Eq. (34) from a cold start;
 *   *q_scale = max |q_bunch| (0 without a bunch) for relative residuals.
 * Needs at least one step since creation or the last tetm_set_fields
 * (TETM_E_STATE). Valid for cold starts. Synchronizes. */
int tetm_charge_residual(tetm_solver* s, double* max_e, double* max_h, double* q_scale);

/* Periodic FP64 balances inside tetm_step (0 = off, the default): after
 * every `every`-th step the solver queues, on its stream and without host
 * synchronisation, the energy of tetm_energy and the charge residuals of
 * tetm_charge_residual for the state just reached, as one record
 * {n, W^{n,e}, max_e, max_h, q_scale} in a device ring of 4096 records
 * (the oldest is overwritten). */
int tetm_set_balance_every(tetm_solver* s, int32_t every);

/* Copy the recorded balances, oldest first, 5 float64 per record, into
 * out[cap] (cap counts records; cap below the record count gives
 * TETM_E_ARG; out may be NULL to query the count *n). Synchronizes. */
int tetm_balance_history(tetm_solver* s, double* out, int32_t cap, int32_t* n);

/* Copy one component (TETM_EX..TETM_HZ) of the current state to / from a
 * host float64 array in the canonical FIT layout. Values on entries that
 * carry no field are ignored on input and zero on output. Both synchronize. */
int tetm_get_fields(tetm_solver* s, int32_t comp, double* host);
int tetm_set_fields(tetm_solver* s, int32_t comp, const double* host);

/* Use this CUDA stream (a cudaStream_t, NULL = legacy default stream) for
 * all later device work of the solve. The stream is not owned. */
int tetm_set_stream(tetm_solver* s, void* cuda_stream);

/* Select the update kernels (TETM_KERNEL_*). With general materials (per-cell
 * eps_r / mu_r that differ) the fused path streams per-entry coefficient
 * arrays and needs the warp-tiled work shape (tile_x = 28) or, in float32,
 * the slab shape 56 x 12 (the defaults); the block-tiled shapes then give
 * TETM_E_UNSUPPORTED. */
int tetm_set_kernel(tetm_solver* s, int32_t kernel);
/* TETM_KERNEL_TWOSTEP (temporal blocking of the sweep, Eq. (23) applied twice
 * per pass over the fields: y^n read once, y^{n+2} written once) needs one
 * material, the TE/TM scheme, a whole grid and a block-tiled shape of 32 x 4,
 * 32 x 8 or 64 x 4 (TETM_E_UNSUPPORTED otherwise). tetm_step runs pairs of
 * steps on it, and single steps on the block-tiled one-step kernel where a
 * pair would skip a balance or a transverse-wake gather and for an odd last
 * step. After a call that ended on a pair the previous state is not kept:
 * tetm_charge_residual answers TETM_E_STATE until a call ends on a single
 * step. Fields equal the one-step kernel's bit for bit; wake samples are
 * summed with atomic adds (equal up to rounding). */

/* Fused-kernel work shape: transverse tile tile_x x tile_y and z-chunk
 * length chunk_z >= 4 of one work item. 56 x 28 selects the float32 slab
 * kernel for one material (one CTA of 512 threads per SM; e_z, h_z staged in
 * shared memory by per-thread asynchronous copies of the quads that carry
 * them), 56 x 12 the slab kernel for material arrays (two CTAs of 256
 * threads per SM; e_z, h_z and the six coefficient arrays staged the same
 * way); each gives TETM_E_UNSUPPORTED for the other kind of solve and in
 * float64; the float32 defaults, chunk 32);
 * tile_x = 28 the warp-tiled kernel (one warp per item, tile_y in {4, 8,
 * 12, 16, 20, 28};
 * the float64 default, 28 x 20 x 32); tile_x = 32 (tile_y in {4, 8, 16}) or
 * 64 (tile_y in {4, 8}) the block-tiled kernel (one material only). Any value
 * 0 keeps the current one. TETM_E_ARG for other values. */
int tetm_set_tiling(tetm_solver* s, int32_t tile_x, int32_t tile_y, int32_t chunk_z);

/* Time-stepping scheme (TETM_SCHEME_*), before the first step. Yee's scheme
 * (Sec. 3, Eq. (7)) is the paper's comparison scheme on the same grid and
 * material matrices: state (e^{n-1/2}, h^n), e^{n+1/2} = e^{n-1/2} +
 * dt M_eps^-1 C~ h^n, h^{n+1} = h^n - dt M_mu^-1 C e^{n+1/2}. It carries no
 * bunch (its step bound (8), c*dt <= (dx^-2 + dy^-2 + dz^-2)^-1/2, excludes
 * the TE/TM scheme's c*dt = dz that the wake needs): initial fields come from
 * tetm_set_fields, where e is read as e^{-1/2} and h as h^0. The fused path
 * is one z-marching launch per step (float32: 56 x 30 owned of 64 x 32 loaded
 * nodes per CTA; float64: 60 x 14 of 64 x 16; any chunk_z >= 4); material
 * arrays run on the reference updates (two launches per step).
 * TETM_E_UNSTABLE if c*dt breaks (8), TETM_E_STATE after the first step,
 * with a bunch, in a batch or with periodic balances on. With Yee's scheme
 * tetm_energy, tetm_charge_residual, tetm_set_balance_every (> 0),
 * tetm_save and tetm_load give TETM_E_UNSUPPORTED (their quantities are the
 * TE/TM scheme's), and tetm_set_tiling accepts only the chunk length. */
int tetm_set_scheme(tetm_solver* s, int32_t scheme);

/* Canary of out-of-place writes: counts, over both field sets and all six
 * components, the device entries that hold a non-zero value although they
 * carry no field (the zero guard ring around the cells and the entries of PEC
 * edges and faces, which every update leaves at zero). A correct run reports
 * 0. Synchronizes; TETM_E_ARG for NULL arguments. */
int tetm_check_guards(tetm_solver* s, int64_t* violations);

/* Snapshot of the solve's bookkeeping. */
int tetm_get_info(tetm_solver* s, tetm_info* info);

/* Device bytes tetm_create would allocate for this grid (0 on a bad grid),
 * for admission control by a caller that budgets device memory. */
int64_t tetm_bytes_needed(const tetm_grid* g);

/* Save the complete state (fields, step counter, wake accumulators) into a
 * caller buffer of cap bytes; *used receives the size (buf may be NULL to
 * query it). tetm_load restores it into a solve created with the same grid
 * and geometry (TETM_E_ARG on a size or grid mismatch). Both synchronize. */
int tetm_save(tetm_solver* s, void* buf, size_t cap, size_t* used);
int tetm_load(tetm_solver* s, const void* buf, size_t size);

/* ---- z-slabs of one solve ---------------------------------------------------
 * The scheme couples neighbouring planes only: an update of planes
 * [k0, k1) reads the state at planes k0 - 1 .. k1 (the TM stage of plane
 * k0 - 1 is recomputed, e_x and e_y of plane k1 enter the TM stage of plane
 * k1 - 1). So a grid splits along z into slabs that advance side by side
 * (Sec. 4, the scheme is easily parallelised) when, before every step, each
 * slab receives
 *   from the slab below: the six components of its last plane (into the
 *   ghost plane below the slab's first plane);
 *   from the slab above: e_x and e_y of its first plane (into the plane
 *   above the slab's last plane).
 * Bunch current and wake stay with the planes that carry them: every slab
 * adds its own planes' samples, the wake of the grid is the sum of the
 * slabs' wakes. The results equal the whole-grid solve's (the same
 * arithmetic per plane; the wake up to the order of that sum).
 *
 * tetm_create_slab: a solve of planes [k_lo, k_hi) (k_hi - k_lo >= 2) of the
 * grid g; eps_r, mu_r, pec cover the whole grid as in tetm_create. Its local
 * plane k is plane k_lo + k of the grid (tetm_get_fields / tetm_set_fields
 * give local planes 0 .. k_hi - k_lo, the last being the neighbour's).
 * tetm_set_bunch takes the grid's bunch line and cold start; the reference
 * kernel, Yee's scheme, the static start, periodic balances and batches
 * are not available for a slab (TETM_E_UNSUPPORTED). */
#define TETM_PLANES_UP 0    /* the message to the slab above: six components of the last plane */
#define TETM_PLANES_DOWN 1  /* the message to the slab below: e_x, e_y of the first plane      */
int tetm_create_slab(const tetm_grid* g, int32_t k_lo, int32_t k_hi, const double* eps_r,
                     const double* mu_r, const uint8_t* pec, tetm_solver** out);
/* Bytes of a message in direction dir (six or two planes of the device
 * layout, (ny + 4) * row pitch entries each); 0 for a bad argument. */
int64_t tetm_plane_bytes(tetm_solver* s, int32_t dir);
/* tetm_export_plane copies the message for direction dir out of the current
 * state into buf; tetm_import_plane copies a message received from the
 * neighbour (a message moving up comes from the slab below) into the
 * current state's ghost plane (TETM_E_STATE when there is no such
 * neighbour). buf is host or device memory of tetm_plane_bytes bytes
 * (pinned host memory or a device buffer for NCCL send/recv); both queue
 * copies on the solve's stream and return: tetm_sync before reading an
 * exported host buffer, and import before the next tetm_step. */
int tetm_export_plane(tetm_solver* s, int32_t dir, void* buf);
int tetm_import_plane(tetm_solver* s, int32_t dir, const void* buf);

/* ---- no-allocation variant ------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that are not allowed to allocate device memory: code whose device memory
 * comes from an arena or allocator owned by a host framework, plugins that
 * may only use buffers handed to them, and real-time loops that cannot pay
 * for cudaMalloc/cudaFree or their implicit synchronisation.
 *
 * tetm_energy_noalloc computes the same discrete energy as tetm_energy
 * for a state the caller keeps in its own device arrays,
 * and allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 * call. Its block partial sums live in one fixed array of 8192 doubles
 * (64 KiB) in the library's device memory, which every GPU that loads the
 * library holds until the process exits.
 *   g       grid; vacuum only (the coefficients follow from dx, dy, dz, cdt);
 *           g->precision says whether fields are float64 or float32.
 *   fields  six device pointers (ex, ey, ez, hx, hy, hz), each in the
 *           canonical FIT layout of this header, (nx+1)(ny+1)(nz+1) entries.
 *   mask    device uint8 per canonical entry, bit c set when component c
 *           carries a field there (PEC geometry); NULL = empty PEC box.
 *   w       device double that receives the energy [J].
 *   stream  cudaStream_t the two kernels are queued on (NULL = legacy stream);
 *           the call returns once they are queued and does not synchronize.
 * At most TETM_NOALLOC_MAX_ENTRIES canonical entries (e.g. 256 x 256 x 499
 * cells); larger grids return TETM_E_TOO_LARGE; a grid that tetm_create
 * would reject (non-finite or non-positive steps, cell counts out of range)
 * returns TETM_E_ARG. The first call on a device, and in each further
 * driver context a caller makes current on it, looks up the scratch array's
 * device address (cudaGetSymbolAddress) with that device current and caches
 * it; make that first call before any stream capture. Calls share the
 * scratch array: calls whose kernels overlap on the
 * GPU (several streams or host threads at once) race and must be serialised
 * by the caller. */
#define TETM_NOALLOC_MAX_ENTRIES 33554432
int tetm_energy_noalloc(const tetm_grid* g, const void* const fields[6], const uint8_t* mask,
                        double* w, void* stream);

/* ---- batches of solves ------------------------------------------------------
 * A batch advances several solves together: every batch step is one launch
 * over the work items of all members (the slab kernel for float32 members
 * whose first member has its 56 x 28 tile, the float32 default; the
 * warp-tiled kernel otherwise), followed by a device-side advance of every
 * member (field-set swap, step count, retirement at its step limit). Members keep their own grid, geometry,
 * bunch, wake and step counter; the paper's scheme is applied to each member
 * exactly as by tetm_step (the results are bit-identical to stepping each
 * solve alone). */
typedef struct tetm_batch tetm_batch;

/* Group n distinct solves of one precision and one uniform material each.
 * step_limits[i] >= 0: member i stops when its step counter reaches it
 * (NULL or a negative entry: no limit). Members take the first member's
 * tile (the slab kernel's 56 x 28 in float32, else the warp-tiled kernel
 * with the first member's tile height); each keeps its own z-chunk length. graph_steps > 0:
 * runs of that many steps are captured once as a CUDA graph and replayed;
 * 0 launches every step directly. While in the batch a member rejects
 * tetm_step, tetm_set_fields, tetm_set_kernel, tetm_set_tiling and tetm_load
 * (TETM_E_STATE); read-only calls (tetm_wake, tetm_get_fields, tetm_energy,
 * tetm_charge_residual) remain valid after tetm_batch_sync. Remove a member
 * (tetm_batch_remove) or destroy the batch before destroying the member. */
int tetm_batch_create(tetm_solver* const* solvers, const int64_t* step_limits, int32_t n,
                      int32_t graph_steps, tetm_batch** out);

/* Queue nsteps batch steps; each member advances min(nsteps, limit - step).
 * If a launch fails (TETM_E_CUDA) the batch refuses further steps
 * (TETM_E_STATE) and each member's step count and current field set are
 * re-read from its device descriptor, so member reads see the steps the
 * device did take. */
int tetm_batch_step(tetm_batch* b, int32_t nsteps);

/* Wait for the batch's stream (synchronizes). */
int tetm_batch_sync(tetm_batch* b);

/* Members, members below their limit, and (member, item) work entries. */
int tetm_batch_info(tetm_batch* b, int32_t* n_members, int32_t* n_active, int32_t* work_items);

/* Release the batch (synchronizes); members become independent again. */
void tetm_batch_destroy(tetm_batch* b);

/* Slot table: an empty batch of `capacity` >= 1 slots for members of one
 * precision (TETM_FP32 / TETM_FP64) on one tile (tile_x, tile_y: 56 x 28
 * selects the float32 slab kernel; otherwise tile_x = 28 and tile_y one of
 * the warp-tiled kernel's heights). Members join and leave between calls of
 * tetm_batch_step without rebuilding the batch: joining writes the member's
 * descriptor into a free slot and leaving clears the slot's active flag,
 * both queued on the batch's stream, and the combined work list is uploaded
 * before the next step (stream-ordered, from pinned host memory). The
 * captured graph is kept across membership changes; it is captured again
 * only when the work list outgrows its device buffer or a member needs a
 * larger transverse-wake grid. */
int tetm_batch_create_slots(int32_t capacity, int32_t precision, int32_t tile_x, int32_t tile_y,
                            int32_t graph_steps, tetm_batch** out);

/* Join: solve s (same precision, one uniform material, TE/TM scheme, not a
 * z-slab, not in a batch: TETM_E_ARG / TETM_E_UNSUPPORTED) takes a free
 * slot (TETM_E_STATE when all are taken; *slot, which may be NULL, receives
 * its index) and advances with the batch until its step counter reaches
 * step_limit (< 0: no limit). The batch's stream first waits for the work
 * queued on s's stream (its creation); the host does not wait. s takes the
 * batch's tile (its work list is rebuilt if it had another). */
int tetm_batch_add(tetm_batch* b, tetm_solver* s, int64_t step_limit, int32_t* slot);

/* Leave: s (a member, else TETM_E_ARG) gives up its slot after the steps
 * queued so far; s's stream then waits for them, so reads and tetm_destroy
 * queued on s see its final state. The host does not wait. */
int tetm_batch_remove(tetm_batch* b, tetm_solver* s);

/* Wait until at most max_pending >= 0 tetm_batch_step calls are still
 * unfinished on the device (0: all done), bounding how far the host queues
 * ahead of the GPU. *busy_s (may be NULL) receives the device time of the
 * batch's finished calls so far (from events bracketing each call on the
 * batch's stream: time the GPU spent on the batch, not idle gaps between
 * calls). Calls are tracked in a ring of 64: a 65th unfinished call first
 * waits for the oldest. */
int tetm_batch_wait(tetm_batch* b, int32_t max_pending, double* busy_s);

/* Static description of a return code. */
/* Measured fused multiply-add rate of the current device in TFLOP/s (2 flops
 * per FMA) for TETM_FP64 or TETM_FP32 arithmetic: eight independent chains
 * per thread on every SM, timed with CUDA events on the given stream (NULL:
 * the default stream). The float64 rate is the ALU roofline of the float64
 * update kernels. Synchronizes. */
int tetm_measure_fma_rate(int32_t precision, double* tflops, void* stream);

const char* tetm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* TETM_H */
