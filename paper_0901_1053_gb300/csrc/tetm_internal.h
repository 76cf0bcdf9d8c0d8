// Internal declarations of libtetm: device layout, kernel argument blocks and
// the launchers each translation unit provides. Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "tetm.h"

namespace tetm {

constexpr double kC = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.0 / (kEps0 * kC * kC);

// One activity bit per component and node index: bit c set <=> the object of
// component c attached to that node carries a field (non-PEC edge, face with
// two non-PEC cells inside the box). Components: ex ey ez hx hy hz = 0..5.
constexpr int kEX = 0, kEY = 1, kEZ = 2, kHX = 3, kHY = 4, kHZ = 5;

// Device layout of every per-node array (fields, mask, coefficients):
// planes k = -1..nz+1, rows j = -2..ny+1, columns i = -ox..px-ox-1, x fastest.
// Index (i, j, k) of the canonical FIT layout maps to idx(i, j, k). All
// entries outside the cells (index nx, ny or nz and the guard ring around)
// hold zero and are inactive, so every stencil and prefetch reads them
// without bounds checks.
struct Layout {
  int nx, ny, nz;
  int ox;            // column of i = 0 (16-byte aligned)
  long long px;      // row pitch in elements
  long long sz;      // plane stride in elements, (ny + 4) * px
  long long count;   // elements per array, (nz + 3) * sz
  __host__ __device__ __forceinline__ long long idx(int i, int j, int k) const {
    return ((long long)(k + 1) * (ny + 4) + (j + 2)) * px + (i + ox);
  }
};

Layout make_layout(int nx, int ny, int nz, int elem_bytes);

// Bunch data as the kernels see it (all device pointers).
template <typename T>
struct BunchDev {
  int on;               // 0: no bunch
  int i0, j0;           // bunch line node
  int c0;               // start offset in cells
  long long kshift;     // the bunch head is at plane n + kshift at step n (0: cold start)
  int m_min, m_max;     // wake window
  double inv_q;         // 1/Q
  const T* J;           // J[d + c0] = c*Q_cell(d)/dz [A], d = -c0..c0-1
  double* W;            // W[m - m_min], float64 accumulators
  // transverse wake on the observer line (obs_i, obs_j): W_x at the x-edge
  // line (obs_i + 1/2, obs_j) from e_x^n and h_y^{n+1/2}, W_y at the y-edge
  // line (obs_i, obs_j + 1/2) from e_y^n and h_x^{n+1/2}, float64
  int obs_on;           // the transverse wake is gathered (an observer was set)
  int obs_i, obs_j;
  double tw_ex, tw_hy;  // W_x += tw_ex e_x + tw_hy h_y
  double tw_ey, tw_hx;  // W_y += tw_ey e_y + tw_hx h_x
  double* WX;           // [m - m_min]
  double* WY;
};

// Transverse wake samples of plane k (step n -> n+1): W_x from the old e_x
// and the new h_y of the x-edge at the observer line, W_y from the old e_y
// and the new h_x of the y-edge; sample m = n + kshift - k - c0 as for W.
template <typename T>
__device__ __forceinline__ void gather_wx(const BunchDev<T>& b, long long n, int k, T ex_old, T hy_new) {
  const long long mm = (n + b.kshift) - k - b.c0;
  if (mm >= b.m_min && mm <= b.m_max)
    b.WX[mm - b.m_min] += b.tw_ex * (double)ex_old + b.tw_hy * (double)hy_new;
}
template <typename T>
__device__ __forceinline__ void gather_wy(const BunchDev<T>& b, long long n, int k, T ey_old, T hx_new) {
  const long long mm = (n + b.kshift) - k - b.c0;
  if (mm >= b.m_min && mm <= b.m_max)
    b.WY[mm - b.m_min] += b.tw_ey * (double)ey_old + b.tw_hx * (double)hx_new;
}

// Per-component coefficients: either one constant per component with the
// activity mask, or (material runs) one array per component.
template <typename T>
struct Coefs {
  const uint8_t* mask;  // activity bits, device layout
  T u[6];               // update coefficients alpha*M^-1 (ex,ey,hx,hy), 2 alpha*M^-1 (ez,hz)
  const T* ua[6];       // per-entry update coefficients, or nullptr
};

template <typename T>
struct StepArgs {
  const T* in[6];       // state y^n (fused: read only)
  T* out[6];            // fused: state y^{n+1}; reference: == in (updated in place)
  Coefs<T> co;
  Layout L;
  long long n;          // step index of the state being advanced
  BunchDev<T> b;
  // fused-kernel work decomposition
  int tiles_x, tiles_y, chunk_z, n_chunks;
  const int* work;      // optional list of active (tile, chunk) items; nullptr = all
  int n_work;
};

// One member of a batch as the batched kernels see it: its step arguments
// (advanced on the device: ping-pong pointers swapped and n incremented after
// every batch step) and whether it still has steps to take.
template <typename T>
struct BatchMember {
  StepArgs<T> a;
  long long limit;  // last step index + 1 this member may reach
  int active;       // 0 once a.n == limit
  int cur;          // the field set a.in points to (0 or 1)
};

// ---- launchers (kernels_step.cu) -----------------------------------------
template <typename T>
cudaError_t launch_reference_step(const StepArgs<T>& a, cudaStream_t st);
template <typename T>
cudaError_t launch_fused_step(const StepArgs<T>& a, int tile_x, int tile_y, cudaStream_t st);
bool fused_shape_ok(int tile_x, int tile_y);
// two steps per pass of the block-tiled sweep (temporal blocking); shapes
// 32 x 4, 32 x 8, 64 x 4; one material
template <typename T>
cudaError_t launch_fused_two_steps(const StepArgs<T>& a, int tile_x, int tile_y, cudaStream_t st);
bool fused2_shape_ok(int tile_x, int tile_y);
// ---- warp-tiled fused step (kernels_warp.cu): tile 28 x tile_y ----------
template <typename T>
cudaError_t launch_fused_warp_step(const StepArgs<T>& a, int tile_x, int tile_y, cudaStream_t st);
bool warp_shape_ok(int tile_x, int tile_y);
// one step of every active member of a batch (work = (member, item) pairs,
// their number read from device memory at n_work, at most n_bound: the grid
// is sized from n_bound so a captured launch stays valid while the list
// changes), then the device-side advance of all n_members slots
template <typename T>
cudaError_t launch_fused_warp_batch(const BatchMember<T>* members, int n_members, const int2* work,
                                    const int* n_work, int n_bound, int tile_y, int nz_max, cudaStream_t st);
// after a batch step: every active member swaps its sets, counts the step
// and retires at its limit
template <typename T>
cudaError_t launch_batch_advance(BatchMember<T>* members, int n_members, cudaStream_t st);

// ---- block-tiled float32 step with a shared-memory ring (kernels_slab.cu):
// tile 56 x 28, one CTA of 512 threads per SM; with coefficient arrays (mat)
// tile 56 x 12, two CTAs of 256 threads per SM ------------------------------
bool slab_shape_ok(int tile_x, int tile_y, bool mat);
// one step of every active member of a float32 batch on the slab kernel
// (work = (member, item) pairs counted at n_work in device memory, at most
// n_bound; sched as below), the transverse wakes, then the device-side
// advance of all n_members slots
cudaError_t launch_fused_slab_batch(BatchMember<float>* members, int n_members, const int2* work,
                                    const int* n_work, int n_bound, int* sched, int nz_max, cudaStream_t st);
// sched: two ints of device memory, zero before the first launch, that the
// kernel's dynamic schedule uses and leaves zero (nullptr: static order)
// (a.co.ua[0] set: the per-entry coefficient arrays of material runs)
cudaError_t launch_fused_slab_step(const StepArgs<float>& a, int* sched, cudaStream_t st);

// ---- Yee's E/M leapfrog, Eq. (7) (kernels_yee.cu): the step arguments carry
// dt M^-1 as the per-component constants --------------------------------------
template <typename T>
cudaError_t launch_yee_reference_step(const StepArgs<T>& a, cudaStream_t st);
template <typename T>
cudaError_t launch_yee_fused_step(const StepArgs<T>& a, cudaStream_t st);
void yee_shape(int elem_bytes, int* tile_x, int* tile_y);  // owned tile of the fused kernel

// transverse wake of a ping-pong step (kernels_step.cu): after the step
// kernel, before the sets are swapped
template <typename T>
cudaError_t launch_transverse_after_step(const StepArgs<T>& a, cudaStream_t st);
template <typename T>
cudaError_t launch_transverse_after_batch_step(const BatchMember<T>* members, int n_members, int nz_max,
                                               cudaStream_t st);

// ---- diagnostics (kernels_diag.cu) ----------------------------------------
struct DiagScratch {
  double* part;   // per-block partials
  int cap;        // entries of part
  double* out;    // device result slots (at least 8)
};

// The fused kernels' work items, which the balance reductions also walk:
// entries outside them lie in cells that carry no field.
struct WorkView {
  const int* items;  // active (tile, chunk) items; nullptr = every item
  int n_items;
  int tile_x, tile_y, chunk_z, tiles_x, tiles_y;
};

// Float64 fields with material arrays: the discrete energy W^{n,e} into
// *result (device) from the minv_a[c] arrays and their reciprocals m_a[c]
// (0 where minv_a is 0). Instantiated for double.
template <typename T>
cudaError_t launch_energy(const T* const f[6], const uint8_t* mask, const double* minv,
                          const double* const minv_a[6], const double* const m_a[6], const Layout& L, double alpha,
                          const WorkView& wv, const DiagScratch& s, double* result,
                          cudaStream_t st);

// Float64 fields with material arrays: the charge residuals of the last step
// into device slots, *res_e = max|qe - qbunch|, *res_h = max|qh|. Instantiated
// for double.
template <typename T>
cudaError_t launch_charge(const T* const cur[6], const T* const prev[6], const uint8_t* mask,
                          const double* minv, const double* const minv_a[6], const double* const m_a[6],
                          const Layout& L,
                          double alpha, const double* qline, int i0, int j0, const WorkView& wv,
                          const DiagScratch& s, double* res_e, double* res_h, cudaStream_t st);

// One material (minv[c] constants): the energy into *res_w and, when prev is
// not null, the charge residuals into *res_e, *res_h, in one pass (the
// launches above do the same for material arrays).
template <typename T>
cudaError_t launch_balances(const T* const cur[6], const T* const prev[6], const uint8_t* mask,
                            const double* minv, const Layout& L, double alpha, const double* qline, int i0,
                            int j0, const WorkView& wv, const DiagScratch& s, double* res_w, double* res_e,
                            double* res_h, cudaStream_t st);

// Float32 fields with material arrays: the energy into *res_w and, when prev
// is not null, the charge residuals into *res_e, *res_h, in one pass of
// float32-pair arithmetic; m[c]: M = 1/M^-1 per entry, a[c]: alpha^2 M^-1 per
// entry (c = kHX, kHY, kEX, kEY), both as (hi, lo) float32 pairs.
cudaError_t launch_balances_mat_f32(const float* const cur[6], const float* const prev[6], const uint8_t* mask,
                                   const float2* const m[6], const float2* const a[6], const Layout& L,
                                   double alpha, const double* qline, int i0, int j0, const WorkView& wv,
                                   const DiagScratch& s, double* res_w, double* res_e, double* res_h,
                                   cudaStream_t st);

// Truncated Gaussian bunch charge in the dual cell of each node k = 0..nz of
// the bunch line at bunch-centre position zc; *qmax = max |ql[k]|; *tag = tag.
cudaError_t launch_bunch_charge(double q, double sigma, double dz, double zc, int nz, double* ql,
                                double* qmax, double tag, double* tag_out, cudaStream_t st);

}  // namespace tetm

// The solve behind a tetm_solver* handle (host bookkeeping and device arrays).
struct tetm_solver {
  tetm_grid g;
  size_t esz;
  tetm::Layout L;
  void* set[2][6];
  int cur;
  uint8_t* mask;
  double minv_c[6];
  double* minv_a[6];
  double* m_a[6];  // float64 fields: 1 / minv_a (0 where minv_a is 0), for the balances
  float2* mp[6];   // float32 fields: the same as (hi, lo) float32 pairs
  float2* ap[6];   // float32 fields: alpha^2 minv_a as pairs (kHX, kHY, kEX, kEY)
  void* ua[6];
  bool uniform;
  bool vacuum;    // no material arrays (eps_r = mu_r = 1)
  double alpha;   // dt/2
  cudaStream_t stream;
  int scheme;     // TETM_SCHEME_*
  int kernel;
  int tile_x, tile_y, chunk_z;
  int* sched;                    // the slab kernel's schedule counters (two ints)
  int tiles_x, tiles_y, n_chunks;
  int* work;
  int n_work;
  std::vector<int> work_host;  // host copy of the work list
  bool in_batch;               // stepped by a tetm_batch
  bool work_dirty;
  // bunch
  bool bunch;
  int i0, j0, c0, m_min, m_max;
  long long kshift;   // static start: head at plane step + kshift
  double sigma, q;
  std::vector<double> qcell;
  void* J;
  double* W;          // [3][nw]: W, then the transverse W_x, W_y
  bool obs_on;        // transverse wake gathered (tetm_set_observer was called)
  int obs_i, obs_j;   // its observer line
  double* qline;
  // periodic balances: records {n, W, max_e, max_h, q_scale}
  int bal_every;
  double* hist;
  int hist_cap;
  long long hist_count;
  // state
  long long step;
  bool prev_valid;
  tetm::DiagScratch diag;
  double* staging;
  long long staging_elems;
  long long device_bytes;
  long long active_cells;
  // z-slab of a larger grid: planes [k_lo, k_lo + g.nz) of nz_all (whole grid: 0, g.nz)
  int k_lo;
  int nz_all;
  bool is_slab() const { return k_lo > 0 || g.nz < nz_all; }
};

namespace tetm {
// step arguments of a solve for the fused (ping-pong) or reference kernel
template <typename T>
StepArgs<T> step_args(tetm_solver* s, bool fused);
// (re)build the list of (tile, chunk) work items that own a field-carrying cell
int rebuild_work(tetm_solver* s);
// Device memory of solves and batches comes from one stream-ordered pool per
// device: allocation and release are queued on the given stream, so neither
// waits for work queued on other streams (cudaFree waits for the whole
// device, which would stall a batch running beside a solve being created or
// destroyed on another host thread). Memory is usable on other streams once
// the allocating stream has reached the allocation.
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st);
void dev_free(void* p, cudaStream_t st);
}  // namespace tetm
