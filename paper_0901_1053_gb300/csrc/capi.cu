// C ABI of libtetm (include/tetm.h): solve lifetime, geometry, bunch,
// stepping, wake, diagnostics and checkpoints. Host logic only; the update
// and reduction kernels live in kernels_step.cu and kernels_diag.cu.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "tetm_internal.h"
#include <nvtx3/nvToolsExt.h>

using namespace tetm;

namespace tetm {

Layout make_layout(int nx, int ny, int nz, int elem_bytes) {
  Layout L;
  L.nx = nx;
  L.ny = ny;
  L.nz = nz;
  // i = 0 after the guard columns: at column 8 in float32 (the 56-column tiles
  // of the slab kernel then write whole 32-byte sectors, and its tensor copies
  // start on 16-byte boundaries), at 2 in float64
  L.ox = elem_bytes == 4 ? 8 : 2;
  // rows on 32-byte sectors; float32 rows a multiple of 16 entries, so the
  // byte-wide activity rows are 16-byte strides for tensor copies
  const int align = elem_bytes == 4 ? 16 : 32 / elem_bytes;
  long long px = L.ox + nx + 3;                    // >= 2 zero columns past nx, plus one
                                                   // so a column pair starting at nx + 1 stays in the row
  px = (px + align - 1) / align * align;
  L.px = px;
  L.sz = (long long)(ny + 4) * px;
  L.count = (long long)(nz + 3) * L.sz;            // planes -1 .. nz+1
  return L;
}

}  // namespace tetm

namespace {

// ---------------------------------------------------------------------------
// Geometry on the device (staircase reading of the material matrices)
// ---------------------------------------------------------------------------
struct GeomIn {
  const uint8_t* pec;    // per cell of the whole grid or nullptr
  const double* eps;     // per cell of the whole grid or nullptr
  const double* mu;      // per cell of the whole grid or nullptr
  int nx, ny, nz;        // nz: planes of this solve
  int k_off, nz_all;     // z-slab: global plane of local plane 0, planes of the whole grid
  double dx, dy, dz;
};

// cell (ci, cj, ck) of this solve (ck local): PEC outside the whole grid
__device__ __forceinline__ bool gpec(const GeomIn& g, long ci, long cj, long ck) {
  ck += g.k_off;
  if (ci < 0 || cj < 0 || ck < 0 || ci >= g.nx || cj >= g.ny || ck >= g.nz_all) return true;
  return g.pec ? g.pec[ci + (long)g.nx * (cj + (long)g.ny * ck)] != 0 : false;
}
__device__ __forceinline__ double gval(const double* a, const GeomIn& g, long ci, long cj, long ck) {
  return a ? a[ci + (long)g.nx * (cj + (long)g.ny * (ck + g.k_off))] : 1.0;
}

// Edge along `axis` at node (i,j,k): the four cells around it.
__device__ double edge_minv(const GeomIn& g, int axis, long i, long j, long k) {
  long c[4][3];
  double len, area;
  if (axis == 0) {
    long t[4][3] = {{i, j - 1, k - 1}, {i, j, k - 1}, {i, j - 1, k}, {i, j, k}};
    memcpy(c, t, sizeof(c)); len = g.dx; area = g.dy * g.dz;
  } else if (axis == 1) {
    long t[4][3] = {{i - 1, j, k - 1}, {i, j, k - 1}, {i - 1, j, k}, {i, j, k}};
    memcpy(c, t, sizeof(c)); len = g.dy; area = g.dx * g.dz;
  } else {
    long t[4][3] = {{i - 1, j - 1, k}, {i, j - 1, k}, {i - 1, j, k}, {i, j, k}};
    memcpy(c, t, sizeof(c)); len = g.dz; area = g.dx * g.dy;
  }
  double e = 0.0;
  for (int q = 0; q < 4; ++q) {
    if (gpec(g, c[q][0], c[q][1], c[q][2])) return 0.0;
    e += gval(g.eps, g, c[q][0], c[q][1], c[q][2]);
  }
  return len / (kEps0 * 0.25 * e * area);
}

// Face normal to `axis` at node (i,j,k): the two cells sharing it.
__device__ double face_minv(const GeomIn& g, int axis, long i, long j, long k) {
  long c[2][3];
  double len, area;
  if (axis == 0) {
    long t[2][3] = {{i - 1, j, k}, {i, j, k}};
    memcpy(c, t, sizeof(c)); len = g.dx; area = g.dy * g.dz;
  } else if (axis == 1) {
    long t[2][3] = {{i, j - 1, k}, {i, j, k}};
    memcpy(c, t, sizeof(c)); len = g.dy; area = g.dx * g.dz;
  } else {
    long t[2][3] = {{i, j, k - 1}, {i, j, k}};
    memcpy(c, t, sizeof(c)); len = g.dz; area = g.dx * g.dy;
  }
  double r = 0.0;
  for (int q = 0; q < 2; ++q) {
    if (gpec(g, c[q][0], c[q][1], c[q][2])) return 0.0;
    r += 1.0 / gval(g.mu, g, c[q][0], c[q][1], c[q][2]);
  }
  return len * 0.5 * r / (kMu0 * area);
}

struct MinvOut {
  double* a[6];  // per-entry M^-1 arrays (material runs) or nullptr
};

// Activity bits (and M^-1 arrays) of the node entries of planes k_first ..
// nz: k_first = 0 for a whole grid, -1 for a z-slab whose plane below its
// first one is a ghost plane with the geometry of the whole grid.
__global__ void build_geometry(GeomIn g, Layout L, int k_first, uint8_t* mask, MinvOut mo) {
  const long long total = (long long)(g.nx + 1) * (g.ny + 1) * (g.nz + 1 - k_first);
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int i = (int)(q % (g.nx + 1));
  const int j = (int)((q / (g.nx + 1)) % (g.ny + 1));
  const int k = k_first + (int)(q / ((long long)(g.nx + 1) * (g.ny + 1)));
  const long long id = L.idx(i, j, k);
  double v[6] = {0, 0, 0, 0, 0, 0};
  const bool kin = k + g.k_off < g.nz_all;  // the edge or face along z lies inside the whole grid
  if (i < g.nx) v[kEX] = edge_minv(g, 0, i, j, k);
  if (j < g.ny) v[kEY] = edge_minv(g, 1, i, j, k);
  if (kin) v[kEZ] = edge_minv(g, 2, i, j, k);
  if (j < g.ny && kin) v[kHX] = face_minv(g, 0, i, j, k);
  if (i < g.nx && kin) v[kHY] = face_minv(g, 1, i, j, k);
  if (i < g.nx && j < g.ny) v[kHZ] = face_minv(g, 2, i, j, k);
  uint8_t m = 0;
  for (int c = 0; c < 6; ++c) {
    if (v[c] != 0.0) m |= (uint8_t)(1u << c);
    if (mo.a[c]) mo.a[c][id] = v[c];
  }
  mask[id] = m;
}

template <typename T>
__global__ void scale_coef(const double* minv, double s, long long n, T* out) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) out[q] = (T)(s * minv[q]);
}
// M = 1/M^-1 per entry (0 where M^-1 is 0: an entry without a field), for the
// balances, which would otherwise divide at every use
__global__ void recip_coef(const double* minv, long long n, double* out) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) out[q] = minv[q] != 0.0 ? 1.0 / minv[q] : 0.0;
}
// The same (recip) or s M^-1 as a (hi, lo) float32 pair whose sum is the
// float64 value to 2^-48, for the float32-pair balances
__global__ void pair_coef(const double* minv, double s, bool recip, long long n, float2* out) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double v = minv[q];
  const double x = recip ? (v != 0.0 ? 1.0 / v : 0.0) : s * v;
  const float hi = (float)x;
  out[q] = make_float2(hi, (float)(x - (double)hi));
}

// Canonical FIT layout <-> device layout, for planes [k0, k0 + nk).
template <typename T>
__global__ void to_canonical(const T* src, Layout L, int k0, int nk, double* dst) {
  const long long total = (long long)(L.nx + 1) * (L.ny + 1) * nk;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int i = (int)(q % (L.nx + 1));
  const int j = (int)((q / (L.nx + 1)) % (L.ny + 1));
  const int k = k0 + (int)(q / ((long long)(L.nx + 1) * (L.ny + 1)));
  dst[q] = (double)src[L.idx(i, j, k)];
}
template <typename T>
__global__ void from_canonical(const double* src, Layout L, int k0, int nk, const uint8_t* mask,
                               int comp, T* dst) {
  const long long total = (long long)(L.nx + 1) * (L.ny + 1) * nk;
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= total) return;
  const int i = (int)(q % (L.nx + 1));
  const int j = (int)((q / (L.nx + 1)) % (L.ny + 1));
  const int k = k0 + (int)(q / ((long long)(L.nx + 1) * (L.ny + 1)));
  const long long id = L.idx(i, j, k);
  dst[id] = ((mask[id] >> comp) & 1) ? (T)src[q] : T(0);
}

// Per fused work item (tile, z-chunk): the number of its own cells that
// carry a field (0: the item lies in PEC and is skipped).
__global__ void item_counts(const uint8_t* mask, Layout L, int tx, int ty, int cz, int tiles_x,
                            int tiles_y, int n_items, int* counts) {
  __shared__ int total;
  const int item = blockIdx.x;
  if (item >= n_items) return;
  if (threadIdx.x == 0) total = 0;
  __syncthreads();
  const int ntile = tiles_x * tiles_y;
  const int tile = item % ntile, chunk = item / ntile;
  const int i0 = (tile % tiles_x) * tx, j0 = (tile / tiles_x) * ty, k0 = chunk * cz;
  int c = 0;
  const int cells = tx * ty * cz;
  for (int q = threadIdx.x; q < cells; q += blockDim.x) {
    const int i = i0 + q % tx, j = j0 + (q / tx) % ty, k = k0 + q / (tx * ty);
    if (i < L.nx && j < L.ny && k < L.nz && mask[L.idx(i, j, k)] != 0) ++c;
  }
  atomicAdd(&total, c);
  __syncthreads();
  if (threadIdx.x == 0) counts[item] = total;
}

// Entries of one component that hold a non-zero value where the activity bit
// is clear: the guard ring around the cells and the entries of PEC objects,
// which every update leaves at zero (the canary of an out-of-place write).
template <typename T>
__global__ void guard_scan(const T* f, const uint8_t* mask, long long count, int comp,
                           unsigned long long* out) {
  unsigned long long c = 0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < count;
       q += (long long)gridDim.x * blockDim.x)
    if (f[q] != T(0) && !((mask[q] >> comp) & 1)) ++c;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void count_active(const uint8_t* mask, Layout L, unsigned long long* out) {
  const long long total = (long long)L.nx * L.ny * L.nz;
  unsigned long long c = 0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % L.nx), j = (int)((q / L.nx) % L.ny), k = (int)(q / ((long long)L.nx * L.ny));
    c += mask[L.idx(i, j, k)] != 0;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, c);
}

double phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

}  // namespace


namespace {

int cuda_fail(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return TETM_E_NOMEM;
  return TETM_E_CUDA;
}
#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_);  \
  } while (0)

int dalloc(tetm_solver* s, void** p, size_t bytes) {
  cudaError_t e = dev_alloc(p, bytes, s->stream);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return cuda_fail(e);
  }
  s->device_bytes += (long long)bytes;
  return TETM_OK;
}

bool grid_ok(const tetm_grid* g) {
  return g && g->nx >= 2 && g->ny >= 2 && g->nz >= 2 && g->dx > 0 && g->dy > 0 && g->dz > 0 &&
         g->cdt >= 0 && (g->precision == TETM_FP64 || g->precision == TETM_FP32) &&
         isfinite(g->dx) && isfinite(g->dy) && isfinite(g->dz) && isfinite(g->cdt) &&
         (long long)g->nx * g->ny < (1LL << 31) && (long long)(g->nx + 1) * (g->ny + 1) * (g->nz + 1) < (1LL << 40);
}

double cdt_of(const tetm_grid* g) { return g->cdt > 0 ? g->cdt : g->dz; }

}  // namespace

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64];
uint64_t g_pool_keep = 0;

cudaMemPool_t lib_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = g_pool_keep;
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = p;
  }
  return g_pool[dev];
}
}  // namespace

cudaError_t tetm::dev_alloc(void** p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  cudaMemPool_t pool = lib_pool();
  if (!pool) return cudaErrorMemoryAllocation;
  return cudaMallocFromPoolAsync(p, bytes ? bytes : 16, pool, st);
}

void tetm::dev_free(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

int tetm::rebuild_work(tetm_solver* s) {
  const Layout& L = s->L;
  s->tiles_x = (L.nx + s->tile_x - 1) / s->tile_x;
  s->tiles_y = (L.ny + s->tile_y - 1) / s->tile_y;
  s->n_chunks = (L.nz + s->chunk_z - 1) / s->chunk_z;
  const long long items = (long long)s->tiles_x * s->tiles_y * s->n_chunks;
  if (items >= (1LL << 31)) return TETM_E_ARG;
  if (s->work) {
    dev_free(s->work, s->stream);
    s->work = nullptr;
  }
  int* counts = nullptr;
  CK(dev_alloc((void**)&counts, sizeof(int) * (size_t)items, s->stream));
  item_counts<<<(unsigned)items, 256, 0, s->stream>>>(s->mask, L, s->tile_x, s->tile_y, s->chunk_z,
                                                      s->tiles_x, s->tiles_y, (int)items, counts);
  std::vector<int> h((size_t)items);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), counts, sizeof(int) * (size_t)items,
                                            cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  dev_free(counts, s->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  // the items that own a field-carrying cell, in grid order: items that run
  // at the same time are neighbours and share their halo rows through L2
  // (ordering the list by work instead was measured 1.3x slower)
  std::vector<int> list;
  list.reserve((size_t)items);
  for (long long q = 0; q < items; ++q)
    if (h[(size_t)q]) list.push_back((int)q);
  s->n_work = (int)list.size();
  s->work_host = list;
  if (3 * s->n_work > s->diag.cap) {  // balance reductions keep three partials per work item
    dev_free(s->diag.part, s->stream);
    s->diag.part = nullptr;
    s->diag.cap = 0;
    const int cap = std::max(2048, 3 * s->n_work);
    CK(dev_alloc((void**)&s->diag.part, sizeof(double) * (size_t)cap, s->stream));
    s->diag.cap = cap;
  }
  if (!list.empty()) {
    CK(dev_alloc((void**)&s->work, sizeof(int) * list.size(), s->stream));
    CK(cudaMemcpyAsync(s->work, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice,
                       s->stream));
    CK(cudaStreamSynchronize(s->stream));
  }
  s->work_dirty = false;
  return TETM_OK;
}

namespace {

}  // namespace

template <typename T>
StepArgs<T> tetm::step_args(tetm_solver* s, bool fused) {
  StepArgs<T> a;
  for (int c = 0; c < 6; ++c) {
    a.in[c] = (const T*)s->set[s->cur][c];
    a.out[c] = fused ? (T*)s->set[1 - s->cur][c] : (T*)s->set[s->cur][c];
    a.co.u[c] = (T)(((c == kEZ || c == kHZ) ? 2.0 * s->alpha : s->alpha) * s->minv_c[c]);
    a.co.ua[c] = (const T*)s->ua[c];
  }
  a.co.mask = s->mask;
  a.L = s->L;
  a.n = s->step;
  a.b.on = s->bunch ? 1 : 0;
  a.b.i0 = s->i0;
  a.b.j0 = s->j0;
  a.b.c0 = s->c0;
  a.b.kshift = s->kshift - s->k_lo;  // plane indices of the kernels are local to a z-slab
  a.b.m_min = s->m_min;
  a.b.m_max = s->m_max;
  a.b.inv_q = s->bunch ? 1.0 / s->q : 0.0;
  a.b.J = (const T*)s->J;
  a.b.W = s->W;
  {
    const int nw = s->bunch ? s->m_max - s->m_min + 1 : 0;
    const double eta0 = kMu0 * kC;
    a.b.obs_on = (s->bunch && s->obs_on) ? 1 : 0;
    a.b.obs_i = s->obs_i;
    a.b.obs_j = s->obs_j;
    a.b.WX = s->bunch ? s->W + nw : nullptr;
    a.b.WY = s->bunch ? s->W + 2 * nw : nullptr;
    const double iq = s->bunch ? 1.0 / s->q : 0.0;
    // E_x - c mu0 H_y and E_y + c mu0 H_x times dz/Q, with e = E * (edge
    // length) and h = H * (dual edge length): dy for h_y, dx for h_x
    a.b.tw_ex = s->g.dz * iq / s->g.dx;
    a.b.tw_hy = -eta0 * s->g.dz * iq / s->g.dy;
    a.b.tw_ey = s->g.dz * iq / s->g.dy;
    a.b.tw_hx = eta0 * s->g.dz * iq / s->g.dx;
  }
  a.tiles_x = s->tiles_x;
  a.tiles_y = s->tiles_y;
  a.chunk_z = s->chunk_z;
  a.n_chunks = s->n_chunks;
  a.work = s->work;
  a.n_work = s->n_work;
  return a;
}
template StepArgs<float> tetm::step_args<float>(tetm_solver*, bool);
template StepArgs<double> tetm::step_args<double>(tetm_solver*, bool);

namespace {

// Queue the FP64 balances of the step just taken into device slots:
// rec[0] = n, rec[1] = W^{n,e}, rec[2] = max|qe - qbunch|, rec[3] = max|qh|,
// rec[4] = max|qbunch|. No host synchronisation.
WorkView work_view(const tetm_solver* s) {
  WorkView v;
  v.items = s->work;
  v.n_items = s->n_work;
  v.tile_x = s->tile_x;
  v.tile_y = s->tile_y;
  v.chunk_z = s->chunk_z;
  v.tiles_x = s->tiles_x;
  v.tiles_y = s->tiles_y;
  return v;
}

template <typename T>
int queue_balances(tetm_solver* s, double* rec) {
  const double zc = ((double)(s->step + s->kshift - s->k_lo - 1) + 0.5 - s->c0) * s->g.dz;
  CK(launch_bunch_charge(s->bunch ? s->q : 0.0, s->bunch ? s->sigma : 1.0, s->g.dz, zc, s->g.nz,
                         s->qline, rec + 4, (double)s->step, rec, s->stream));
  const T *cur[6], *prv[6];
  const double *ma[6], *mr[6];
  for (int c = 0; c < 6; ++c) {
    cur[c] = (const T*)s->set[s->cur][c];
    prv[c] = (const T*)s->set[1 - s->cur][c];
    ma[c] = s->minv_a[c];
    mr[c] = s->m_a[c];
  }
  const WorkView wv = work_view(s);
  if constexpr (sizeof(T) == 4) {
    if (!s->uniform) {  // float32 fields, material arrays: one float32-pair pass
      CK(launch_balances_mat_f32((const float* const*)cur, (const float* const*)prv, s->mask, s->mp, s->ap, s->L,
                                 s->alpha, s->bunch ? s->qline : nullptr, s->i0, s->j0, wv, s->diag, rec + 1,
                                 rec + 2, rec + 3, s->stream));
      return TETM_OK;
    }
  }
  if (s->uniform) {  // one pass for both
    CK(launch_balances<T>(cur, prv, s->mask, s->minv_c, s->L, s->alpha, s->bunch ? s->qline : nullptr, s->i0,
                          s->j0, wv, s->diag, rec + 1, rec + 2, rec + 3, s->stream));
    return TETM_OK;
  }
  if constexpr (sizeof(T) == 8) {  // float64 fields, material arrays: two float64 passes
    CK(launch_energy<T>(cur, s->mask, s->minv_c, ma, mr, s->L, s->alpha, wv, s->diag, rec + 1, s->stream));
    CK(launch_charge<T>(cur, prv, s->mask, s->minv_c, ma, mr, s->L, s->alpha,
                        s->bunch ? s->qline : nullptr, s->i0, s->j0, wv, s->diag, rec + 2, rec + 3,
                        s->stream));
  }
  return TETM_OK;
}

// Yee's scheme (Eq. (7)): the fused launch (ping-pong) for one material,
// else the two in-place reference launches
template <typename T>
int do_yee_steps(tetm_solver* s, int n) {
  const bool fused = s->kernel == TETM_KERNEL_FUSED && s->uniform;
  for (int q = 0; q < n; ++q) {
    StepArgs<T> a = step_args<T>(s, fused);
    for (int c = 0; c < 6; ++c) a.co.u[c] = (T)(2.0 * s->alpha * s->minv_c[c]);  // dt M^-1
    a.b.on = 0;
    a.b.obs_on = 0;
    if (fused) {
      if (s->n_work > 0) CK(launch_yee_fused_step<T>(a, s->stream));
      s->cur = 1 - s->cur;
    } else {
      CK(launch_yee_reference_step<T>(a, s->stream));
    }
    s->step += 1;
  }
  return TETM_OK;
}

template <typename T>
int do_steps(tetm_solver* s, int n) {
  if (s->scheme == TETM_SCHEME_YEE) return do_yee_steps<T>(s, n);
  bool last_pair = false;
  for (int q = 0; q < n; ++q) {
    const bool bal = s->bal_every > 0 && (s->step + 1) % s->bal_every == 0;
    if (s->kernel == TETM_KERNEL_TWOSTEP) {
      // a pair of steps per launch, unless a balance or a transverse gather
      // falls after its first step or a balance after its second (it needs
      // the state before)
      const bool bal2 = s->bal_every > 0 && (s->step + 2) % s->bal_every == 0;
      StepArgs<T> a = step_args<T>(s, true);
      last_pair = q + 1 < n && !bal && !bal2 && !(s->bunch && s->obs_on);
      if (last_pair) {
        if (s->n_work > 0) CK(launch_fused_two_steps<T>(a, s->tile_x, s->tile_y, s->stream));
        s->cur = 1 - s->cur;
        s->step += 2;
        ++q;
        continue;
      }
      if (s->n_work > 0) CK(launch_fused_step<T>(a, s->tile_x, s->tile_y, s->stream));
      if (s->bunch && s->obs_on) CK(launch_transverse_after_step<T>(a, s->stream));
      s->cur = 1 - s->cur;
    } else if (s->kernel == TETM_KERNEL_FUSED) {
      StepArgs<T> a = step_args<T>(s, true);
      if (s->n_work > 0) {
        if (warp_shape_ok(s->tile_x, s->tile_y)) {
          CK(launch_fused_warp_step<T>(a, s->tile_x, s->tile_y, s->stream));
        } else if (slab_shape_ok(s->tile_x, s->tile_y, !s->uniform)) {
          if constexpr (sizeof(T) == 4) {
            CK(launch_fused_slab_step(a, s->sched, s->stream));
          } else {
            return TETM_E_UNSUPPORTED;
          }
        } else {
          CK(launch_fused_step<T>(a, s->tile_x, s->tile_y, s->stream));
        }
      }
      if (s->bunch && s->obs_on) CK(launch_transverse_after_step<T>(a, s->stream));
      s->cur = 1 - s->cur;
    } else {
      if (q == n - 1 || bal) {  // keep y^n beside y^{n+1} for the charge balance
        for (int c = 0; c < 6; ++c)
          CK(cudaMemcpyAsync(s->set[1 - s->cur][c], s->set[s->cur][c], (size_t)s->L.count * s->esz,
                             cudaMemcpyDeviceToDevice, s->stream));
      }
      StepArgs<T> a = step_args<T>(s, false);
      CK(launch_reference_step<T>(a, s->stream));
    }
    s->step += 1;
    if (bal) {
      double* rec = s->hist + 5 * (s->hist_count % s->hist_cap);
      int rc = queue_balances<T>(s, rec);
      if (rc) return rc;
      s->hist_count += 1;
    }
  }
  // after a pair the other field set holds the state two steps back
  if (n > 0) s->prev_valid = !last_pair;
  return TETM_OK;
}

int ensure_staging(tetm_solver* s) {
  if (s->staging) return TETM_OK;
  const long long plane = (long long)(s->L.nx + 1) * (s->L.ny + 1);
  long long nk = std::max(1LL, std::min((long long)s->L.nz + 1, (16LL << 20) / plane));
  s->staging_elems = nk * plane;
  return dalloc(s, (void**)&s->staging, sizeof(double) * (size_t)s->staging_elems);
}

template <typename T>
int get_fields_t(tetm_solver* s, int comp, double* host) {
  const long long plane = (long long)(s->L.nx + 1) * (s->L.ny + 1);
  const int nk_max = (int)(s->staging_elems / plane);
  for (int k0 = 0; k0 <= s->L.nz; k0 += nk_max) {
    const int nk = std::min(nk_max, s->L.nz + 1 - k0);
    const long long n = plane * nk;
    to_canonical<T><<<(unsigned)((n + 255) / 256), 256, 0, s->stream>>>(
        (const T*)s->set[s->cur][comp], s->L, k0, nk, s->staging);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(host + plane * k0, s->staging, sizeof(double) * (size_t)n,
                       cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
  }
  return TETM_OK;
}

template <typename T>
int set_fields_t(tetm_solver* s, int comp, const double* host) {
  const long long plane = (long long)(s->L.nx + 1) * (s->L.ny + 1);
  const int nk_max = (int)(s->staging_elems / plane);
  for (int k0 = 0; k0 <= s->L.nz; k0 += nk_max) {
    const int nk = std::min(nk_max, s->L.nz + 1 - k0);
    const long long n = plane * nk;
    CK(cudaMemcpyAsync(s->staging, host + plane * k0, sizeof(double) * (size_t)n,
                       cudaMemcpyHostToDevice, s->stream));
    from_canonical<T><<<(unsigned)((n + 255) / 256), 256, 0, s->stream>>>(
        s->staging, s->L, k0, nk, s->mask, comp, (T*)s->set[s->cur][comp]);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s->stream));
  }
  return TETM_OK;
}

// releases every device array of the solve, in the order of its stream
void free_all(tetm_solver* s) {
  cudaStream_t st = s->stream;
  for (int b = 0; b < 2; ++b)
    for (int c = 0; c < 6; ++c) dev_free(s->set[b][c], st);
  for (int c = 0; c < 6; ++c) {
    dev_free(s->minv_a[c], st);
    dev_free(s->m_a[c], st);
    dev_free(s->mp[c], st);
    dev_free(s->ap[c], st);
    dev_free(s->ua[c], st);
  }
  dev_free(s->mask, st);
  dev_free(s->work, st);
  dev_free(s->J, st);
  dev_free(s->W, st);
  dev_free(s->qline, st);
  dev_free(s->diag.part, st);
  dev_free(s->diag.out, st);
  dev_free(s->hist, st);
  dev_free(s->staging, st);
  dev_free(s->sched, st);
}

}  // namespace

extern "C" {

const char* tetm_strerror(int code) {
  switch (code) {
    case TETM_OK: return "ok";
    case TETM_E_ARG: return "bad argument";
    case TETM_E_UNSTABLE: return "time step violates the stability bound of Eq. (25)";
    case TETM_E_NOT_MAGIC: return "bunch and wake need c*dt == dz";
    case TETM_E_NOMEM: return "out of memory";
    case TETM_E_CUDA: return "CUDA runtime error";
    case TETM_E_STATE: return "call not valid in the current solver state";
    case TETM_E_TIMEOUT: return "bounded device wait timed out";
    case TETM_E_DIVERGED: return "energy is not finite: the run diverged";
    case TETM_E_UNSUPPORTED: return "unsupported option combination";
    case TETM_E_TOO_LARGE: return "grid larger than the fixed scratch of tetm_energy_noalloc";
    default: return "unknown error";
  }
}

int64_t tetm_bytes_needed(const tetm_grid* g) {
  if (!grid_ok(g)) return 0;
  const size_t esz = g->precision == TETM_FP64 ? 8 : 4;
  const Layout L = make_layout(g->nx, g->ny, g->nz, (int)esz);
  return (int64_t)(12 * esz + 1) * L.count + (int64_t)(1 << 20);
}

}  // extern "C"

namespace {

// A solve of planes [k_lo, k_lo + g->nz) of a grid of nz_all planes (the
// whole grid: k_lo = 0, nz_all = g->nz); the cell arrays cover the whole grid.
int create_impl(const tetm_grid* g, int k_lo, int nz_all, const double* eps_r, const double* mu_r,
                const uint8_t* pec, cudaStream_t st, tetm_solver** out) {
  if (!out) return TETM_E_ARG;
  *out = nullptr;
  if (!grid_ok(g)) return TETM_E_ARG;
  const double cdt = cdt_of(g);
  const double lim_t = 1.0 / sqrt(1.0 / (g->dx * g->dx) + 1.0 / (g->dy * g->dy));
  if (cdt > g->dz * (1.0 + 1e-12) || cdt > lim_t * (1.0 + 1e-12)) return TETM_E_UNSTABLE;
  const long long ncell = (long long)g->nx * g->ny * nz_all;
  // materials: physical (>= 1) and finite; uniform if every cell has the same value
  bool uniform = true;
  double eps_u = 1.0, mu_u = 1.0;
  for (int w = 0; w < 2; ++w) {
    const double* a = w == 0 ? eps_r : mu_r;
    if (!a) continue;
    for (long long q = 0; q < ncell; ++q)
      if (!(a[q] >= 1.0) || !isfinite(a[q])) return TETM_E_ARG;
    for (long long q = 1; q < ncell; ++q)
      if (a[q] != a[0]) { uniform = false; break; }
    (w == 0 ? eps_u : mu_u) = a[0];
  }
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
    cudaGetLastError();
    return TETM_E_CUDA;
  }
  tetm_solver* s = new (std::nothrow) tetm_solver();
  if (!s) return TETM_E_NOMEM;
  s->g = *g;
  s->g.cdt = cdt;
  s->k_lo = k_lo;
  s->nz_all = nz_all;
  s->esz = g->precision == TETM_FP64 ? 8 : 4;
  s->L = make_layout(g->nx, g->ny, g->nz, (int)s->esz);
  s->alpha = 0.5 * cdt / kC;
  s->stream = st;
  s->scheme = TETM_SCHEME_TETM;
  s->kernel = TETM_KERNEL_FUSED;
  s->uniform = uniform;
  s->vacuum = uniform && eps_u == 1.0 && mu_u == 1.0;
  // float32: the slab kernel (kernels_slab.cu; 56 x 12 tiles with
  // coefficient arrays); float64: the warp-tiled kernel (kernels_warp.cu)
  s->tile_x = s->esz == 4 ? 56 : 28;
  s->tile_y = s->esz == 4 ? (uniform ? 28 : 12) : 20;
  s->chunk_z = 32;
  int rc = TETM_OK;
  const size_t fbytes = (size_t)s->L.count * s->esz;
  for (int b = 0; b < 2 && rc == TETM_OK; ++b)
    for (int c = 0; c < 6 && rc == TETM_OK; ++c) {
      rc = dalloc(s, &s->set[b][c], fbytes);
      if (rc == TETM_OK) rc = cudaMemsetAsync(s->set[b][c], 0, fbytes, s->stream) == cudaSuccess ? TETM_OK : TETM_E_CUDA;
    }
  if (rc == TETM_OK) rc = dalloc(s, (void**)&s->mask, (size_t)s->L.count);
  if (rc == TETM_OK) rc = cudaMemsetAsync(s->mask, 0, (size_t)s->L.count, s->stream) == cudaSuccess ? TETM_OK : TETM_E_CUDA;
  if (rc == TETM_OK) rc = dalloc(s, (void**)&s->diag.part, sizeof(double) * 2048);
  if (rc == TETM_OK) rc = dalloc(s, (void**)&s->diag.out, sizeof(double) * 8);
  if (rc == TETM_OK) rc = dalloc(s, (void**)&s->sched, 2 * sizeof(int));
  if (rc == TETM_OK) rc = cudaMemsetAsync(s->sched, 0, 2 * sizeof(int), s->stream) == cudaSuccess ? TETM_OK : TETM_E_CUDA;
  s->diag.cap = 2048;
  s->hist_cap = 4096;
  if (rc == TETM_OK) rc = dalloc(s, (void**)&s->hist, sizeof(double) * 5 * (size_t)s->hist_cap);
  if (rc == TETM_OK) rc = dalloc(s, (void**)&s->qline, sizeof(double) * (size_t)(g->nz + 1));
  MinvOut mo;
  for (int c = 0; c < 6; ++c) mo.a[c] = nullptr;
  if (rc == TETM_OK && !uniform) {
    for (int c = 0; c < 6 && rc == TETM_OK; ++c) {
      rc = dalloc(s, (void**)&s->minv_a[c], sizeof(double) * (size_t)s->L.count);
      if (rc == TETM_OK) rc = cudaMemsetAsync(s->minv_a[c], 0, sizeof(double) * (size_t)s->L.count, s->stream) == cudaSuccess ? TETM_OK : TETM_E_CUDA;
      mo.a[c] = s->minv_a[c];
    }
  }
  // upload the cell arrays, build the mask (and M^-1 arrays) on the device
  GeomIn gi;
  gi.pec = nullptr;
  gi.eps = nullptr;
  gi.mu = nullptr;
  gi.nx = g->nx; gi.ny = g->ny; gi.nz = g->nz;
  gi.k_off = k_lo;
  gi.nz_all = nz_all;
  gi.dx = g->dx; gi.dy = g->dy; gi.dz = g->dz;
  uint8_t* dpec = nullptr;
  double *deps = nullptr, *dmu = nullptr;
  if (rc == TETM_OK && pec) {
    if (dev_alloc((void**)&dpec, (size_t)ncell, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(dpec, pec, (size_t)ncell, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
      rc = TETM_E_CUDA;
    gi.pec = dpec;
  }
  if (rc == TETM_OK && !uniform) {
    for (int w = 0; w < 2 && rc == TETM_OK; ++w) {
      const double* a = w == 0 ? eps_r : mu_r;
      if (!a) continue;
      double** d = w == 0 ? &deps : &dmu;
      if (dev_alloc((void**)d, sizeof(double) * (size_t)ncell, s->stream) != cudaSuccess ||
          cudaMemcpyAsync(*d, a, sizeof(double) * (size_t)ncell, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
        rc = TETM_E_CUDA;
    }
    gi.eps = deps;
    gi.mu = dmu;
  }
  if (rc == TETM_OK) {
    const int k_first = k_lo > 0 ? -1 : 0;  // a z-slab's ghost plane below takes the whole grid's geometry
    const long long total = (long long)(g->nx + 1) * (g->ny + 1) * (g->nz + 1 - k_first);
    build_geometry<<<(unsigned)((total + 255) / 256), 256, 0, s->stream>>>(gi, s->L, k_first, s->mask, mo);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s->stream) != cudaSuccess) rc = TETM_E_CUDA;
  }
  dev_free(dpec, s->stream);
  dev_free(deps, s->stream);
  dev_free(dmu, s->stream);
  // per-component constants for the uniform case (vacuum or one material)
  const double dx = g->dx, dy = g->dy, dz = g->dz;
  s->minv_c[kEX] = dx / (kEps0 * eps_u * dy * dz);
  s->minv_c[kEY] = dy / (kEps0 * eps_u * dx * dz);
  s->minv_c[kEZ] = dz / (kEps0 * eps_u * dx * dy);
  s->minv_c[kHX] = dx / (kMu0 * mu_u * dy * dz);
  s->minv_c[kHY] = dy / (kMu0 * mu_u * dx * dz);
  s->minv_c[kHZ] = dz / (kMu0 * mu_u * dx * dy);
  if (rc == TETM_OK && !uniform) {
    for (int c = 0; c < 6 && rc == TETM_OK; ++c) {
      rc = dalloc(s, &s->ua[c], (size_t)s->L.count * s->esz);
      if (rc != TETM_OK) break;
      const double sc = (c == kEZ || c == kHZ) ? 2.0 * s->alpha : s->alpha;
      const unsigned nb = (unsigned)((s->L.count + 255) / 256);
      // the balances' coefficients: M (and alpha^2 M^-1 of the four
      // transverse components) as float32 pairs for float32 fields, M in
      // float64 for float64 fields
      if (s->esz == 4) {
        const bool a2 = c == kHX || c == kHY || c == kEX || c == kEY;
        rc = dalloc(s, (void**)&s->mp[c], sizeof(float2) * (size_t)s->L.count);
        if (rc == TETM_OK && a2) rc = dalloc(s, (void**)&s->ap[c], sizeof(float2) * (size_t)s->L.count);
        if (rc != TETM_OK) break;
        pair_coef<<<nb, 256, 0, s->stream>>>(s->minv_a[c], 0.0, true, s->L.count, s->mp[c]);
        if (a2) pair_coef<<<nb, 256, 0, s->stream>>>(s->minv_a[c], s->alpha * s->alpha, false, s->L.count, s->ap[c]);
      } else {
        rc = dalloc(s, (void**)&s->m_a[c], sizeof(double) * (size_t)s->L.count);
        if (rc != TETM_OK) break;
        recip_coef<<<nb, 256, 0, s->stream>>>(s->minv_a[c], s->L.count, s->m_a[c]);
      }
      if (s->esz == 8)
        scale_coef<double><<<nb, 256, 0, s->stream>>>(s->minv_a[c], sc, s->L.count, (double*)s->ua[c]);
      else
        scale_coef<float><<<nb, 256, 0, s->stream>>>(s->minv_a[c], sc, s->L.count, (float*)s->ua[c]);
      if (cudaGetLastError() != cudaSuccess) rc = TETM_E_CUDA;
    }
  }
  if (rc == TETM_OK) {
    unsigned long long* cnt = nullptr;
    unsigned long long h = 0;
    if (dev_alloc((void**)&cnt, sizeof(*cnt), s->stream) != cudaSuccess) rc = TETM_E_CUDA;
    if (rc == TETM_OK) {
      cudaMemsetAsync(cnt, 0, sizeof(*cnt), s->stream);
      count_active<<<256, 256, 0, s->stream>>>(s->mask, s->L, cnt);
      if (cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
          cudaStreamSynchronize(s->stream) != cudaSuccess)
        rc = TETM_E_CUDA;
      dev_free(cnt, s->stream);
    }
    s->active_cells = (long long)h;
  }
  if (rc == TETM_OK) rc = rebuild_work(s);
  if (rc != TETM_OK) {
    free_all(s);
    delete s;
    cudaGetLastError();
    return rc;
  }
  *out = s;
  return TETM_OK;
}

}  // namespace

extern "C" {

int tetm_create(const tetm_grid* g, const double* eps_r, const double* mu_r, const uint8_t* pec,
                tetm_solver** out) {
  return create_impl(g, 0, g ? g->nz : 0, eps_r, mu_r, pec, nullptr, out);
}

int tetm_create_on_stream(const tetm_grid* g, const double* eps_r, const double* mu_r, const uint8_t* pec,
                          void* stream, tetm_solver** out) {
  return create_impl(g, 0, g ? g->nz : 0, eps_r, mu_r, pec, (cudaStream_t)stream, out);
}

int tetm_pool_reserve(uint64_t bytes) {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  g_pool_keep = bytes;
  for (cudaMemPool_t p : g_pool)
    if (p && cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &bytes) != cudaSuccess) {
      cudaGetLastError();
      return TETM_E_CUDA;
    }
  return TETM_OK;
}

int tetm_create_slab(const tetm_grid* g, int32_t k_lo, int32_t k_hi, const double* eps_r, const double* mu_r,
                     const uint8_t* pec, tetm_solver** out) {
  if (!out) return TETM_E_ARG;
  *out = nullptr;
  if (!g || k_lo < 0 || k_hi > g->nz || k_hi - k_lo < 2) return TETM_E_ARG;
  tetm_grid local = *g;
  local.nz = k_hi - k_lo;
  return create_impl(&local, k_lo, g->nz, eps_r, mu_r, pec, nullptr, out);
}

void tetm_destroy(tetm_solver* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream); else cudaDeviceSynchronize();
  free_all(s);
  delete s;
}

int tetm_set_stream(tetm_solver* s, void* st) {
  if (!s) return TETM_E_ARG;
  s->stream = (cudaStream_t)st;
  return TETM_OK;
}

int tetm_set_kernel(tetm_solver* s, int32_t kernel) {
  if (!s || (kernel != TETM_KERNEL_FUSED && kernel != TETM_KERNEL_REFERENCE && kernel != TETM_KERNEL_TWOSTEP))
    return TETM_E_ARG;
  if (s->in_batch) return TETM_E_STATE;
  if (kernel == TETM_KERNEL_TWOSTEP &&
      (!s->uniform || s->is_slab() || s->scheme != TETM_SCHEME_TETM || !fused2_shape_ok(s->tile_x, s->tile_y)))
    return TETM_E_UNSUPPORTED;
  if (kernel == TETM_KERNEL_REFERENCE && s->is_slab()) return TETM_E_UNSUPPORTED;  // it updates ghost planes in place
  // (Yee's scheme runs material arrays on the reference updates whatever the kernel)
  if (kernel == TETM_KERNEL_FUSED && !s->uniform && s->tile_x != 28 && !slab_shape_ok(s->tile_x, s->tile_y, true) &&
      s->scheme == TETM_SCHEME_TETM)
    return TETM_E_UNSUPPORTED;
  s->kernel = kernel;
  return TETM_OK;
}

int tetm_set_tiling(tetm_solver* s, int32_t tile_x, int32_t tile_y, int32_t chunk_z) {
  if (!s) return TETM_E_ARG;
  if (s->in_batch) return TETM_E_STATE;
  const int tx = tile_x ? tile_x : s->tile_x;
  const int ty = tile_y ? tile_y : s->tile_y;
  const int cz = chunk_z ? chunk_z : s->chunk_z;
  if (s->scheme == TETM_SCHEME_YEE) {  // Yee's fused kernel has one tile shape
    if (tx != s->tile_x || ty != s->tile_y) return TETM_E_UNSUPPORTED;
    if (cz < 4) return TETM_E_ARG;
    s->chunk_z = cz;
    return rebuild_work(s);
  }
  const bool slab_u = slab_shape_ok(tx, ty, false), slab_m = slab_shape_ok(tx, ty, true);
  if ((!fused_shape_ok(tx, ty) && !warp_shape_ok(tx, ty) && !slab_u && !slab_m) || cz < 4)
    return TETM_E_ARG;
  // per-entry coefficients (general materials) run on the warp-tiled kernel
  // and on the slab kernel's 56 x 12 tiles; one material on its 56 x 28 tiles
  if (!s->uniform && tx != 28 && !slab_m && s->kernel == TETM_KERNEL_FUSED)
    return TETM_E_UNSUPPORTED;
  if (s->uniform && slab_m && !slab_u) return TETM_E_UNSUPPORTED;
  // the slab kernel is float32 only
  if ((slab_u || slab_m) && s->esz != 4) return TETM_E_UNSUPPORTED;
  if (s->kernel == TETM_KERNEL_TWOSTEP && !fused2_shape_ok(tx, ty)) return TETM_E_UNSUPPORTED;
  if (tx == s->tile_x && ty == s->tile_y && cz == s->chunk_z && s->work) return TETM_OK;
  s->tile_x = tx;
  s->tile_y = ty;
  s->chunk_z = cz;
  return rebuild_work(s);
}

int tetm_set_scheme(tetm_solver* s, int32_t scheme) {
  if (!s || (scheme != TETM_SCHEME_TETM && scheme != TETM_SCHEME_YEE)) return TETM_E_ARG;
  if (scheme == s->scheme) return TETM_OK;
  if (s->is_slab() || s->kernel == TETM_KERNEL_TWOSTEP) return TETM_E_UNSUPPORTED;
  if (s->step != 0 || s->bunch || s->in_batch || s->bal_every > 0) return TETM_E_STATE;
  if (scheme == TETM_SCHEME_YEE) {
    const double dx = s->g.dx, dy = s->g.dy, dz = s->g.dz;
    const double lim = 1.0 / sqrt(1.0 / (dx * dx) + 1.0 / (dy * dy) + 1.0 / (dz * dz));  // Eq. (8)
    if (s->g.cdt > lim * (1.0 + 1e-12)) return TETM_E_UNSTABLE;
    yee_shape((int)s->esz, &s->tile_x, &s->tile_y);
  } else {  // the TE/TM scheme's default work shape
    s->tile_x = s->esz == 4 ? 56 : 28;
    s->tile_y = s->esz == 4 ? (s->uniform ? 28 : 12) : 20;
  }
  s->scheme = scheme;
  return rebuild_work(s);
}

int tetm_set_bunch(tetm_solver* s, double sigma_z, double charge, int32_t i0, int32_t j0) {
  if (!s || !(sigma_z > 0) || !isfinite(sigma_z) || charge == 0 || !isfinite(charge)) return TETM_E_ARG;
  if (i0 < 1 || i0 > s->g.nx - 1 || j0 < 1 || j0 > s->g.ny - 1) return TETM_E_ARG;
  if (s->scheme == TETM_SCHEME_YEE) return TETM_E_UNSUPPORTED;
  if (fabs(s->g.cdt - s->g.dz) > 1e-12 * s->g.dz) return TETM_E_NOT_MAGIC;
  if (s->step != 0 || s->bunch) return TETM_E_STATE;
  const double dz = s->g.dz;
  const int c0 = (int)ceil(5.0 * sigma_z / dz - 1e-12);
  const int m_max = (int)ceil(15.0 * sigma_z / dz - 1e-12);
  if (c0 < 1 || c0 > (1 << 20)) return TETM_E_ARG;
  std::vector<double> qc((size_t)(2 * c0));
  for (int d = -c0; d < c0; ++d) {
    const double lo = std::max((double)d * dz, -5.0 * sigma_z);
    const double hi = std::min((double)(d + 1) * dz, 5.0 * sigma_z);
    qc[(size_t)(d + c0)] = hi > lo ? charge * (phi(hi / sigma_z) - phi(lo / sigma_z)) : 0.0;
  }
  const int nw = m_max + c0 + 2;
  void* J = nullptr;
  double* W = nullptr;
  if (dev_alloc(&J, s->esz * qc.size(), s->stream) != cudaSuccess ||
      dev_alloc((void**)&W, 3 * sizeof(double) * nw, s->stream) != cudaSuccess) {
    dev_free(J, s->stream);
    dev_free(W, s->stream);
    cudaGetLastError();
    return TETM_E_NOMEM;
  }
  // J from a host vector that lives until the stream has read it (the
  // synchronisation below), all on the solve's stream
  int rc = TETM_OK;
  std::vector<double> j64;
  std::vector<float> j32;
  cudaError_t e = cudaSuccess;
  if (s->esz == 8) {
    j64.resize(qc.size());
    for (size_t q = 0; q < qc.size(); ++q) j64[q] = kC * qc[q] / dz;
    e = cudaMemcpyAsync(J, j64.data(), sizeof(double) * j64.size(), cudaMemcpyHostToDevice, s->stream);
  } else {
    j32.resize(qc.size());
    for (size_t q = 0; q < qc.size(); ++q) j32[q] = (float)(kC * qc[q] / dz);
    e = cudaMemcpyAsync(J, j32.data(), sizeof(float) * j32.size(), cudaMemcpyHostToDevice, s->stream);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(W, 0, 3 * sizeof(double) * nw, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) rc = TETM_E_CUDA;
  if (rc != TETM_OK) {
    dev_free(J, s->stream);
    dev_free(W, s->stream);
    cudaGetLastError();
    return rc;
  }
  s->J = J;
  s->W = W;
  s->device_bytes += (long long)(s->esz * qc.size() + 3 * sizeof(double) * nw);
  s->qcell = qc;
  s->bunch = true;
  s->i0 = i0;
  s->j0 = j0;
  s->obs_on = false;
  s->obs_i = i0;
  s->obs_j = j0;
  s->c0 = c0;
  s->m_min = -c0 - 1;
  s->m_max = m_max;
  s->sigma = sigma_z;
  s->q = charge;
  return TETM_OK;
}

int tetm_step(tetm_solver* s, int32_t n) {
  if (!s || n < 0) return TETM_E_ARG;
  if (s->in_batch) return TETM_E_STATE;
  if (s->kernel == TETM_KERNEL_FUSED && s->work_dirty) {
    int rc = rebuild_work(s);
    if (rc) return rc;
  }
  nvtxRangePushA("tetm_step");  // a range in a profiler's timeline (no cost without one)
  const int rc = s->esz == 8 ? do_steps<double>(s, n) : do_steps<float>(s, n);
  nvtxRangePop();
  return rc;
}

int tetm_sync(tetm_solver* s) {
  if (!s) return TETM_E_ARG;
  CK(cudaStreamSynchronize(s->stream));
  return TETM_OK;
}

int tetm_wake(tetm_solver* s, double* out, int32_t cap, int32_t* n_out, double* s0, double* ds) {
  if (!s) return TETM_E_ARG;
  if (!s->bunch) return TETM_E_STATE;
  const int nw = s->m_max - s->m_min + 1;
  if (n_out) *n_out = nw;
  if (s0) *s0 = s->m_min * s->g.dz;
  if (ds) *ds = s->g.dz;
  if (out) {
    if (cap < nw) return TETM_E_ARG;
    CK(cudaMemcpyAsync(out, s->W, sizeof(double) * nw, cudaMemcpyDeviceToHost, s->stream));
  }
  CK(cudaStreamSynchronize(s->stream));
  return TETM_OK;
}

int tetm_set_observer(tetm_solver* s, int32_t i, int32_t j) {
  if (!s) return TETM_E_ARG;
  if (s->in_batch || !s->bunch || s->step != 0) return TETM_E_STATE;
  if (i < 0 || i > s->g.nx - 1 || j < 0 || j > s->g.ny - 1) return TETM_E_ARG;
  s->obs_on = true;
  s->obs_i = i;
  s->obs_j = j;
  return TETM_OK;
}

int tetm_transverse_wake(tetm_solver* s, double* wx, double* wy, int32_t cap, int32_t* n_out, double* s0,
                         double* ds) {
  if (!s) return TETM_E_ARG;
  if (!s->bunch || !s->obs_on) return TETM_E_STATE;
  const int nw = s->m_max - s->m_min + 1;
  if (n_out) *n_out = nw;
  if (s0) *s0 = s->m_min * s->g.dz;
  if (ds) *ds = s->g.dz;
  if ((wx || wy) && cap < nw) return TETM_E_ARG;
  if (wx) CK(cudaMemcpyAsync(wx, s->W + nw, sizeof(double) * nw, cudaMemcpyDeviceToHost, s->stream));
  if (wy) CK(cudaMemcpyAsync(wy, s->W + 2 * nw, sizeof(double) * nw, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return TETM_OK;
}

int tetm_energy(tetm_solver* s, double* w) {
  if (!s || !w) return TETM_E_ARG;
  if (s->scheme != TETM_SCHEME_TETM) return TETM_E_UNSUPPORTED;
  const double *ma[6], *mr[6];
  for (int c = 0; c < 6; ++c) {
    ma[c] = s->minv_a[c];
    mr[c] = s->m_a[c];
  }
  cudaError_t e;
  if (s->esz == 8) {
    const double* f[6];
    for (int c = 0; c < 6; ++c) f[c] = (const double*)s->set[s->cur][c];
    e = s->uniform ? launch_balances<double>(f, nullptr, s->mask, s->minv_c, s->L, s->alpha, nullptr, 0, 0,
                                             work_view(s), s->diag, s->diag.out, nullptr, nullptr, s->stream)
                   : launch_energy<double>(f, s->mask, s->minv_c, ma, mr, s->L, s->alpha, work_view(s), s->diag,
                                           s->diag.out, s->stream);
  } else {
    const float* f[6];
    for (int c = 0; c < 6; ++c) f[c] = (const float*)s->set[s->cur][c];
    e = s->uniform ? launch_balances<float>(f, nullptr, s->mask, s->minv_c, s->L, s->alpha, nullptr, 0, 0,
                                            work_view(s), s->diag, s->diag.out, nullptr, nullptr, s->stream)
                   : launch_balances_mat_f32(f, nullptr, s->mask, s->mp, s->ap, s->L, s->alpha, nullptr, 0, 0,
                                             work_view(s), s->diag, s->diag.out, nullptr, nullptr, s->stream);
  }
  CK(e);
  CK(cudaMemcpyAsync(w, s->diag.out, sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return isfinite(*w) ? TETM_OK : TETM_E_DIVERGED;
}

int tetm_charge_residual(tetm_solver* s, double* max_e, double* max_h, double* q_scale) {
  if (!s) return TETM_E_ARG;
  if (s->scheme != TETM_SCHEME_TETM) return TETM_E_UNSUPPORTED;
  if (!s->prev_valid || s->step < 1) return TETM_E_STATE;
  int rc = s->esz == 8 ? queue_balances<double>(s, s->diag.out) : queue_balances<float>(s, s->diag.out);
  if (rc) return rc;
  double h[5];
  CK(cudaMemcpyAsync(h, s->diag.out, sizeof(h), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (max_e) *max_e = h[2];
  if (max_h) *max_h = h[3];
  if (q_scale) *q_scale = h[4];
  return TETM_OK;
}

int tetm_set_balance_every(tetm_solver* s, int32_t every) {
  if (!s || every < 0) return TETM_E_ARG;
  // a z-slab's ghost planes of the new state arrive only with the next exchange
  if (every > 0 && s->is_slab()) return TETM_E_UNSUPPORTED;
  if (every > 0 && s->scheme != TETM_SCHEME_TETM) return TETM_E_UNSUPPORTED;
  s->bal_every = every;
  return TETM_OK;
}

int tetm_balance_history(tetm_solver* s, double* out, int32_t cap, int32_t* n_out) {
  if (!s) return TETM_E_ARG;
  const long long n = std::min<long long>(s->hist_count, s->hist_cap);
  if (n_out) *n_out = (int32_t)n;
  if (out && n > 0) {
    if (cap < n) return TETM_E_ARG;
    std::vector<double> h((size_t)(5 * s->hist_cap));
    CK(cudaMemcpyAsync(h.data(), s->hist, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    const long long first = s->hist_count - n;
    for (long long r = 0; r < n; ++r) {
      const long long slot = (first + r) % s->hist_cap;
      memcpy(out + 5 * r, h.data() + 5 * slot, 5 * sizeof(double));
    }
  } else {
    CK(cudaStreamSynchronize(s->stream));
  }
  return TETM_OK;
}

int tetm_get_fields(tetm_solver* s, int32_t comp, double* host) {
  if (!s || !host || comp < 0 || comp > 5) return TETM_E_ARG;
  int rc = ensure_staging(s);
  if (rc) return rc;
  return s->esz == 8 ? get_fields_t<double>(s, comp, host) : get_fields_t<float>(s, comp, host);
}

int tetm_set_fields(tetm_solver* s, int32_t comp, const double* host) {
  if (!s || !host || comp < 0 || comp > 5) return TETM_E_ARG;
  if (s->in_batch) return TETM_E_STATE;
  int rc = ensure_staging(s);
  if (rc) return rc;
  rc = s->esz == 8 ? set_fields_t<double>(s, comp, host) : set_fields_t<float>(s, comp, host);
  s->prev_valid = false;
  return rc;
}

int tetm_check_guards(tetm_solver* s, int64_t* violations) {
  if (!s || !violations) return TETM_E_ARG;
  unsigned long long* cnt = nullptr;
  unsigned long long h = 0;
  CK(dev_alloc((void**)&cnt, sizeof(*cnt), s->stream));
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(*cnt), s->stream);
  for (int b = 0; b < 2 && e == cudaSuccess; ++b)
    for (int c = 0; c < 6 && e == cudaSuccess; ++c) {
      if (s->esz == 8)
        guard_scan<double><<<1024, 256, 0, s->stream>>>((const double*)s->set[b][c], s->mask, s->L.count, c, cnt);
      else
        guard_scan<float><<<1024, 256, 0, s->stream>>>((const float*)s->set[b][c], s->mask, s->L.count, c, cnt);
      e = cudaGetLastError();
    }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  dev_free(cnt, s->stream);
  CK(e);
  *violations = (int64_t)h;
  return TETM_OK;
}

int64_t tetm_plane_bytes(tetm_solver* s, int32_t dir) {
  if (!s || (dir != TETM_PLANES_UP && dir != TETM_PLANES_DOWN)) return 0;
  return (int64_t)(dir == TETM_PLANES_UP ? 6 : 2) * s->L.sz * (int64_t)s->esz;
}

int tetm_export_plane(tetm_solver* s, int32_t dir, void* buf) {
  if (!s || !buf || (dir != TETM_PLANES_UP && dir != TETM_PLANES_DOWN)) return TETM_E_ARG;
  if (s->scheme != TETM_SCHEME_TETM || s->in_batch) return TETM_E_STATE;
  const size_t pb = (size_t)s->L.sz * s->esz;
  // up: every component of the last plane the solve owns; down: e_x, e_y of its first
  const int k = dir == TETM_PLANES_UP ? s->L.nz - 1 : 0;
  const int comps[6] = {kEX, kEY, kEZ, kHX, kHY, kHZ};
  const int nc = dir == TETM_PLANES_UP ? 6 : 2;
  char* p = static_cast<char*>(buf);
  for (int q = 0; q < nc; ++q) {
    const char* src = static_cast<const char*>(s->set[s->cur][comps[q]]) + (size_t)(k + 1) * pb;
    CK(cudaMemcpyAsync(p + q * pb, src, pb, cudaMemcpyDefault, s->stream));
  }
  return TETM_OK;
}

int tetm_import_plane(tetm_solver* s, int32_t dir, const void* buf) {
  if (!s || !buf || (dir != TETM_PLANES_UP && dir != TETM_PLANES_DOWN)) return TETM_E_ARG;
  if (s->scheme != TETM_SCHEME_TETM || s->in_batch) return TETM_E_STATE;
  // a message moving up fills the ghost plane below the first owned plane
  // (needs a neighbour below: k_lo > 0); one moving down fills e_x, e_y of
  // the plane above the last owned one (needs a neighbour above)
  if (dir == TETM_PLANES_UP ? s->k_lo == 0 : s->k_lo + s->L.nz >= s->nz_all) return TETM_E_STATE;
  const size_t pb = (size_t)s->L.sz * s->esz;
  const int k = dir == TETM_PLANES_UP ? -1 : s->L.nz;
  const int comps[6] = {kEX, kEY, kEZ, kHX, kHY, kHZ};
  const int nc = dir == TETM_PLANES_UP ? 6 : 2;
  const char* p = static_cast<const char*>(buf);
  for (int q = 0; q < nc; ++q) {
    char* dst = static_cast<char*>(s->set[s->cur][comps[q]]) + (size_t)(k + 1) * pb;
    CK(cudaMemcpyAsync(dst, p + q * pb, pb, cudaMemcpyDefault, s->stream));
  }
  return TETM_OK;
}

int tetm_get_info(tetm_solver* s, tetm_info* info) {
  if (!s || !info) return TETM_E_ARG;
  memset(info, 0, sizeof(*info));
  info->step = s->step;
  info->device_bytes = s->device_bytes;
  info->active_cells = s->active_cells;
  info->processed_cells = (long long)s->n_work * s->tile_x * s->tile_y * s->chunk_z;
  info->kernel = s->kernel;
  info->precision = s->g.precision;
  info->tile_x = s->tile_x;
  info->tile_y = s->tile_y;
  info->chunk_z = s->chunk_z;
  info->work_items = s->n_work;
  info->wake_len = s->bunch ? s->m_max - s->m_min + 1 : 0;
  info->uniform_material = s->uniform ? 1 : 0;
  return TETM_OK;
}

// Checkpoint format: a fixed header, the six arrays of the current state in
// the device layout, then the wake accumulators.
struct CkptHeader {
  char magic[8];
  int32_t nx, ny, nz, precision;
  double dx, dy, dz, cdt;
  int64_t step;
  int64_t count;
  int32_t bunch, nw;
  int64_t kshift;
  int32_t obs_i, obs_j;
};

int tetm_save(tetm_solver* s, void* buf, size_t cap, size_t* used) {
  if (!s) return TETM_E_ARG;
  if (s->scheme != TETM_SCHEME_TETM) return TETM_E_UNSUPPORTED;
  const int nw = s->bunch ? s->m_max - s->m_min + 1 : 0;
  const size_t fb = (size_t)s->L.count * s->esz;
  const size_t need = sizeof(CkptHeader) + 6 * fb + 3 * sizeof(double) * (size_t)nw;
  if (used) *used = need;
  if (!buf) return TETM_OK;
  if (cap < need) return TETM_E_ARG;
  CkptHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, "TETMCKP3", 8);
  h.nx = s->g.nx; h.ny = s->g.ny; h.nz = s->g.nz; h.precision = s->g.precision;
  h.dx = s->g.dx; h.dy = s->g.dy; h.dz = s->g.dz; h.cdt = s->g.cdt;
  h.step = s->step;
  h.count = s->L.count;
  h.bunch = s->bunch;
  h.nw = nw;
  h.kshift = s->kshift;
  h.obs_i = (s->bunch && s->obs_on) ? s->obs_i : -1;  // -1: no transverse wake
  h.obs_j = (s->bunch && s->obs_on) ? s->obs_j : -1;
  char* p = (char*)buf;
  memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  for (int c = 0; c < 6; ++c, p += fb)
    CK(cudaMemcpyAsync(p, s->set[s->cur][c], fb, cudaMemcpyDeviceToHost, s->stream));
  if (nw) CK(cudaMemcpyAsync(p, s->W, 3 * sizeof(double) * nw, cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return TETM_OK;
}

int tetm_load(tetm_solver* s, const void* buf, size_t size) {
  if (!s || !buf || size < sizeof(CkptHeader)) return TETM_E_ARG;
  if (s->scheme != TETM_SCHEME_TETM) return TETM_E_UNSUPPORTED;
  if (s->in_batch) return TETM_E_STATE;
  CkptHeader h;
  memcpy(&h, buf, sizeof(h));
  const int nw = s->bunch ? s->m_max - s->m_min + 1 : 0;
  const size_t fb = (size_t)s->L.count * s->esz;
  if (memcmp(h.magic, "TETMCKP3", 8) != 0 || h.nx != s->g.nx || h.ny != s->g.ny || h.nz != s->g.nz ||
      h.precision != s->g.precision || h.count != s->L.count || h.bunch != (int)s->bunch || h.nw != nw ||
      h.dx != s->g.dx || h.dy != s->g.dy || h.dz != s->g.dz || h.cdt != s->g.cdt ||
      h.kshift != s->kshift)
    return TETM_E_ARG;
  const int oi = (s->bunch && s->obs_on) ? s->obs_i : -1, oj = (s->bunch && s->obs_on) ? s->obs_j : -1;
  if (h.obs_i != oi || h.obs_j != oj) return TETM_E_ARG;
  if (size < sizeof(CkptHeader) + 6 * fb + 3 * sizeof(double) * (size_t)nw) return TETM_E_ARG;
  const char* p = (const char*)buf + sizeof(h);
  for (int c = 0; c < 6; ++c, p += fb)
    CK(cudaMemcpyAsync(s->set[s->cur][c], p, fb, cudaMemcpyHostToDevice, s->stream));
  if (nw) CK(cudaMemcpyAsync(s->W, p, 3 * sizeof(double) * nw, cudaMemcpyHostToDevice, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  s->step = h.step;
  s->prev_valid = false;
  return TETM_OK;
}

}  // extern "C"
