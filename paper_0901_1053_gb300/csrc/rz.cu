// Rotationally symmetric explicit TE/TM scheme (Sec. 4.3, Eq. (24)): a set of
// azimuthal modes advanced together on one (r, z) grid, with a ring bunch and
// the wake of every mode.
//
// Device layout. Every per-entry array (fields of one component of one mode,
// mask) has rows k = -1..nz+1 and, per row, entries i = -or..pr-or-1 with the
// axis i = 0 at column `or`; entry (i, k) of the canonical layout sits at
// (k+1)*pr + i + or. Entries outside 0..nr, 0..nz hold zero and are
// inactive, so the stencils and prefetches read them without bounds checks.
// Field sets: [mode][component][row][column], two sets (ping-pong).
//
// Metric. In the vacuum staircase geometry every coefficient depends on r
// alone: per mode and radial index the kernel keeps alpha*M^-1 of e_r, e_phi,
// h_r, h_phi, 2 alpha*M^-1 of e_z, h_z and the two diagonal factors of
// (24) in registers; one activity byte per entry (shared by all modes) says
// which objects are non-PEC.
//
// Kernel. One warp per (mode, radial tile of 28 entries, z chunk) item; the
// 32 lanes cover the tile and two halo entries on each side, which is what
// the r-differences of the ten updates reach. The warp marches through the
// chunk plane by plane: at plane k it completes the TM stage (h_phi, h_r,
// e_z) with the old e of plane k+1 and then the TE stage (e_phi, e_r, h_z)
// with the new h of planes k-1 and k, so each plane is read once and written
// once. The TM stage of the plane before the chunk is recomputed (not
// written) to supply h^{n+1/2} at k0-1. Loads of the next planes are held in
// a register ring.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "tetm_internal.h"
#include "tetm_rz.h"

namespace {

using tetm::kC;
using tetm::kEps0;
using tetm::kMu0;

constexpr int kER = TETM_RZ_ER, kEP = TETM_RZ_EPHI, kEZ = TETM_RZ_EZ;
constexpr int kHR = TETM_RZ_HR, kHP = TETM_RZ_HPHI, kHZ = TETM_RZ_HZ;
constexpr double kPi = 3.14159265358979323846;
constexpr int kTile = 28;  // entries a warp owns
constexpr int kRing = 4;   // planes prefetched into registers
// per-mode coefficient rows: alpha M^-1 (er, ephi, hr, hphi), 2 alpha M^-1
// (ez, hz), and the diagonal factors 2 alpha M^-1 / (1 + alpha^2 m^2 M^-1 M^-1)
// of e_z (paired with h_r) and h_z (paired with e_r)
enum { kCoER = 0, kCoEP, kCoEZ, kCoHR, kCoHP, kCoHZ, kCoFEZ, kCoFHZ, kNCo };

struct RzLayout {
  int nr, nz, orr;
  long long pr;     // row pitch (elements)
  long long rows;   // nz + 3
  long long cs;     // elements per array, rows * pr
  __host__ __device__ __forceinline__ long long idx(int i, int k) const {
    return (long long)(k + 1) * pr + i + orr;
  }
};

RzLayout make_rz_layout(int nr, int nz, int esz) {
  RzLayout L;
  L.nr = nr;
  L.nz = nz;
  L.orr = 16 / esz;
  const long long al = 32 / esz;
  L.pr = (L.orr + nr + 3 + al - 1) / al * al;
  L.rows = nz + 3;
  L.cs = L.rows * L.pr;
  return L;
}

template <typename T>
struct RzArgs {
  const T* in;
  T* out;
  RzLayout L;
  const uint8_t* mask;
  const T* coef;          // [mode][kNCo][pr]
  int m_lo, n_modes;
  int tiles, chunk_z;
  const int* work;        // active (chunk * tiles + tile)
  int n_work;
  int b_on, i0, c0, m_min, nw;
  long long n;            // step being taken (n -> n+1)
  const T* J;             // [mode][2 c0]: share * c * Q_cell / dz
  double* W;              // [mode][nw]
  double inv_q;
};

template <typename T>
__device__ __forceinline__ T shfl_dn(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }
template <typename T>
__device__ __forceinline__ T shfl_up(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }

__device__ __forceinline__ float ldg_early(const float* p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ double ldg_early(const double* p) {
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint8_t ldg_early(const uint8_t* p) {
  unsigned short v;
  asm volatile("ld.global.nc.u8 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
  return (uint8_t)v;
}

template <typename T>
struct PlaneIn {
  T er1, ep1;          // plane k+1 (old e)
  T ez, hr, hp, hz;    // plane k
  uint8_t m;           // activity bits of plane k
};

template <typename T>
__device__ __forceinline__ void rz_item(const RzArgs<T>& a, int witem) {
  const int lane = threadIdx.x & 31;
  const int mode = witem % a.n_modes;
  const int rest = a.work[witem / a.n_modes];
  const int tile = rest % a.tiles, chunk = rest / a.tiles;
  const RzLayout L = a.L;
  const int gi = tile * kTile - 2 + lane;
  const int ci = min(gi, L.nr + 1);
  const bool own = lane >= 2 && lane < kTile + 2 && gi <= L.nr;
  const int k0 = chunk * a.chunk_z;
  const int k1 = min(k0 + a.chunk_z, L.nz);
  const long long cs = L.cs;
  const long long mb = (long long)mode * 6 * cs;
  const T* __restrict__ ib = a.in + mb + ci + L.orr;
  T* __restrict__ ob = a.out + mb + ci + L.orr;
  const uint8_t* __restrict__ mk = a.mask + ci + L.orr;
  const long long PR = L.pr;

  const T* co = a.coef + (long long)mode * kNCo * PR + ci + L.orr;
  const T cER = co[kCoER * PR], cEP = co[kCoEP * PR], cEZ = co[kCoEZ * PR];
  const T cHR = co[kCoHR * PR], cHP = co[kCoHP * PR], cHZ = co[kCoHZ * PR];
  const T fEZ = co[kCoFEZ * PR], fHZ = co[kCoFHZ * PR];
  const T mm = T(a.m_lo + mode);
  const bool src = a.b_on && gi == a.i0;
  const T* __restrict__ J = a.J + (long long)mode * 2 * a.c0;

  auto load = [&](int k, PlaneIn<T>& d) {
    const long long r = (long long)(min(k, L.nz) + 1) * PR;
    d.er1 = ldg_early(ib + kER * cs + r + PR);
    d.ep1 = ldg_early(ib + kEP * cs + r + PR);
    d.ez = ldg_early(ib + kEZ * cs + r);
    d.hr = ldg_early(ib + kHR * cs + r);
    d.hp = ldg_early(ib + kHP * cs + r);
    d.hz = ldg_early(ib + kHZ * cs + r);
    d.m = ldg_early(mk + r);
  };

  const int kstart = k0 - 1;
  T er0 = ib[kER * cs + (long long)(kstart + 1) * PR];
  T ep0 = ib[kEP * cs + (long long)(kstart + 1) * PR];
  T hr_p = T(0), hp_p = T(0);
  PlaneIn<T> ring[kRing];
#pragma unroll
  for (int u = 0; u < kRing; ++u) load(kstart + u, ring[u]);

  for (int kb = kstart; kb < k1; kb += kRing) {
#pragma unroll
    for (int u = 0; u < kRing; ++u) {
      const int k = kb + u;
      if (k >= k1) break;
      const PlaneIn<T> d = ring[u];
      load(k + kRing, ring[u]);
      const uint8_t m = d.m;
      const T CER = (m & 1) ? cER : T(0), CEP = (m & 2) ? cEP : T(0);
      const T CHR = (m & 8) ? cHR : T(0), CHP = (m & 16) ? cHP : T(0);
      const T FEZ = (m & 4) ? ((m & 8) ? fEZ : cEZ) : T(0);
      const T FHZ = (m & 32) ? ((m & 1) ? fHZ : cHZ) : T(0);
      // TM stage, plane k
      const T der = d.er1 - er0, dep = d.ep1 - ep0;
      const T hpa = d.hp + CHP * (der - (shfl_dn(d.ez) - d.ez));
      const T hra = d.hr + CHR * (-dep + mm * d.ez);
      T cur = (shfl_up(hpa) - hpa) - mm * hra;
      if (src && k >= 0) {
        const long long dd = (long long)k - a.n + a.c0;
        if (dd >= -a.c0 && dd < a.c0) cur -= J[dd + a.c0];
      }
      const T ezn = d.ez + FEZ * cur;
      const T hpn = hpa + CHP * (der - (shfl_dn(ezn) - ezn));
      const T hrn = hra + CHR * (-dep + mm * ezn);
      // TE stage, plane k
      const T dhr = hr_p - hrn, dhp = hp_p - hpn;
      const T epa = ep0 + CEP * (dhr - (shfl_up(d.hz) - d.hz));
      const T era = er0 + CER * (-dhp + mm * d.hz);
      const T hzn = d.hz + FHZ * ((shfl_dn(epa) - epa) - mm * era);
      const T epn = epa + CEP * (dhr - (shfl_up(hzn) - hzn));
      const T ern = era + CER * (-dhp + mm * hzn);
      if (own && k >= k0) {
        const long long r = (long long)(k + 1) * PR;
        ob[kEZ * cs + r] = ezn;
        ob[kHR * cs + r] = hrn;
        ob[kHP * cs + r] = hpn;
        ob[kEP * cs + r] = epn;
        ob[kER * cs + r] = ern;
        ob[kHZ * cs + r] = hzn;
        if (src) {
          const long long w = a.n - k - a.c0 - a.m_min;
          if (w >= 0 && w < a.nw) a.W[(long long)mode * a.nw + w] -= (double)ezn * a.inv_q;
        }
      }
      er0 = d.er1;
      ep0 = d.ep1;
      hr_p = hrn;
      hp_p = hpn;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(128) rz_step_kernel(const RzArgs<T> a) {
  const int nitems = a.n_work * a.n_modes;
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); w < nitems; w += nwarps)
    rz_item<T>(a, w);
}

// Activity bits from the cell geometry (staircase; the rules of the
// per-radian metric): bit c set <=> object c at entry (i, k) is non-PEC.
__device__ __forceinline__ bool cell_pec(const uint8_t* pec, int nr, int nz, int ci, int ck) {
  if (ci >= nr || ck < 0 || ck >= nz || ci < 0) return true;
  return pec ? pec[ci + (long long)nr * ck] != 0 : false;
}

__global__ void rz_build_mask(const uint8_t* pec, RzLayout L, uint8_t* mask) {
  const long long total = L.cs;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(q / L.pr) - 1;
    const int i = (int)(q % L.pr) - L.orr;
    uint8_t b = 0;
    if (i >= 0 && i <= L.nr && k >= 0 && k <= L.nz) {
      const int nr = L.nr, nz = L.nz;
      if (i < nr && !cell_pec(pec, nr, nz, i, k - 1) && !cell_pec(pec, nr, nz, i, k)) b |= 1 << kER;
      if (i > 0 && !cell_pec(pec, nr, nz, i - 1, k - 1) && !cell_pec(pec, nr, nz, i, k - 1) &&
          !cell_pec(pec, nr, nz, i - 1, k) && !cell_pec(pec, nr, nz, i, k))
        b |= 1 << kEP;
      if (k < nz) {
        if (i == 0) {
          if (!cell_pec(pec, nr, nz, 0, k)) b |= 1 << kEZ;
        } else if (!cell_pec(pec, nr, nz, i - 1, k) && !cell_pec(pec, nr, nz, i, k)) {
          b |= 1 << kEZ;
        }
      }
      if (i > 0 && k < nz && !cell_pec(pec, nr, nz, i - 1, k) && !cell_pec(pec, nr, nz, i, k))
        b |= 1 << kHR;
      if (i < nr && k < nz && !cell_pec(pec, nr, nz, i, k)) b |= 1 << kHP;
      if (i < nr && !cell_pec(pec, nr, nz, i, k - 1) && !cell_pec(pec, nr, nz, i, k)) b |= 1 << kHZ;
    }
    mask[q] = b;
  }
}

// A (radial tile, z chunk) pair is worth a work item when one of its owned
// entries carries a field.
__global__ void rz_item_flags(const uint8_t* mask, RzLayout L, int tiles, int chunk_z,
                              int n_chunks, int* flags) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= tiles * n_chunks) return;
  const int tile = q % tiles, chunk = q / tiles;
  const int i_lo = tile * kTile, i_hi = min(i_lo + kTile, L.nr + 1);
  const int k_lo = chunk * chunk_z, k_hi = min(k_lo + chunk_z, L.nz);
  int any = 0;
  for (int k = k_lo; k < k_hi && !any; ++k)
    for (int i = i_lo; i < i_hi; ++i)
      if (mask[L.idx(i, k)]) { any = 1; break; }
  flags[q] = any;
}

// Canonical <-> device layout for one array; `act` zeroes inactive entries
// (mask bit c clear or the mode's metric zero there).
template <typename T>
__global__ void rz_to_canonical(const T* src, RzLayout L, double* dst) {
  const long long n = (long long)(L.nr + 1) * (L.nz + 1);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % (L.nr + 1)), k = (int)(q / (L.nr + 1));
    dst[q] = (double)src[L.idx(i, k)];
  }
}

template <typename T>
__global__ void rz_from_canonical(const double* src, RzLayout L, const uint8_t* mask, int comp,
                                  const double* metric, T* dst) {
  const long long n = (long long)(L.nr + 1) * (L.nz + 1);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % (L.nr + 1)), k = (int)(q / (L.nr + 1));
    const long long id = L.idx(i, k);
    const bool act = ((mask[id] >> comp) & 1) && metric[i] != 0.0;
    dst[id] = act ? (T)src[q] : T(0);
  }
}

// Discrete energy per radian, 0.5 <Q^{e,r} y, y> (Sec. 4.4): the weighted
// squares of all six components, minus alpha^2/2 times the radial part of
// the splitting operator (M_mu_phi^-1 (P_r e_z)^2 and M_eps_phi^-1
// (P_r^T h_z)^2), plus alpha times the longitudinal coupling
// h_phi P_z e_r - h_r P_z e_phi. metric: [6][pr] unscaled M^-1 of the mode
// (zero where the mode has no object). One partial per block.
constexpr int kEnergyBlocks = 512;
constexpr int kEnergyThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kEnergyThreads)
rz_energy_partial(const T* f, RzLayout L, const uint8_t* mask, const double* metric, double alpha,
                  double* partial) {
  const long long cs = L.cs, PR = L.pr;
  const long long n = (long long)(L.nr + 1) * (L.nz + 1);
  double acc = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % (L.nr + 1)), k = (int)(q / (L.nr + 1));
    const long long id = L.idx(i, k);
    const uint8_t m = mask[id];
    double w = 0.0;
    double c[6];
    for (int comp = 0; comp < 6; ++comp) {
      c[comp] = ((m >> comp) & 1) ? metric[comp * PR + i] : 0.0;
      if (c[comp] != 0.0) {
        const double v = (double)f[comp * cs + id];
        w += 0.5 * v * v / c[comp];
      }
    }
    const double ez = (double)f[kEZ * cs + id], hz = (double)f[kHZ * cs + id];
    const double t1 = (double)f[kEZ * cs + id + 1] - ez;
    const double t2 = (double)f[kHZ * cs + id - 1] - hz;
    const double r = c[kHP] * t1 * t1 + c[kEP] * t2 * t2;
    const double l = (double)f[kHP * cs + id] * ((double)f[kER * cs + id + PR] - (double)f[kER * cs + id]) -
                     (double)f[kHR * cs + id] * ((double)f[kEP * cs + id + PR] - (double)f[kEP * cs + id]);
    acc += w - 0.5 * alpha * alpha * r + alpha * l;
  }
  __shared__ double sh[kEnergyThreads / 32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < kEnergyThreads / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
  }
}

__global__ void rz_energy_final(const double* partial, int n, double* out) {
  double v = 0.0;
  for (int q = threadIdx.x; q < n; q += 32) v += partial[q];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) *out = v;
}

double rz_phi(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

int rz_fail(cudaError_t e) {
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? TETM_E_NOMEM : TETM_E_CUDA;
}

bool rz_grid_ok(const tetm_rz_grid* g) {
  if (!g) return false;
  if (g->nr < 2 || g->nz < 2 || g->nr > (1 << 20) || g->nz > (1 << 28)) return false;
  if (g->m_lo < 0 || g->m_hi < g->m_lo || g->m_hi - g->m_lo + 1 > TETM_RZ_MAX_MODES) return false;
  if (g->precision != TETM_FP64 && g->precision != TETM_FP32) return false;
  if (!(g->dr > 0) || !(g->dz > 0) || !isfinite(g->dr) || !isfinite(g->dz)) return false;
  if (!(g->cdt >= 0) || !isfinite(g->cdt)) return false;
  return true;
}

}  // namespace

struct tetm_rz {
  tetm_rz_grid g;
  RzLayout L;
  int esz = 8;
  int n_modes = 1;
  double cdt = 0, alpha = 0;
  void* set[2] = {nullptr, nullptr};
  int cur = 0;
  uint8_t* mask = nullptr;
  void* coef = nullptr;          // [mode][kNCo][pr], T
  double* metric = nullptr;      // [mode][6][pr]
  int* work = nullptr;
  int n_work = 0, tiles = 0, chunk_z = 32, n_chunks = 0;
  bool work_dirty = true;
  long long processed = 0;
  int* flags = nullptr;
  int flags_cap = 0;
  // bunch
  bool bunch = false;
  int i0 = 0, c0 = 0, m_min = 0, m_max = 0, nw = 0;
  double q = 0, sigma = 0;
  void* J = nullptr;
  double* W = nullptr;
  double* partial = nullptr;     // energy partials + result
  long long step = 0;
  long long device_bytes = 0;
  cudaStream_t own = nullptr, st = nullptr;
  int resident = 0;
};

namespace {

template <typename T>
int rz_launch_steps(tetm_rz* s, long long n) {
  RzArgs<T> a;
  a.L = s->L;
  a.mask = s->mask;
  a.coef = static_cast<const T*>(s->coef);
  a.m_lo = s->g.m_lo;
  a.n_modes = s->n_modes;
  a.tiles = s->tiles;
  a.chunk_z = s->chunk_z;
  a.work = s->work;
  a.n_work = s->n_work;
  a.b_on = s->bunch ? 1 : 0;
  a.i0 = s->i0;
  a.c0 = s->c0;
  a.m_min = s->m_min;
  a.nw = s->nw;
  a.J = static_cast<const T*>(s->J);
  a.W = s->W;
  a.inv_q = s->bunch ? 1.0 / s->q : 0.0;
  const int items = s->n_work * s->n_modes;
  const int blocks = std::max(1, std::min(s->resident, (items + 3) / 4));
  for (long long t = 0; t < n; ++t) {
    a.in = static_cast<const T*>(s->set[s->cur]);
    a.out = static_cast<T*>(s->set[s->cur ^ 1]);
    a.n = s->step;
    if (items > 0) {
      rz_step_kernel<T><<<blocks, 128, 0, s->st>>>(a);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return rz_fail(e);
    }
    s->cur ^= 1;
    s->step += 1;
  }
  return TETM_OK;
}

// Blocks of 4 warps the step kernel keeps resident on the whole device.
template <typename T>
int rz_occupancy(tetm_rz* s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rz_step_kernel<T>, 128, 0);
  if (e != cudaSuccess) return rz_fail(e);
  s->resident = std::max(1, sms * per_sm);
  return TETM_OK;
}

int rz_rebuild_work(tetm_rz* s) {
  const RzLayout& L = s->L;
  s->tiles = (L.nr + 1 + kTile - 1) / kTile;
  s->n_chunks = (L.nz + s->chunk_z - 1) / s->chunk_z;
  const int nf = s->tiles * s->n_chunks;
  if (nf > s->flags_cap) {
    cudaFree(s->flags);
    s->flags = nullptr;
    s->flags_cap = 0;
    cudaError_t e = cudaMalloc(&s->flags, sizeof(int) * (size_t)nf);
    if (e != cudaSuccess) return rz_fail(e);
    s->flags_cap = nf;
  }
  rz_item_flags<<<(nf + 255) / 256, 256, 0, s->st>>>(s->mask, L, s->tiles, s->chunk_z, s->n_chunks,
                                                      s->flags);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rz_fail(e);
  std::vector<int> fl((size_t)nf);
  e = cudaMemcpyAsync(fl.data(), s->flags, sizeof(int) * (size_t)nf, cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return rz_fail(e);
  std::vector<int> w;
  long long processed = 0;
  for (int q = 0; q < nf; ++q) {
    if (!fl[(size_t)q]) continue;
    w.push_back(q);
    const int tile = q % s->tiles, chunk = q / s->tiles;
    const int width = std::min(kTile, L.nr + 1 - tile * kTile);
    const int planes = std::min(s->chunk_z, L.nz - chunk * s->chunk_z);
    processed += (long long)width * planes;
  }
  cudaFree(s->work);
  s->work = nullptr;
  if (!w.empty()) {
    e = cudaMalloc(&s->work, sizeof(int) * w.size());
    if (e != cudaSuccess) return rz_fail(e);
    e = cudaMemcpy(s->work, w.data(), sizeof(int) * w.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return rz_fail(e);
  }
  s->n_work = (int)w.size();
  s->processed = processed * s->n_modes;
  s->work_dirty = false;
  return TETM_OK;
}

// Per-radian metric of one mode at radial index i (unscaled M^-1; zero where
// the mode has no object) and the update coefficients derived from it.
void rz_metric_row(const tetm_rz_grid& g, int m, int i, double out[6]) {
  const double dr = g.dr, dz = g.dz;
  const double ri = i * dr, rh = (i + 0.5) * dr;
  out[kER] = i < g.nr ? dr / (kEps0 * rh * dz) : 0.0;
  out[kEP] = (i > 0 && i < g.nr) ? ri / (kEps0 * dr * dz) : 0.0;
  if (i == 0) out[kEZ] = m == 0 ? dz / (kEps0 * dr * dr / 4.0) : 0.0;
  else out[kEZ] = i < g.nr ? dz / (kEps0 * ri * dr) : 0.0;
  out[kHR] = (i > 0 && i < g.nr) ? dr / (kMu0 * ri * dz) : 0.0;
  out[kHP] = i < g.nr ? rh / (kMu0 * dr * dz) : 0.0;
  out[kHZ] = i < g.nr ? dz / (kMu0 * rh * dr) : 0.0;
}

template <typename T>
int rz_upload_coefs(tetm_rz* s) {
  const long long PR = s->L.pr;
  std::vector<T> co((size_t)s->n_modes * kNCo * PR, T(0));
  std::vector<double> me((size_t)s->n_modes * 6 * PR, 0.0);
  const double a = s->alpha;
  for (int mi = 0; mi < s->n_modes; ++mi) {
    const int m = s->g.m_lo + mi;
    for (int i = 0; i <= s->g.nr; ++i) {
      double c[6];
      rz_metric_row(s->g, m, i, c);
      const long long col = i + s->L.orr;
      for (int comp = 0; comp < 6; ++comp) me[((size_t)mi * 6 + comp) * PR + col] = c[comp];
      T* row = co.data() + (size_t)mi * kNCo * PR + col;
      row[kCoER * PR] = (T)(a * c[kER]);
      row[kCoEP * PR] = (T)(a * c[kEP]);
      row[kCoHR * PR] = (T)(a * c[kHR]);
      row[kCoHP * PR] = (T)(a * c[kHP]);
      row[kCoEZ * PR] = (T)(2.0 * a * c[kEZ]);
      row[kCoHZ * PR] = (T)(2.0 * a * c[kHZ]);
      const double mm = (double)m * m;
      row[kCoFEZ * PR] = (T)(2.0 * a * c[kEZ] / (1.0 + a * a * mm * c[kEZ] * c[kHR]));
      row[kCoFHZ * PR] = (T)(2.0 * a * c[kHZ] / (1.0 + a * a * mm * c[kHZ] * c[kER]));
    }
  }
  cudaError_t e = cudaMemcpy(s->coef, co.data(), sizeof(T) * co.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(s->metric, me.data(), sizeof(double) * me.size(), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? TETM_OK : rz_fail(e);
}

size_t rz_field_bytes(const RzLayout& L, int esz, int n_modes) {
  return (size_t)n_modes * 6 * (size_t)L.cs * (size_t)esz;
}

bool rz_mode_ok(const tetm_rz* s, int mode) { return s && mode >= 0 && mode < s->n_modes; }

}  // namespace

extern "C" {

int64_t tetm_rz_bytes_needed(const tetm_rz_grid* g) {
  if (!rz_grid_ok(g)) return 0;
  const int esz = g->precision == TETM_FP64 ? 8 : 4;
  const int nm = g->m_hi - g->m_lo + 1;
  const RzLayout L = make_rz_layout(g->nr, g->nz, esz);
  return (int64_t)(2 * rz_field_bytes(L, esz, nm) + (size_t)L.cs +
                   (size_t)nm * L.pr * (kNCo * esz + 6 * 8)) + (int64_t)(1 << 20);
}

int tetm_rz_create(const tetm_rz_grid* g, const double* eps_r, const double* mu_r,
                   const uint8_t* pec, tetm_rz** out) {
  if (!out) return TETM_E_ARG;
  *out = nullptr;
  if (!rz_grid_ok(g)) return TETM_E_ARG;
  if (eps_r || mu_r) return TETM_E_UNSUPPORTED;
  const double cdt = g->cdt > 0 ? g->cdt : std::min(g->dr, g->dz);
  if (cdt > g->dz * (1.0 + 1e-12) || cdt > g->dr * (1.0 + 1e-12)) return TETM_E_UNSTABLE;
  tetm_rz* s = new (std::nothrow) tetm_rz();
  if (!s) return TETM_E_NOMEM;
  s->g = *g;
  s->g.cdt = cdt;
  s->cdt = cdt;
  s->alpha = 0.5 * (cdt / kC);
  s->esz = g->precision == TETM_FP64 ? 8 : 4;
  s->n_modes = g->m_hi - g->m_lo + 1;
  s->L = make_rz_layout(g->nr, g->nz, s->esz);
  int rc = TETM_OK;
  uint8_t* dpec = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete s;
    return rz_fail(e);
  }
  s->st = s->own;
  const size_t fb = rz_field_bytes(s->L, s->esz, s->n_modes);
  const size_t cob = (size_t)s->n_modes * kNCo * s->L.pr * s->esz;
  const size_t meb = (size_t)s->n_modes * 6 * s->L.pr * sizeof(double);
  do {
    if ((e = cudaMalloc(&s->set[0], fb)) != cudaSuccess) break;
    if ((e = cudaMalloc(&s->set[1], fb)) != cudaSuccess) break;
    if ((e = cudaMalloc(&s->mask, (size_t)s->L.cs)) != cudaSuccess) break;
    if ((e = cudaMalloc(&s->coef, cob)) != cudaSuccess) break;
    if ((e = cudaMalloc(&s->metric, meb)) != cudaSuccess) break;
    if ((e = cudaMalloc(&s->partial, sizeof(double) * (kEnergyBlocks + 1))) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(s->set[0], 0, fb, s->st)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(s->set[1], 0, fb, s->st)) != cudaSuccess) break;
    if (pec) {
      const size_t nb = (size_t)g->nr * g->nz;
      if ((e = cudaMalloc(&dpec, nb)) != cudaSuccess) break;
      if ((e = cudaMemcpy(dpec, pec, nb, cudaMemcpyHostToDevice)) != cudaSuccess) break;
    }
    rz_build_mask<<<1024, 256, 0, s->st>>>(dpec, s->L, s->mask);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = cudaStreamSynchronize(s->st)) != cudaSuccess) break;
  } while (0);
  cudaFree(dpec);
  if (e != cudaSuccess) rc = rz_fail(e);
  if (rc == TETM_OK) rc = s->esz == 8 ? rz_upload_coefs<double>(s) : rz_upload_coefs<float>(s);
  if (rc == TETM_OK) rc = s->esz == 8 ? rz_occupancy<double>(s) : rz_occupancy<float>(s);
  if (rc == TETM_OK) rc = rz_rebuild_work(s);
  if (rc != TETM_OK) {
    tetm_rz_destroy(s);
    return rc;
  }
  s->device_bytes = (long long)(2 * fb + (size_t)s->L.cs + cob + meb);
  *out = s;
  return TETM_OK;
}

int tetm_rz_set_bunch(tetm_rz* s, double sigma, double q, int32_t i0) {
  if (!s || !(sigma > 0) || !isfinite(sigma) || q == 0 || !isfinite(q)) return TETM_E_ARG;
  if (i0 < 0 || i0 >= s->g.nr || (i0 == 0 && s->g.m_hi != 0)) return TETM_E_ARG;
  if (fabs(s->cdt - s->g.dz) > 1e-12 * s->g.dz) return TETM_E_NOT_MAGIC;
  if (s->step != 0 || s->bunch) return TETM_E_STATE;
  const double dz = s->g.dz;
  const int c0 = (int)ceil(5.0 * sigma / dz - 1e-12);
  const int m_max = (int)ceil(15.0 * sigma / dz - 1e-12);
  if (c0 < 1 || c0 > (1 << 20)) return TETM_E_ARG;
  const int nw = m_max + c0 + 2;
  std::vector<double> qc((size_t)(2 * c0));
  for (int d = -c0; d < c0; ++d) {
    const double lo = std::max((double)d * dz, -5.0 * sigma);
    const double hi = std::min((double)(d + 1) * dz, 5.0 * sigma);
    qc[(size_t)(d + c0)] = hi > lo ? q * (rz_phi(hi / sigma) - rz_phi(lo / sigma)) : 0.0;
  }
  const size_t nj = (size_t)s->n_modes * 2 * c0;
  std::vector<double> jd(nj);
  std::vector<float> jf(nj);
  for (int mi = 0; mi < s->n_modes; ++mi) {
    const double share = (s->g.m_lo + mi == 0 ? 1.0 : 2.0) / (2.0 * kPi);
    for (int d = 0; d < 2 * c0; ++d) {
      const double v = share * kC * qc[(size_t)d] / dz;
      jd[(size_t)mi * 2 * c0 + d] = v;
      jf[(size_t)mi * 2 * c0 + d] = (float)v;
    }
  }
  void* J = nullptr;
  double* W = nullptr;
  cudaError_t e = cudaMalloc(&J, (size_t)s->esz * nj);
  if (e == cudaSuccess) e = cudaMalloc(&W, sizeof(double) * (size_t)s->n_modes * nw);
  if (e == cudaSuccess)
    e = cudaMemcpy(J, s->esz == 8 ? (const void*)jd.data() : (const void*)jf.data(),
                   (size_t)s->esz * nj, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(W, 0, sizeof(double) * (size_t)s->n_modes * nw);
  if (e != cudaSuccess) {
    cudaFree(J);
    cudaFree(W);
    return rz_fail(e);
  }
  s->J = J;
  s->W = W;
  s->bunch = true;
  s->i0 = i0;
  s->c0 = c0;
  s->m_min = -c0 - 1;
  s->m_max = m_max;
  s->nw = nw;
  s->q = q;
  s->sigma = sigma;
  s->device_bytes += (long long)((size_t)s->esz * nj + sizeof(double) * (size_t)s->n_modes * nw);
  return TETM_OK;
}

int tetm_rz_step(tetm_rz* s, int64_t n) {
  if (!s || n < 0) return TETM_E_ARG;
  if (s->work_dirty) {
    int rc = rz_rebuild_work(s);
    if (rc) return rc;
  }
  return s->esz == 8 ? rz_launch_steps<double>(s, n) : rz_launch_steps<float>(s, n);
}

int tetm_rz_sync(tetm_rz* s) {
  if (!s) return TETM_E_ARG;
  cudaError_t e = cudaStreamSynchronize(s->st);
  return e == cudaSuccess ? TETM_OK : rz_fail(e);
}

int tetm_rz_wake(tetm_rz* s, int32_t mode, double* out, int32_t cap, int32_t* n_out, double* s0,
                 double* ds) {
  if (!rz_mode_ok(s, mode)) return TETM_E_ARG;
  if (!s->bunch) return TETM_E_STATE;
  if (n_out) *n_out = s->nw;
  if (s0) *s0 = s->m_min * s->g.dz;
  if (ds) *ds = s->g.dz;
  if (!out) return TETM_OK;
  if (cap < s->nw) return TETM_E_ARG;
  cudaError_t e = cudaMemcpyAsync(out, s->W + (size_t)mode * s->nw, sizeof(double) * s->nw,
                                  cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  return e == cudaSuccess ? TETM_OK : rz_fail(e);
}

int tetm_rz_energy(tetm_rz* s, int32_t mode, double* w) {
  if (!rz_mode_ok(s, mode) || !w) return TETM_E_ARG;
  const size_t off = (size_t)mode * 6 * s->L.cs * s->esz;
  const char* f = static_cast<const char*>(s->set[s->cur]) + off;
  const double* me = s->metric + (size_t)mode * 6 * s->L.pr + s->L.orr;
  if (s->esz == 8)
    rz_energy_partial<double><<<kEnergyBlocks, kEnergyThreads, 0, s->st>>>(
        reinterpret_cast<const double*>(f), s->L, s->mask, me, s->alpha, s->partial);
  else
    rz_energy_partial<float><<<kEnergyBlocks, kEnergyThreads, 0, s->st>>>(
        reinterpret_cast<const float*>(f), s->L, s->mask, me, s->alpha, s->partial);
  rz_energy_final<<<1, 32, 0, s->st>>>(s->partial, kEnergyBlocks, s->partial + kEnergyBlocks);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w, s->partial + kEnergyBlocks, sizeof(double), cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  return e == cudaSuccess ? TETM_OK : rz_fail(e);
}

int tetm_rz_get_fields(tetm_rz* s, int32_t mode, int32_t comp, double* out) {
  if (!rz_mode_ok(s, mode) || comp < 0 || comp > 5 || !out) return TETM_E_ARG;
  const size_t n = (size_t)(s->g.nr + 1) * (s->g.nz + 1);
  double* tmp = nullptr;
  cudaError_t e = cudaMallocAsync(&tmp, sizeof(double) * n, s->st);
  if (e != cudaSuccess) return rz_fail(e);
  const size_t off = ((size_t)mode * 6 + comp) * s->L.cs * s->esz;
  const char* f = static_cast<const char*>(s->set[s->cur]) + off;
  if (s->esz == 8)
    rz_to_canonical<double><<<512, 256, 0, s->st>>>(reinterpret_cast<const double*>(f), s->L, tmp);
  else
    rz_to_canonical<float><<<512, 256, 0, s->st>>>(reinterpret_cast<const float*>(f), s->L, tmp);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, sizeof(double) * n, cudaMemcpyDeviceToHost, s->st);
  cudaFreeAsync(tmp, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  return e == cudaSuccess ? TETM_OK : rz_fail(e);
}

int tetm_rz_set_fields(tetm_rz* s, int32_t mode, int32_t comp, const double* in) {
  if (!rz_mode_ok(s, mode) || comp < 0 || comp > 5 || !in) return TETM_E_ARG;
  const size_t n = (size_t)(s->g.nr + 1) * (s->g.nz + 1);
  double* tmp = nullptr;
  cudaError_t e = cudaMallocAsync(&tmp, sizeof(double) * n, s->st);
  if (e != cudaSuccess) return rz_fail(e);
  e = cudaMemcpyAsync(tmp, in, sizeof(double) * n, cudaMemcpyHostToDevice, s->st);
  const size_t off = ((size_t)mode * 6 + comp) * s->L.cs * s->esz;
  char* f = static_cast<char*>(s->set[s->cur]) + off;
  const double* me = s->metric + ((size_t)mode * 6 + comp) * s->L.pr + s->L.orr;
  if (e == cudaSuccess) {
    if (s->esz == 8)
      rz_from_canonical<double><<<512, 256, 0, s->st>>>(tmp, s->L, s->mask, comp, me,
                                                        reinterpret_cast<double*>(f));
    else
      rz_from_canonical<float><<<512, 256, 0, s->st>>>(tmp, s->L, s->mask, comp, me,
                                                       reinterpret_cast<float*>(f));
    e = cudaGetLastError();
  }
  cudaFreeAsync(tmp, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  return e == cudaSuccess ? TETM_OK : rz_fail(e);
}

int tetm_rz_set_tiling(tetm_rz* s, int32_t chunk_z) {
  if (!s || chunk_z < 4 || chunk_z > (1 << 20)) return TETM_E_ARG;
  s->chunk_z = chunk_z;
  s->work_dirty = true;
  return rz_rebuild_work(s);
}

int tetm_rz_set_stream(tetm_rz* s, void* cuda_stream) {
  if (!s) return TETM_E_ARG;
  s->st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : s->own;
  return TETM_OK;
}

int tetm_rz_get_info(tetm_rz* s, tetm_rz_info* info) {
  if (!s || !info) return TETM_E_ARG;
  info->step = s->step;
  info->device_bytes = s->device_bytes;
  info->processed_cells = s->processed;
  info->n_modes = s->n_modes;
  info->chunk_z = s->chunk_z;
  info->work_items = s->n_work * s->n_modes;
  info->wake_len = s->bunch ? s->nw : 0;
  info->resident_warps = 4 * s->resident;
  info->pad = 0;
  return TETM_OK;
}

int tetm_rz_destroy(tetm_rz* s) {
  if (!s) return TETM_OK;
  if (s->own) cudaStreamSynchronize(s->own);
  if (s->st && s->st != s->own) cudaStreamSynchronize(s->st);
  cudaFree(s->set[0]);
  cudaFree(s->set[1]);
  cudaFree(s->mask);
  cudaFree(s->coef);
  cudaFree(s->metric);
  cudaFree(s->work);
  cudaFree(s->flags);
  cudaFree(s->J);
  cudaFree(s->W);
  cudaFree(s->partial);
  if (s->own) cudaStreamDestroy(s->own);
  cudaGetLastError();
  delete s;
  return TETM_OK;
}

}  // extern "C"
