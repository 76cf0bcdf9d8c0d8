// tetm_energy_noalloc: the discrete-energy reduction for callers that may not
// allocate device memory (code that runs under an external memory arena or
// allocator hook, inside a host framework that owns every device allocation,
// or in a real-time loop where cudaMalloc/cudaFree and their implicit device
// synchronisation are not allowed). The caller passes its own device arrays
// for the state and for the result; the block partial sums live in a fixed
// file-scope device array instead of solver-owned scratch.
#include <cuda.h>
#include <math.h>

#include <mutex>

#include "tetm_internal.h"

namespace tetm {
namespace {

constexpr int kNaBlock = 256;                 // threads per block
constexpr int kNaPerThread = 16;              // entries per thread
constexpr long long kNaPerBlock = (long long)kNaBlock * kNaPerThread;
constexpr int kNaMaxPartials = TETM_NOALLOC_MAX_ENTRIES / (kNaBlock * kNaPerThread);

// Shared by every call on a device and kept until the process exits; pass 1
// writes every slot it later reads, so nothing needs clearing between calls.
static __device__ __align__(256) double g_noalloc_partials[kNaMaxPartials];

// The array's device address depends on the context the library's module
// is loaded in: a caller on its own driver context sees another address than
// the runtime's primary context of the same device. The address is resolved
// once per (device, context) pair and cached.
constexpr int kMaxDevices = 64, kCtxPerDevice = 8;
std::mutex g_setup_mu;
struct CtxAddr {
  void* ctx;
  double* addr;
};
CtxAddr g_partials_addr[kMaxDevices][kCtxPerDevice];

// the calling thread's current driver context (nullptr when the driver entry
// point is not available: every call then shares one cache slot per device)
void* current_context() {
  using GetCtx = CUresult (*)(CUcontext*);
  static GetCtx fn = nullptr;
  static bool looked = false;
  if (!looked) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<GetCtx>(p);
    looked = true;
  }
  CUcontext c = nullptr;
  if (fn && fn(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

__device__ __forceinline__ double na_warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ double na_block_sum(double v) {
  __shared__ double s[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = na_warp_sum(v);
  if (lane == 0) s[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = threadIdx.x < nw ? s[threadIdx.x] : 0.0;
  if (w == 0) v = na_warp_sum(v);
  return v;
}

struct NaArgs {
  const void* f[6];
  const uint8_t* mask;  // canonical layout, or nullptr: only the box walls are PEC
  int nx, ny, nz;
  long long n;          // (nx+1)(ny+1)(nz+1)
  long long sx, sy, sz;
  double minv[6];       // vacuum M_eps^-1 / M_mu^-1 per component
  double alpha;         // dt/2
};

// Activity of component c at canonical node (i,j,k) in an empty PEC box.
__device__ __forceinline__ bool box_active(int c, int i, int j, int k, int nx, int ny, int nz) {
  const bool ix = i > 0 && i < nx, jy = j > 0 && j < ny, kz = k > 0 && k < nz;
  switch (c) {
    case kEX: return i < nx && jy && kz;
    case kEY: return j < ny && ix && kz;
    case kEZ: return k < nz && ix && jy;
    case kHX: return ix && j < ny && k < nz;
    case kHY: return jy && i < nx && k < nz;
    default:  return kz && i < nx && j < ny;
  }
}

// Pass 1: the energy of Sec. 4.4 in the canonical FIT layout (same terms as
// the solver's energy reduction), one partial per block of kNaPerBlock
// consecutive entries, written to part[blockIdx.x].
template <typename T>
__global__ void na_energy_pass1(NaArgs a, double* part) {
  const T* ex = (const T*)a.f[kEX];
  const T* ey = (const T*)a.f[kEY];
  const T* ez = (const T*)a.f[kEZ];
  const T* hx = (const T*)a.f[kHX];
  const T* hy = (const T*)a.f[kHY];
  const T* hz = (const T*)a.f[kHZ];
  const T* F[6] = {ex, ey, ez, hx, hy, hz};
  auto at = [&](const T* v, long long q) { return (q >= 0 && q < a.n) ? (double)v[q] : 0.0; };
  double acc = 0.0;
  const long long base = (long long)blockIdx.x * kNaPerBlock;
  for (int t = 0; t < kNaPerThread; ++t) {
    const long long q = base + (long long)t * kNaBlock + threadIdx.x;
    if (q >= a.n) break;
    const int i = (int)(q % (a.nx + 1));
    const int j = (int)((q / (a.nx + 1)) % (a.ny + 1));
    const int k = (int)(q / ((long long)(a.nx + 1) * (a.ny + 1)));
    double mi[6];
    double w = 0.0;
    for (int c = 0; c < 6; ++c) {
      const bool on = a.mask ? ((a.mask[q] >> c) & 1) : box_active(c, i, j, k, a.nx, a.ny, a.nz);
      mi[c] = on ? a.minv[c] : 0.0;
      if (on) {
        const double v = (double)F[c][q];
        w += 0.5 * v * v / mi[c];
      }
    }
    const double pyez = at(ez, q + a.sy) - (double)ez[q];
    const double pxez = at(ez, q + a.sx) - (double)ez[q];
    const double ptyhz = at(hz, q - a.sy) - (double)hz[q];
    const double ptxhz = at(hz, q - a.sx) - (double)hz[q];
    const double r = mi[kHX] * pyez * pyez + mi[kHY] * pxez * pxez + mi[kEX] * ptyhz * ptyhz +
                     mi[kEY] * ptxhz * ptxhz;
    const double l = (double)hx[q] * (at(ey, q + a.sz) - (double)ey[q]) -
                     (double)hy[q] * (at(ex, q + a.sz) - (double)ex[q]);
    acc += w - 0.5 * a.alpha * a.alpha * r + a.alpha * l;
  }
  const double b = na_block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

// Pass 2: one block adds the partials in a fixed order.
__global__ void na_energy_pass2(const double* part, int np, double* out) {
  double v = 0.0;
  for (int q = threadIdx.x; q < np; q += blockDim.x) v += part[q];
  v = na_block_sum(v);
  if (threadIdx.x == 0) *out = v;
}

// Device address of the scratch array for the current device and context;
// resolved by the first call in that context (with that device current) and
// cached. A device with more than kCtxPerDevice contexts resolves it on every
// call in the contexts beyond those (cudaGetSymbolAddress allocates nothing).
int partials_on_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return TETM_E_CUDA;
  }
  void* ctx = current_context();
  std::lock_guard<std::mutex> lk(g_setup_mu);
  CtxAddr* slots = g_partials_addr[dev];
  int free_slot = -1;
  for (int q = 0; q < kCtxPerDevice; ++q) {
    if (slots[q].addr && slots[q].ctx == ctx) {
      *out = slots[q].addr;
      return TETM_OK;
    }
    if (!slots[q].addr && free_slot < 0) free_slot = q;
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    return TETM_E_CUDA;
  }
  if (free_slot >= 0) slots[free_slot] = CtxAddr{ctx, (double*)p};
  *out = (double*)p;
  return TETM_OK;
}

}  // namespace
}  // namespace tetm

using namespace tetm;

extern "C" int tetm_energy_noalloc(const tetm_grid* g, const void* const fields[6],
                                   const uint8_t* mask, double* w, void* stream) {
  // the checks of tetm_create's grid (finite, positive steps, cell counts in
  // range), then the size limit of the scratch array
  if (!g || !fields || !w || g->nx < 2 || g->ny < 2 || g->nz < 2 || !(g->dx > 0) ||
      !(g->dy > 0) || !(g->dz > 0) || !(g->cdt >= 0) || !isfinite(g->dx) || !isfinite(g->dy) ||
      !isfinite(g->dz) || !isfinite(g->cdt) || (g->precision != TETM_FP64 && g->precision != TETM_FP32) ||
      (long long)g->nx * g->ny >= (1LL << 31) ||
      ((long long)g->nx + 1) * ((long long)g->ny + 1) * ((long long)g->nz + 1) >= (1LL << 40))
    return TETM_E_ARG;
  for (int c = 0; c < 6; ++c)
    if (!fields[c]) return TETM_E_ARG;
  const long long n = ((long long)g->nx + 1) * ((long long)g->ny + 1) * ((long long)g->nz + 1);
  if (n > (long long)TETM_NOALLOC_MAX_ENTRIES) return TETM_E_TOO_LARGE;
  double* part = nullptr;
  int rc = partials_on_current_device(&part);
  if (rc) return rc;
  NaArgs a;
  for (int c = 0; c < 6; ++c) a.f[c] = fields[c];
  a.mask = mask;
  a.nx = g->nx;
  a.ny = g->ny;
  a.nz = g->nz;
  a.n = n;
  a.sx = 1;
  a.sy = (long long)g->nx + 1;
  a.sz = ((long long)g->nx + 1) * ((long long)g->ny + 1);
  const double dx = g->dx, dy = g->dy, dz = g->dz;
  a.minv[kEX] = dx / (kEps0 * dy * dz);
  a.minv[kEY] = dy / (kEps0 * dx * dz);
  a.minv[kEZ] = dz / (kEps0 * dx * dy);
  a.minv[kHX] = dx / (kMu0 * dy * dz);
  a.minv[kHY] = dy / (kMu0 * dx * dz);
  a.minv[kHZ] = dz / (kMu0 * dx * dy);
  a.alpha = 0.5 * (g->cdt > 0 ? g->cdt : g->dz) / kC;
  const int nb = (int)((n + kNaPerBlock - 1) / kNaPerBlock);
  cudaStream_t st = (cudaStream_t)stream;
  if (g->precision == TETM_FP64)
    na_energy_pass1<double><<<nb, kNaBlock, 0, st>>>(a, part);
  else
    na_energy_pass1<float><<<nb, kNaBlock, 0, st>>>(a, part);
  na_energy_pass2<<<1, 1024, 0, st>>>(part, nb, w);
  if (cudaGetLastError() != cudaSuccess) return TETM_E_CUDA;
  return TETM_OK;
}
