// FP64 balance checks on the device: the discrete energy of Sec. 4.4 and the
// second-order charges of Sec. 4.5, Eqs. (34) and (35). Both are two-pass
// reductions with a fixed launch shape, so the summation order (and with it
// the float64 result) is the same on every call: pass 1 reduces a fixed
// strided subset per thread, then each block with warp shuffles, into one
// partial per block; pass 2 reduces the partials in one block.
#include "tetm_internal.h"

namespace tetm {

namespace {

constexpr int kBlock = 256;
constexpr int kMaxBlocks = 2048;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Block reduction of one value per thread; result valid in thread 0.
template <bool MAX>
__device__ double block_reduce(double v) {
  __shared__ double s[32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = MAX ? warp_max(v) : warp_sum(v);
  if (lane == 0) s[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? s[threadIdx.x] : 0.0;
  if (w == 0) v = MAX ? warp_max(v) : warp_sum(v);
  __syncthreads();
  return v;
}

struct MinvView {
  const uint8_t* mask;
  double c[6];          // M^-1 constants (uniform material)
  double r[6];          // their reciprocals M = 1/M^-1
  const double* a[6];   // per-entry M^-1 (material runs) or nullptr
  __device__ __forceinline__ double operator()(int comp, long long id) const {
    if (a[comp]) return a[comp][id];
    return ((mask[id] >> comp) & 1) ? c[comp] : 0.0;
  }
  // M = 1/M^-1 of an active entry (0 for inactive ones)
  __device__ __forceinline__ double m(int comp, long long id) const {
    if (a[comp]) {
      const double v = a[comp][id];
      return v != 0.0 ? 1.0 / v : 0.0;
    }
    return ((mask[id] >> comp) & 1) ? r[comp] : 0.0;
  }
};

// Energy density of node index (i,j,k): Sec. 4.4, W = 1/2 <Q^e y, y> with
// Q^e = [[I - a^2 R_0, a L], [a L^T, I - a^2 R_1]], in integral variables.
template <typename T>
__global__ void energy_pass1(const T* __restrict__ ex, const T* __restrict__ ey,
                             const T* __restrict__ ez, const T* __restrict__ hx,
                             const T* __restrict__ hy, const T* __restrict__ hz, MinvView mv,
                             Layout L, double alpha, double* part) {
  const long long total = (long long)L.nx * L.ny * L.nz;
  const long long stride = (long long)gridDim.x * blockDim.x;
  double acc = 0.0;
  const long long sx = 1, sy = L.px, sz = L.sz;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
    const int i = (int)(q % L.nx);
    const int j = (int)((q / L.nx) % L.ny);
    const int k = (int)(q / ((long long)L.nx * L.ny));
    const long long id = L.idx(i, j, k);
    if (mv.mask[id] == 0) continue;  // no field object here: every term is zero
    const T* f[6] = {ex, ey, ez, hx, hy, hz};
    double w = 0.0;
    double mi[6];
    for (int c = 0; c < 6; ++c) {
      mi[c] = mv(c, id);
      if (mi[c] != 0.0) {
        const double v = (double)f[c][id];
        w += 0.5 * v * v * mv.m(c, id);
      }
    }
    const double pyez = (double)ez[id + sy] - (double)ez[id];
    const double pxez = (double)ez[id + sx] - (double)ez[id];
    const double ptyhz = (double)hz[id - sy] - (double)hz[id];
    const double ptxhz = (double)hz[id - sx] - (double)hz[id];
    const double r = mi[kHX] * pyez * pyez + mi[kHY] * pxez * pxez + mi[kEX] * ptyhz * ptyhz +
                     mi[kEY] * ptxhz * ptxhz;
    const double l = (double)hx[id] * ((double)ey[id + sz] - (double)ey[id]) -
                     (double)hy[id] * ((double)ex[id + sz] - (double)ex[id]);
    acc += w - 0.5 * alpha * alpha * r + alpha * l;
  }
  const double b = block_reduce<false>(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = b;
}

template <bool MAX>
__global__ void reduce_pass2(const double* part, int n, double* out) {
  double v = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) v = MAX ? fmax(v, part[q]) : v + part[q];
  v = block_reduce<MAX>(v);
  if (threadIdx.x == 0) *out = v;
}

// Electric displacement-like flux of Eq. (35) on edge e: M_eps (e1 + e0)/2 for
// ex, ey; for ez the (I - a^2 r_0) corrected M_eps ez.
template <typename T>
__device__ __forceinline__ double dbar(const T* f1, const T* f0, const MinvView& mv, int comp,
                                       long long e) {
  return 0.5 * ((double)f1[e] + (double)f0[e]) * mv.m(comp, e);
}
template <typename T>
__device__ __forceinline__ double dz_tilde(const T* ez, const MinvView& mv, long long e,
                                           long long sx, long long sy, double a2) {
  const double mi = mv(kEZ, e);
  if (mi == 0.0) return 0.0;
  auto t1 = [&](long long f) { return mv(kHX, f) * ((double)ez[f + sy] - (double)ez[f]); };
  auto t2 = [&](long long f) { return mv(kHY, f) * ((double)ez[f + sx] - (double)ez[f]); };
  const double r = (t1(e - sy) - t1(e)) + (t2(e - sx) - t2(e));
  return (double)ez[e] * mv.m(kEZ, e) - a2 * r;
}
template <typename T>
__device__ __forceinline__ double bbar(const T* f1, const T* f0, const MinvView& mv, int comp,
                                       long long f) {
  return 0.5 * ((double)f1[f] + (double)f0[f]) * mv.m(comp, f);
}
template <typename T>
__device__ __forceinline__ double bz_tilde(const T* hz, const MinvView& mv, long long f,
                                           long long sx, long long sy, double a2) {
  const double mi = mv(kHZ, f);
  if (mi == 0.0) return 0.0;
  auto t3 = [&](long long e) { return mv(kEX, e) * ((double)hz[e - sy] - (double)hz[e]); };
  auto t4 = [&](long long e) { return mv(kEY, e) * ((double)hz[e - sx] - (double)hz[e]); };
  const double r = (t3(f + sy) - t3(f)) + (t4(f + sx) - t4(f));
  return (double)hz[f] * mv.m(kHZ, f) - a2 * r;
}

struct ChargeFields {
  const void* cur[6];
  const void* prev[6];
};

template <typename T>
__global__ void charge_pass1(ChargeFields cf, MinvView mv, Layout L, double alpha,
                             const double* qline, int i0, int j0, double* part_e, double* part_h) {
  const T* const* cur = reinterpret_cast<const T* const*>(cf.cur);
  const T* const* prv = reinterpret_cast<const T* const*>(cf.prev);
  const long long total = (long long)(L.nx + 1) * (L.ny + 1) * (L.nz + 1);
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long sx = 1, sy = L.px, sz = L.sz;
  const double a2 = alpha * alpha;
  double me = 0.0, mh = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
    const int i = (int)(q % (L.nx + 1));
    const int j = (int)((q / (L.nx + 1)) % (L.ny + 1));
    const int k = (int)(q / ((long long)(L.nx + 1) * (L.ny + 1)));
    const long long n = L.idx(i, j, k);
    const uint8_t m0 = mv.mask[n];
    if (m0 == 0) continue;  // neither the node's edges nor the cell's faces start here
    // Eq. (35) at node n: six incident edges active
    if ((m0 & 7) == 7 && mv(kEX, n) != 0.0 && mv(kEX, n - sx) != 0.0 && mv(kEY, n) != 0.0 &&
        mv(kEY, n - sy) != 0.0 && mv(kEZ, n) != 0.0 && mv(kEZ, n - sz) != 0.0) {
      const double qe =
          -(dbar(cur[kEX], prv[kEX], mv, kEX, n - sx) - dbar(cur[kEX], prv[kEX], mv, kEX, n)) -
          (dbar(cur[kEY], prv[kEY], mv, kEY, n - sy) - dbar(cur[kEY], prv[kEY], mv, kEY, n)) -
          (dz_tilde(cur[kEZ], mv, n - sz, sx, sy, a2) - dz_tilde(cur[kEZ], mv, n, sx, sy, a2));
      const double qb = (qline && i == i0 && j == j0) ? qline[k] : 0.0;
      me = fmax(me, fabs(qe - qb));
    }
    // Eq. (34) at the cell whose lower node is n: six faces active
    if ((m0 & 56) == 56 && mv(kHX, n) != 0.0 && mv(kHX, n + sx) != 0.0 && mv(kHY, n) != 0.0 &&
        mv(kHY, n + sy) != 0.0 && mv(kHZ, n) != 0.0 && mv(kHZ, n + sz) != 0.0) {
      const double qh =
          (bbar(cur[kHX], prv[kHX], mv, kHX, n + sx) - bbar(cur[kHX], prv[kHX], mv, kHX, n)) +
          (bbar(cur[kHY], prv[kHY], mv, kHY, n + sy) - bbar(cur[kHY], prv[kHY], mv, kHY, n)) +
          (bz_tilde(prv[kHZ], mv, n + sz, sx, sy, a2) - bz_tilde(prv[kHZ], mv, n, sx, sy, a2));
      mh = fmax(mh, fabs(qh));
    }
  }
  const double be = block_reduce<true>(me);
  const double bh = block_reduce<true>(mh);
  if (threadIdx.x == 0) {
    part_e[blockIdx.x] = be;
    part_h[blockIdx.x] = bh;
  }
}

MinvView make_view(const uint8_t* mask, const double* minv, const double* const minv_a[6]) {
  MinvView v;
  v.mask = mask;
  for (int c = 0; c < 6; ++c) {
    v.c[c] = minv ? minv[c] : 0.0;
    v.r[c] = (minv && minv[c] != 0.0) ? 1.0 / minv[c] : 0.0;
    v.a[c] = minv_a ? minv_a[c] : nullptr;
  }
  return v;
}

int blocks_for(long long total, int cap) {
  long long b = (total + kBlock - 1) / kBlock;
  if (b > cap) b = cap;
  if (b > kMaxBlocks) b = kMaxBlocks;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

template <typename T>
cudaError_t launch_energy(const T* const f[6], const uint8_t* mask, const double* minv,
                          const double* const minv_a[6], const Layout& L, double alpha,
                          const DiagScratch& s, double* result, cudaStream_t st) {
  const int nb = blocks_for((long long)L.nx * L.ny * L.nz, s.cap);
  energy_pass1<T><<<nb, kBlock, 0, st>>>(f[0], f[1], f[2], f[3], f[4], f[5],
                                          make_view(mask, minv, minv_a), L, alpha, s.part);
  reduce_pass2<false><<<1, 1024, 0, st>>>(s.part, nb, result);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_charge(const T* const cur[6], const T* const prev[6], const uint8_t* mask,
                          const double* minv, const double* const minv_a[6], const Layout& L,
                          double alpha, const double* qline, int i0, int j0,
                          const DiagScratch& s, double* res_e, double* res_h, cudaStream_t st) {
  const int nb = blocks_for((long long)(L.nx + 1) * (L.ny + 1) * (L.nz + 1), s.cap / 2);
  ChargeFields cf;
  for (int c = 0; c < 6; ++c) {
    cf.cur[c] = cur[c];
    cf.prev[c] = prev[c];
  }
  charge_pass1<T><<<nb, kBlock, 0, st>>>(cf, make_view(mask, minv, minv_a), L, alpha, qline,
                                          i0, j0, s.part, s.part + nb);
  reduce_pass2<true><<<1, 1024, 0, st>>>(s.part, nb, res_e);
  reduce_pass2<true><<<1, 1024, 0, st>>>(s.part + nb, nb, res_h);
  return cudaGetLastError();
}

namespace {
// Charge of the +-5 sigma truncated Gaussian inside [zc + lo, zc + hi] per
// node: the closed form the charge law (35) telescopes to from a cold start.
__global__ void bunch_charge_kernel(double q, double sigma, double dz, double zc, int nz,
                                    double* ql, double* qmax, double tag, double* tag_out) {
  double m = 0.0;
  const double r2 = 0.70710678118654752440;  // 1/sqrt(2)
  for (int k = threadIdx.x; k <= nz; k += blockDim.x) {
    const double lo = fmax(k * dz - 0.5 * dz - zc, -5.0 * sigma);
    const double hi = fmin(k * dz + 0.5 * dz - zc, 5.0 * sigma);
    double v = 0.0;
    if (q != 0.0 && hi > lo) v = q * 0.5 * (erfc(-hi / sigma * r2) - erfc(-lo / sigma * r2));
    ql[k] = v;
    m = fmax(m, fabs(v));
  }
  m = block_reduce<true>(m);
  if (threadIdx.x == 0) {
    *qmax = m;
    if (tag_out) *tag_out = tag;
  }
}
}  // namespace

cudaError_t launch_bunch_charge(double q, double sigma, double dz, double zc, int nz, double* ql,
                                double* qmax, double tag, double* tag_out, cudaStream_t st) {
  bunch_charge_kernel<<<1, 1024, 0, st>>>(q, sigma, dz, zc, nz, ql, qmax, tag, tag_out);
  return cudaGetLastError();
}

template cudaError_t launch_energy<float>(const float* const[6], const uint8_t*, const double*,
                                          const double* const[6], const Layout&, double,
                                          const DiagScratch&, double*, cudaStream_t);
template cudaError_t launch_energy<double>(const double* const[6], const uint8_t*, const double*,
                                           const double* const[6], const Layout&, double,
                                           const DiagScratch&, double*, cudaStream_t);
template cudaError_t launch_charge<float>(const float* const[6], const float* const[6],
                                          const uint8_t*, const double*, const double* const[6],
                                          const Layout&, double, const double*, int, int,
                                          const DiagScratch&, double*, double*, cudaStream_t);
template cudaError_t launch_charge<double>(const double* const[6], const double* const[6],
                                           const uint8_t*, const double*, const double* const[6],
                                           const Layout&, double, const double*, int, int,
                                           const DiagScratch&, double*, double*, cudaStream_t);

}  // namespace tetm
