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

// Cells of one work item, column by column: thread t takes columns t,
// t + blockDim, ... of the tile and marches through the item's z-planes.
struct ItemCells {
  int i0, j0, k0, k1, tx, ty;
  __device__ ItemCells(const WorkView& wv, const Layout& L, int item) {
    const int ntile = wv.tiles_x * wv.tiles_y;
    const int tile = item % ntile, chunk = item / ntile;
    tx = wv.tile_x;
    ty = wv.tile_y;
    i0 = (tile % wv.tiles_x) * wv.tile_x;
    j0 = (tile / wv.tiles_x) * wv.tile_y;
    k0 = chunk * wv.chunk_z;
    k1 = min(k0 + wv.chunk_z, L.nz);
  }
};

// Energy of Sec. 4.4, W = 1/2 <Q^e y, y> with Q^e = [[I - a^2 R_0, a L],
// [a L^T, I - a^2 R_1]], in integral variables: the share of node index
// (i,j,k) is 1/2 sum_c M_c f_c^2 - a^2/2 (M_mux^-1 (P_y ez)^2 +
// M_muy^-1 (P_x ez)^2 + M_epsx^-1 (P_y^T hz)^2 + M_epsy^-1 (P_x^T hz)^2)
// + a (hx P_z ey - hy P_z ex). One partial per work item.
template <typename T>
__global__ void energy_items(const T* __restrict__ ex, const T* __restrict__ ey,
                             const T* __restrict__ ez, const T* __restrict__ hx,
                             const T* __restrict__ hy, const T* __restrict__ hz, MinvView mv,
                             Layout L, WorkView wv, double alpha, double* part) {
  const int item = wv.items ? wv.items[blockIdx.x] : (int)blockIdx.x;
  const ItemCells ic(wv, L, item);
  const long long sx = 1, sy = L.px, sz = L.sz;
  const T* f[6] = {ex, ey, ez, hx, hy, hz};
  const bool uniform = mv.a[0] == nullptr;
  // uniform material: per-component sums of squares, scaled once at the end
  double sq[6] = {0, 0, 0, 0, 0, 0};
  double rq[4] = {0, 0, 0, 0};  // (P_y ez)^2 on hx faces, (P_x ez)^2 on hy faces, (P_y^T hz)^2 on ex, (P_x^T hz)^2 on ey
  double acc = 0.0;             // cross terms (and everything, for material arrays)
  for (int c = threadIdx.x; c < ic.tx * ic.ty; c += blockDim.x) {
    const int i = ic.i0 + c % ic.tx, j = ic.j0 + c / ic.tx;
    if (i >= L.nx || j >= L.ny) continue;
    for (int k = ic.k0; k < ic.k1; ++k) {
      const long long id = L.idx(i, j, k);
      const uint8_t m = mv.mask[id];
      if (m == 0) continue;  // no field object here: every term is zero
      const double pyez = (double)ez[id + sy] - (double)ez[id];
      const double pxez = (double)ez[id + sx] - (double)ez[id];
      const double ptyhz = (double)hz[id - sy] - (double)hz[id];
      const double ptxhz = (double)hz[id - sx] - (double)hz[id];
      const double l = (double)hx[id] * ((double)ey[id + sz] - (double)ey[id]) -
                       (double)hy[id] * ((double)ex[id + sz] - (double)ex[id]);
      if (uniform) {
        // inactive entries hold zero fields, so their squares add nothing
        for (int q = 0; q < 6; ++q) {
          const double v = (double)f[q][id];
          sq[q] += v * v;
        }
        if (m & 8) rq[0] += pyez * pyez;
        if (m & 16) rq[1] += pxez * pxez;
        if (m & 1) rq[2] += ptyhz * ptyhz;
        if (m & 2) rq[3] += ptxhz * ptxhz;
        acc += alpha * l;
      } else {
        double w = 0.0;
        for (int q = 0; q < 6; ++q) {
          const double v = (double)f[q][id];
          w += 0.5 * v * v * mv.m(q, id);
        }
        const double r = mv(kHX, id) * pyez * pyez + mv(kHY, id) * pxez * pxez +
                         mv(kEX, id) * ptyhz * ptyhz + mv(kEY, id) * ptxhz * ptxhz;
        acc += w - 0.5 * alpha * alpha * r + alpha * l;
      }
    }
  }
  if (uniform) {
    for (int q = 0; q < 6; ++q) acc += 0.5 * mv.r[q] * sq[q];
    acc -= 0.5 * alpha * alpha *
           (mv.c[kHX] * rq[0] + mv.c[kHY] * rq[1] + mv.c[kEX] * rq[2] + mv.c[kEY] * rq[3]);
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

// Charge balances over the nodes and cells of one work item. Marching up a
// column, the corrected z-fluxes of Eq. (35) and Eq. (34) on the edge/face
// below are those computed one plane earlier.
template <typename T>
__global__ void charge_items(ChargeFields cf, MinvView mv, Layout L, WorkView wv, double alpha,
                             const double* qline, int i0, int j0, double* part_e, double* part_h) {
  const T* const* cur = reinterpret_cast<const T* const*>(cf.cur);
  const T* const* prv = reinterpret_cast<const T* const*>(cf.prev);
  const int item = wv.items ? wv.items[blockIdx.x] : (int)blockIdx.x;
  const ItemCells ic(wv, L, item);
  const long long sx = 1, sy = L.px, sz = L.sz;
  const double a2 = alpha * alpha;
  double me = 0.0, mh = 0.0;
  for (int c = threadIdx.x; c < ic.tx * ic.ty; c += blockDim.x) {
    const int i = ic.i0 + c % ic.tx, j = ic.j0 + c / ic.tx;
    if (i >= L.nx || j >= L.ny) continue;
    long long n = L.idx(i, j, ic.k0);
    double dz_below = dz_tilde(cur[kEZ], mv, n - sz, sx, sy, a2);  // edge (i,j,k0-1/2)
    double bz_here = bz_tilde(prv[kHZ], mv, n, sx, sy, a2);        // face (i+1/2,j+1/2,k0)
    for (int k = ic.k0; k < ic.k1; ++k, n += sz) {
      const double dz_here = dz_tilde(cur[kEZ], mv, n, sx, sy, a2);
      const double bz_above = bz_tilde(prv[kHZ], mv, n + sz, sx, sy, a2);
      const uint8_t m0 = mv.mask[n];
      // Eq. (35) at node n: six incident edges active
      if ((m0 & 7) == 7 && mv(kEX, n - sx) != 0.0 && mv(kEY, n - sy) != 0.0 &&
          mv(kEZ, n - sz) != 0.0) {
        const double qe =
            -(dbar(cur[kEX], prv[kEX], mv, kEX, n - sx) - dbar(cur[kEX], prv[kEX], mv, kEX, n)) -
            (dbar(cur[kEY], prv[kEY], mv, kEY, n - sy) - dbar(cur[kEY], prv[kEY], mv, kEY, n)) -
            (dz_below - dz_here);
        const double qb = (qline && i == i0 && j == j0) ? qline[k] : 0.0;
        me = fmax(me, fabs(qe - qb));
      }
      // Eq. (34) at the cell whose lower node is n: six faces active
      if ((m0 & 56) == 56 && mv(kHX, n + sx) != 0.0 && mv(kHY, n + sy) != 0.0 &&
          mv(kHZ, n + sz) != 0.0) {
        const double qh =
            (bbar(cur[kHX], prv[kHX], mv, kHX, n + sx) - bbar(cur[kHX], prv[kHX], mv, kHX, n)) +
            (bbar(cur[kHY], prv[kHY], mv, kHY, n + sy) - bbar(cur[kHY], prv[kHY], mv, kHY, n)) +
            (bz_above - bz_here);
        mh = fmax(mh, fabs(qh));
      }
      dz_below = dz_here;
      bz_here = bz_above;
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


}  // namespace

template <typename T>
cudaError_t launch_energy(const T* const f[6], const uint8_t* mask, const double* minv,
                          const double* const minv_a[6], const Layout& L, double alpha,
                          const WorkView& wv, const DiagScratch& s, double* result,
                          cudaStream_t st) {
  const int nb = wv.n_items;
  if (nb > s.cap) return cudaErrorInvalidValue;
  if (nb == 0) return cudaMemsetAsync(result, 0, sizeof(double), st);
  energy_items<T><<<nb, kBlock, 0, st>>>(f[0], f[1], f[2], f[3], f[4], f[5],
                                          make_view(mask, minv, minv_a), L, wv, alpha, s.part);
  reduce_pass2<false><<<1, 1024, 0, st>>>(s.part, nb, result);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_charge(const T* const cur[6], const T* const prev[6], const uint8_t* mask,
                          const double* minv, const double* const minv_a[6], const Layout& L,
                          double alpha, const double* qline, int i0, int j0, const WorkView& wv,
                          const DiagScratch& s, double* res_e, double* res_h, cudaStream_t st) {
  const int nb = wv.n_items;
  if (2 * nb > s.cap) return cudaErrorInvalidValue;
  if (nb == 0) {
    cudaError_t e = cudaMemsetAsync(res_e, 0, sizeof(double), st);
    return e != cudaSuccess ? e : cudaMemsetAsync(res_h, 0, sizeof(double), st);
  }
  ChargeFields cf;
  for (int c = 0; c < 6; ++c) {
    cf.cur[c] = cur[c];
    cf.prev[c] = prev[c];
  }
  charge_items<T><<<nb, kBlock, 0, st>>>(cf, make_view(mask, minv, minv_a), L, wv, alpha, qline,
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
                                          const WorkView&, const DiagScratch&, double*,
                                          cudaStream_t);
template cudaError_t launch_energy<double>(const double* const[6], const uint8_t*, const double*,
                                           const double* const[6], const Layout&, double,
                                           const WorkView&, const DiagScratch&, double*,
                                           cudaStream_t);
template cudaError_t launch_charge<float>(const float* const[6], const float* const[6],
                                          const uint8_t*, const double*, const double* const[6],
                                          const Layout&, double, const double*, int, int,
                                          const WorkView&, const DiagScratch&, double*, double*,
                                          cudaStream_t);
template cudaError_t launch_charge<double>(const double* const[6], const double* const[6],
                                           const uint8_t*, const double*, const double* const[6],
                                           const Layout&, double, const double*, int, int,
                                           const WorkView&, const DiagScratch&, double*, double*,
                                           cudaStream_t);

}  // namespace tetm
