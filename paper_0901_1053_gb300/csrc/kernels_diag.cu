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

// binary32 -> binary64 widening on the integer pipe (IEEE 754: the
// significand moves up by 29 bits and the exponent is rebiased by
// 1023 - 127 = 896, or set to all ones for infinities and NaNs, which keep
// their payload): exact for every normal value, zero, infinity and NaN.
// Subnormal values (below 2^-126) become zero of the same sign; a field value
// that small changes a balance term by less than 2^-126 of its normal
// neighbours. On this part the float64 unit, which the conversion
// instruction also occupies, is the balances' bottleneck.
__device__ __forceinline__ double wide(float f) {
  const unsigned u = __float_as_uint(f), a = u & 0x7FFFFFFFu;
  const bool normal = a >= 0x00800000u;
  const unsigned bias = a >= 0x7F800000u ? 0x70000000u : 0x38000000u;
  const unsigned hi = (u & 0x80000000u) | (normal ? (a >> 3) + bias : 0u);
  const unsigned lo = normal ? u << 29 : 0u;
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ double wide(double d) { return d; }

struct MinvView {
  const uint8_t* mask;
  double c[6];          // M^-1 constants (uniform material)
  double r[6];          // their reciprocals M = 1/M^-1
  const double* a[6];   // per-entry M^-1 (material runs) or nullptr
  const double* ra[6];  // and per-entry M = 1/M^-1 (0 where M^-1 is 0), formed once per solve
  __device__ __forceinline__ double operator()(int comp, long long id) const {
    if (a[comp]) return a[comp][id];
    return ((mask[id] >> comp) & 1) ? c[comp] : 0.0;
  }
  // M = 1/M^-1 of an active entry (0 for inactive ones)
  __device__ __forceinline__ double m(int comp, long long id) const {
    if (ra[comp]) return ra[comp][id];
    if (a[comp]) {  // per-entry M^-1 without its reciprocals
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
// [a L^T, I - a^2 R_1]], in integral variables, for float64 fields with
// per-entry material matrices: the share of node index (i,j,k) is
// 1/2 sum_c M_c f_c^2 - a^2/2 (M_mux^-1 (P_y ez)^2 + M_muy^-1 (P_x ez)^2 +
// M_epsx^-1 (P_y^T hz)^2 + M_epsy^-1 (P_x^T hz)^2) + a (hx P_z ey - hy P_z ex).
// One partial per work item.
template <typename T>
__global__ void energy_items(const T* __restrict__ ex, const T* __restrict__ ey,
                             const T* __restrict__ ez, const T* __restrict__ hx,
                             const T* __restrict__ hy, const T* __restrict__ hz, MinvView mv,
                             Layout L, WorkView wv, double alpha, double* part) {
  const int item = wv.items ? wv.items[blockIdx.x] : (int)blockIdx.x;
  const ItemCells ic(wv, L, item);
  const long long sx = 1, sy = L.px, sz = L.sz;
  const T* f[6] = {ex, ey, ez, hx, hy, hz};
  double acc = 0.0;
  for (int c = threadIdx.x; c < ic.tx * ic.ty; c += blockDim.x) {
    const int i = ic.i0 + c % ic.tx, j = ic.j0 + c / ic.tx;
    if (i >= L.nx || j >= L.ny) continue;
    for (int k = ic.k0; k < ic.k1; ++k) {
      const long long id = L.idx(i, j, k);
      const uint8_t m = mv.mask[id];
      if (m == 0) continue;  // no field object here: every term is zero
      const double pyez = wide(ez[id + sy]) - wide(ez[id]);
      const double pxez = wide(ez[id + sx]) - wide(ez[id]);
      const double ptyhz = wide(hz[id - sy]) - wide(hz[id]);
      const double ptxhz = wide(hz[id - sx]) - wide(hz[id]);
      const double l = wide(hx[id]) * (wide(ey[id + sz]) - wide(ey[id])) -
                       wide(hy[id]) * (wide(ex[id + sz]) - wide(ex[id]));
      double w = 0.0;
      for (int q = 0; q < 6; ++q) {
        const double v = wide(f[q][id]);
        w += 0.5 * v * v * mv.m(q, id);
      }
      const double r = mv(kHX, id) * pyez * pyez + mv(kHY, id) * pxez * pxez +
                       mv(kEX, id) * ptyhz * ptyhz + mv(kEY, id) * ptxhz * ptxhz;
      acc += w - 0.5 * alpha * alpha * r + alpha * l;
    }
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
  return 0.5 * (wide(f1[e]) + wide(f0[e])) * mv.m(comp, e);
}
template <typename T>
__device__ __forceinline__ double dz_tilde(const T* ez, const MinvView& mv, long long e,
                                           long long sx, long long sy, double a2) {
  const double mi = mv(kEZ, e);
  if (mi == 0.0) return 0.0;
  auto t1 = [&](long long f) { return mv(kHX, f) * (wide(ez[f + sy]) - wide(ez[f])); };
  auto t2 = [&](long long f) { return mv(kHY, f) * (wide(ez[f + sx]) - wide(ez[f])); };
  const double r = (t1(e - sy) - t1(e)) + (t2(e - sx) - t2(e));
  return wide(ez[e]) * mv.m(kEZ, e) - a2 * r;
}
template <typename T>
__device__ __forceinline__ double bbar(const T* f1, const T* f0, const MinvView& mv, int comp,
                                       long long f) {
  return 0.5 * (wide(f1[f]) + wide(f0[f])) * mv.m(comp, f);
}
template <typename T>
__device__ __forceinline__ double bz_tilde(const T* hz, const MinvView& mv, long long f,
                                           long long sx, long long sy, double a2) {
  const double mi = mv(kHZ, f);
  if (mi == 0.0) return 0.0;
  auto t3 = [&](long long e) { return mv(kEX, e) * (wide(hz[e - sy]) - wide(hz[e])); };
  auto t4 = [&](long long e) { return mv(kEY, e) * (wide(hz[e - sx]) - wide(hz[e])); };
  const double r = (t3(f + sy) - t3(f)) + (t4(f + sx) - t4(f));
  return wide(hz[f]) * mv.m(kHZ, f) - a2 * r;
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


// One material (the vacuum case included): M^-1 and M = 1 / M^-1 per
// component for the active entries, and the products the balances use.
struct UniformCoef {
  double c[6], r[6];
  double half_r[6];      // M / 2
  double a2c_hx, a2c_hy; // alpha^2 M^-1 of h_x, h_y faces
  double a2c_ex, a2c_ey; // alpha^2 M^-1 of e_x, e_y edges
  // float32 fields: the charges' ten coefficients, signs folded in, as float32
  // pairs (hi + lo equals the float64 value to 2^-48): Eq. (35) a2c_hx (Wy),
  // a2c_hy (Wx), -M_ez (Z), -M_ey/2 (Y), -M_ex/2 (X); Eq. (34) M_hx/2 (Bx),
  // M_hy/2 (By), M_hz (Hz), -a2c_ex (T3), -a2c_ey (T4)
  float qc[10][2];
};
template <typename T>
struct BalanceFields {
  const T* cur[6];   // y^n
  const T* prev[6];  // y^{n-1} (charges only)
};

// The energy of Sec. 4.4 and, with CHARGE, the charge residuals of Eqs. (35)
// and (34) in one pass over the nodes of a work item, for one material. A
// face that carries no field has both of its boundary edges in PEC, so the
// terms that the face coefficients weight, (P_y ez)^2, (P_x ez)^2 and the
// hx, hy parts of the corrected e_z flux, need no activity test (their ez
// values are zero); the terms that the edge coefficients weight keep it.
// Along z each thread carries the corrected z-fluxes of the node below and of
// its own face. Partials per block: energy, max |qe - qbunch|, max |qh|.
template <typename T, bool CHARGE>
__global__ void __launch_bounds__(256, 2) balance_items(BalanceFields<T> bf, const uint8_t* __restrict__ mask, UniformCoef uc, Layout L,
                              WorkView wv, double alpha, const double* qline, int i0, int j0, double* part_w,
                              double* part_e, double* part_h) {
  const T* __restrict__ ex = bf.cur[kEX];
  const T* __restrict__ ey = bf.cur[kEY];
  const T* __restrict__ ez = bf.cur[kEZ];
  const T* __restrict__ hx = bf.cur[kHX];
  const T* __restrict__ hy = bf.cur[kHY];
  const T* __restrict__ hz = bf.cur[kHZ];
  const int item = wv.items ? wv.items[blockIdx.x] : (int)blockIdx.x;
  const ItemCells ic(wv, L, item);
  const long long sx = 1, sy = L.px, sz = L.sz;
  const double a2 = alpha * alpha;
  double sq[6] = {0, 0, 0, 0, 0, 0};
  double rq[4] = {0, 0, 0, 0};
  double cross = 0.0, me = 0.0, mh = 0.0;
  // corrected z-flux of the active ez edge e (Eq. (35)) and of the active hz
  // face f of the previous state (Eq. (34))
  auto dz_at = [&](long long e) {
    const double z = wide(ez[e]);
    const double r = uc.a2c_hx * ((z - wide(ez[e - sy])) - (wide(ez[e + sy]) - z)) +
                     uc.a2c_hy * ((z - wide(ez[e - sx])) - (wide(ez[e + sx]) - z));
    return fma(z, uc.r[kEZ], -r);
  };
  auto bz_at = [&](long long f) {
    const T* __restrict__ phz = bf.prev[kHZ];
    const double z = wide(phz[f]);
    const unsigned mf = mask[f];
    const double t3a = (mask[f + sy] & 1) ? z - wide(phz[f + sy]) : 0.0;
    const double t3b = (mf & 1) ? wide(phz[f - sy]) - z : 0.0;
    const double t4a = (mask[f + sx] & 2) ? z - wide(phz[f + sx]) : 0.0;
    const double t4b = (mf & 2) ? wide(phz[f - sx]) - z : 0.0;
    const double r = uc.a2c_ex * (t3a - t3b) + uc.a2c_ey * (t4a - t4b);
    return fma(z, uc.r[kHZ], -r);
  };
  for (int c = threadIdx.x; c < ic.tx * ic.ty; c += blockDim.x) {
    const int i = ic.i0 + c % ic.tx, j = ic.j0 + c / ic.tx;
    if (i >= L.nx || j >= L.ny) continue;
    long long n = L.idx(i, j, ic.k0);
    double dz_prev = 0.0, bz_cur = 0.0;  // dz~ of the edge below, bz~ of this node's face
    bool dz_ok = false, bz_ok = false;
    for (int k = ic.k0; k < ic.k1; ++k, n += sz) {
      const unsigned m0 = mask[n];
      if (m0 == 0) {  // no field object here: every term is zero, and so is dz~
        dz_prev = 0.0;
        dz_ok = true;
        bz_ok = false;
        continue;
      }
      const double vex = wide(ex[n]), vey = wide(ey[n]), vez = wide(ez[n]);
      const double vhx = wide(hx[n]), vhy = wide(hy[n]), vhz = wide(hz[n]);
      sq[kEX] = fma(vex, vex, sq[kEX]);
      sq[kEY] = fma(vey, vey, sq[kEY]);
      sq[kEZ] = fma(vez, vez, sq[kEZ]);
      sq[kHX] = fma(vhx, vhx, sq[kHX]);
      sq[kHY] = fma(vhy, vhy, sq[kHY]);
      sq[kHZ] = fma(vhz, vhz, sq[kHZ]);
      const double Ly = wide(ez[n + sy]) - vez, Lx = wide(ez[n + sx]) - vez;
      rq[0] = fma(Ly, Ly, rq[0]);
      rq[1] = fma(Lx, Lx, rq[1]);
      if (m0 & 1) {
        const double Hy = wide(hz[n - sy]) - vhz;
        rq[2] = fma(Hy, Hy, rq[2]);
      }
      if (m0 & 2) {
        const double Hx = wide(hz[n - sx]) - vhz;
        rq[3] = fma(Hx, Hx, rq[3]);
      }
      const double dey = wide(ey[n + sz]) - vey, dex = wide(ex[n + sz]) - vex;
      cross = fma(vhx, dey, fma(-vhy, dex, cross));
      if constexpr (CHARGE) {
        double dz_here = 0.0;
        if (m0 & 4) {
          const double Lyd = vez - wide(ez[n - sy]), Lxd = vez - wide(ez[n - sx]);
          const double r = uc.a2c_hx * (Lyd - Ly) + uc.a2c_hy * (Lxd - Lx);
          dz_here = fma(vez, uc.r[kEZ], -r);
        }
        // Eq. (35) at node n: its six incident edges carry a field
        if ((m0 & 7) == 7 && (mask[n - sx] & 1) && (mask[n - sy] & 2) && (mask[n - sz] & 4)) {
          const double dzb = dz_ok ? dz_prev : dz_at(n - sz);
          const T* __restrict__ pex = bf.prev[kEX];
          const T* __restrict__ pey = bf.prev[kEY];
          const double sxn = vex + wide(pex[n]), sxl = wide(ex[n - sx]) + wide(pex[n - sx]);
          const double syn = vey + wide(pey[n]), syd = wide(ey[n - sy]) + wide(pey[n - sy]);
          double qe = -uc.half_r[kEX] * (sxl - sxn) - uc.half_r[kEY] * (syd - syn) - (dzb - dz_here);
          if (qline && i == i0 && j == j0) qe -= qline[k];
          me = fmax(me, fabs(qe));
        }
        dz_prev = dz_here;
        dz_ok = true;
        // Eq. (34) at the cell whose lower node is n: its six faces carry a field
        if ((m0 & 56) == 56 && (mask[n + sx] & 8) && (mask[n + sy] & 16) && (mask[n + sz] & 32)) {
          const double bzh = bz_ok ? bz_cur : bz_at(n);
          const double bza = bz_at(n + sz);
          const T* __restrict__ phx = bf.prev[kHX];
          const T* __restrict__ phy = bf.prev[kHY];
          const double bxn = vhx + wide(phx[n]), bxr = wide(hx[n + sx]) + wide(phx[n + sx]);
          const double byn = vhy + wide(phy[n]), byu = wide(hy[n + sy]) + wide(phy[n + sy]);
          const double qh = uc.half_r[kHX] * (bxr - bxn) + uc.half_r[kHY] * (byu - byn) + (bza - bzh);
          mh = fmax(mh, fabs(qh));
          bz_cur = bza;
          bz_ok = true;
        } else {
          bz_ok = false;
        }
      }
    }
  }
  double w = 0.0;
  for (int q = 0; q < 6; ++q) w += 0.5 * uc.r[q] * sq[q];
  w -= 0.5 * a2 * (uc.c[kHX] * rq[0] + uc.c[kHY] * rq[1] + uc.c[kEX] * rq[2] + uc.c[kEY] * rq[3]);
  w += alpha * cross;
  const double bw = block_reduce<false>(w);
  if (threadIdx.x == 0) part_w[blockIdx.x] = bw;
  if constexpr (CHARGE) {
    const double be = block_reduce<true>(me);
    const double bh = block_reduce<true>(mh);
    if (threadIdx.x == 0) {
      part_e[blockIdx.x] = be;
      part_h[blockIdx.x] = bh;
    }
  }
}

// ---- float32 fields: error-free transformations on the float32 pipe -------
// A float32 value pair (hi, lo) stands for the exact sum hi + lo. two_sum and
// two_prod are the error-free sum (Knuth) and product (with a fused
// multiply-add) of two float32 values; sums of a few float32 values with
// integer coefficients come out exactly, or within 2^-47 of their size, as a
// pair, and enter float64 through the exact widening and one float64 add.
struct F2 {
  float hi, lo;
};
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return F2{s, e};
}
__device__ __forceinline__ F2 two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return F2{p, fmaf(a, b, -p)};
}
// running sum of signed float32 terms
__device__ __forceinline__ F2 f2_add(F2 s, float v) {
  const F2 t = two_sum(s.hi, v);
  return F2{t.hi, __fadd_rn(s.lo, t.lo)};
}
__device__ __forceinline__ double f2_wide(F2 s) { return wide(s.hi) + wide(s.lo); }
// accumulator += (p + e) for a product term p + e with |e| << |p|
__device__ __forceinline__ void f2_acc(F2& acc, float p, float e) {
  const F2 t = two_sum(acc.hi, p);
  const float lo = __fadd_rn(t.lo, __fadd_rn(acc.lo, e));
  const float hi = __fadd_rn(t.hi, lo);
  acc = F2{hi, __fsub_rn(lo, __fsub_rn(hi, t.hi))};
}
// acc += a^2 (a float32), acc += d^2 and acc += a d (d a pair)
__device__ __forceinline__ void acc_sq(F2& acc, float a) {
  const F2 p = two_prod(a, a);
  f2_acc(acc, p.hi, p.lo);
}
__device__ __forceinline__ void acc_sq2(F2& acc, F2 d) {
  const F2 p = two_prod(d.hi, d.hi);
  f2_acc(acc, p.hi, fmaf(2.f * d.hi, d.lo, p.lo));
}
__device__ __forceinline__ void acc_mul2(F2& acc, float a, F2 d) {
  const F2 p = two_prod(a, d.hi);
  f2_acc(acc, p.hi, fmaf(a, d.lo, p.lo));
}

// acc += c t for a coefficient pair c and a term pair t, on the float32 pipe
// (the product's dropped part c.lo t.lo is below 2^-48 of it)
__device__ __forceinline__ void acc_prod(F2& acc, F2 c, F2 t) {
  const F2 p = two_prod(c.hi, t.hi);
  f2_acc(acc, p.hi, fmaf(c.hi, t.lo, fmaf(c.lo, t.hi, p.lo)));
}

constexpr int kFlush = 8;  // nodes per float32-pair partial before it joins the float64 sum
constexpr int kPre = 4;    // planes of L2 prefetch ahead of the node being summed

// balance_items for float32 fields: the same quantities, formed term by term
// with the transformations above. Energy: eleven pair accumulators (six
// squares, four link squares, the cross term) flushed into float64 sums every
// kFlush nodes. Charges: Eq. (35) at node n is
//   -M_x/2 X - M_y/2 Y - M_z Z + a^2 M_hx^-1 Wy + a^2 M_hy^-1 Wx,
// X = (ex1 + ex0)(n - sx) - (ex1 + ex0)(n), Y likewise in y, Z = ez(n - sz) -
// ez(n), Wy = Ly(n - sz) - Ly(n) with Ly(e) = 2 ez(e) - ez(e - sy) - ez(e + sy)
// (Wx likewise in x): five integer combinations of float32 values. Eq. (34)
// at the cell of lower node n is M_hx/2 Bx + M_hy/2 By + M_z Hz - a^2 M_ex^-1
// T3 - a^2 M_ey^-1 T4 over the previous h_z with the e_x, e_y edge tests.
template <bool CHARGE>
__global__ void __launch_bounds__(256, 4)
balance_items_f32(BalanceFields<float> bf, const uint8_t* __restrict__ mask, UniformCoef uc, Layout L,
                  WorkView wv, double alpha, const double* qline, int i0, int j0, double* part_w,
                  double* part_e, double* part_h) {
  const float* __restrict__ ex = bf.cur[kEX];
  const float* __restrict__ ey = bf.cur[kEY];
  const float* __restrict__ ez = bf.cur[kEZ];
  const float* __restrict__ hx = bf.cur[kHX];
  const float* __restrict__ hy = bf.cur[kHY];
  const float* __restrict__ hz = bf.cur[kHZ];
  const int item = wv.items ? wv.items[blockIdx.x] : (int)blockIdx.x;
  const ItemCells ic(wv, L, item);
  const long long sx = 1, sy = L.px, sz = L.sz;
  // weights of the eleven sums in the energy
  const double a2h = 0.5 * alpha * alpha;
  const double wt[11] = {uc.half_r[0], uc.half_r[1], uc.half_r[2], uc.half_r[3], uc.half_r[4], uc.half_r[5],
                         -a2h * uc.c[kHX], -a2h * uc.c[kHY], -a2h * uc.c[kEX], -a2h * uc.c[kEY], alpha};
  F2 acc[11];
#pragma unroll
  for (int q = 0; q < 11; ++q) acc[q] = F2{0.f, 0.f};
  double w = 0.0;
  int cnt = 0;
  double me = 0.0, mh = 0.0;
  // each charge is summed as one float32 pair (coefficient pairs from the
  // parameters) and widened once
  auto cq = [&](int q) { return F2{uc.qc[q][0], uc.qc[q][1]}; };
  auto flush = [&]() {
#pragma unroll
    for (int q = 0; q < 11; ++q) {
      w = fma(wt[q], f2_wide(acc[q]), w);
      acc[q] = F2{0.f, 0.f};
    }
    cnt = 0;
  };
  // the entries of this thread's node kPre planes on, into L2 ahead of use
  // (the kernel is bound by the latency of its loads)
  auto prefetch = [&](long long m) {
#pragma unroll
    for (int q = 0; q < 6; ++q) asm volatile("prefetch.global.L2 [%0];" ::"l"(bf.cur[q] + m));
    if constexpr (CHARGE) {
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if (q != kEZ) asm volatile("prefetch.global.L2 [%0];" ::"l"(bf.prev[q] + m));
    }
    asm volatile("prefetch.global.L2 [%0];" ::"l"(mask + m));
  };
  for (int c = threadIdx.x; c < ic.tx * ic.ty; c += blockDim.x) {
    const int i = ic.i0 + c % ic.tx, j = ic.j0 + c / ic.tx;
    if (i >= L.nx || j >= L.ny) continue;
    long long n = L.idx(i, j, ic.k0);
    for (int d = 0; d < kPre && ic.k0 + d < ic.k1; ++d) prefetch(n + d * sz);
    for (int k = ic.k0; k < ic.k1; ++k, n += sz) {
      if (k + kPre < ic.k1) prefetch(n + kPre * sz);
      const unsigned m0 = mask[n];
      if (m0 == 0) continue;  // no field object here: every term is zero
      const float vex = ex[n], vey = ey[n], vez = ez[n], vhx = hx[n], vhy = hy[n], vhz = hz[n];
      acc_sq(acc[kEX], vex);
      acc_sq(acc[kEY], vey);
      acc_sq(acc[kEZ], vez);
      acc_sq(acc[kHX], vhx);
      acc_sq(acc[kHY], vhy);
      acc_sq(acc[kHZ], vhz);
      acc_sq2(acc[6], two_sum(ez[n + sy], -vez));
      acc_sq2(acc[7], two_sum(ez[n + sx], -vez));
      if (m0 & 1) acc_sq2(acc[8], two_sum(hz[n - sy], -vhz));
      if (m0 & 2) acc_sq2(acc[9], two_sum(hz[n - sx], -vhz));
      acc_mul2(acc[10], vhx, two_sum(ey[n + sz], -vey));
      acc_mul2(acc[10], -vhy, two_sum(ex[n + sz], -vex));
      if (++cnt == kFlush) flush();
      if constexpr (CHARGE) {
        if ((m0 & 7) == 7 && (mask[n - sx] & 1) && (mask[n - sy] & 2) && (mask[n - sz] & 4)) {
          const float* __restrict__ pex = bf.prev[kEX];
          const float* __restrict__ pey = bf.prev[kEY];
          const F2 X = f2_add(f2_add(f2_add(F2{ex[n - sx], 0.f}, pex[n - sx]), -vex), -pex[n]);
          const F2 Y = f2_add(f2_add(f2_add(F2{ey[n - sy], 0.f}, pey[n - sy]), -vey), -pey[n]);
          const float ezb = ez[n - sz];
          const F2 Z = two_sum(ezb, -vez);
          const F2 Wy = f2_add(f2_add(f2_add(f2_add(f2_add(F2{2.f * ezb, 0.f}, -ez[n - sz - sy]), -ez[n - sz + sy]),
                                             -2.f * vez), ez[n - sy]), ez[n + sy]);
          const F2 Wx = f2_add(f2_add(f2_add(f2_add(f2_add(F2{2.f * ezb, 0.f}, -ez[n - sz - sx]), -ez[n - sz + sx]),
                                             -2.f * vez), ez[n - sx]), ez[n + sx]);
          F2 qs{0.f, 0.f};
          acc_prod(qs, cq(0), Wy);
          acc_prod(qs, cq(1), Wx);
          acc_prod(qs, cq(2), Z);
          acc_prod(qs, cq(3), Y);
          acc_prod(qs, cq(4), X);
          double qe = f2_wide(qs);
          if (qline && i == i0 && j == j0) qe -= qline[k];
          me = fmax(me, fabs(qe));
        }
        if ((m0 & 56) == 56 && (mask[n + sx] & 8) && (mask[n + sy] & 16) && (mask[n + sz] & 32)) {
          const float* __restrict__ phx = bf.prev[kHX];
          const float* __restrict__ phy = bf.prev[kHY];
          const float* __restrict__ phz = bf.prev[kHZ];
          const F2 Bx = f2_add(f2_add(f2_add(F2{hx[n + sx], 0.f}, phx[n + sx]), -vhx), -phx[n]);
          const F2 By = f2_add(f2_add(f2_add(F2{hy[n + sy], 0.f}, phy[n + sy]), -vhy), -phy[n]);
          const long long f1 = n + sz;
          const float z1 = phz[f1], z0 = phz[n];
          const F2 Hz = two_sum(z1, -z0);
          // t3(f) = [e_x(f + sy)] (hz(f) - hz(f + sy)) - [e_x(f)] (hz(f - sy) - hz(f)), T3 = t3(n + sz) - t3(n)
          F2 T3{0.f, 0.f}, T4{0.f, 0.f};
          if (mask[f1 + sy] & 1) T3 = f2_add(f2_add(T3, z1), -phz[f1 + sy]);
          if (mask[f1] & 1) T3 = f2_add(f2_add(T3, -phz[f1 - sy]), z1);
          if (mask[n + sy] & 1) T3 = f2_add(f2_add(T3, -z0), phz[n + sy]);
          if (m0 & 1) T3 = f2_add(f2_add(T3, phz[n - sy]), -z0);
          if (mask[f1 + sx] & 2) T4 = f2_add(f2_add(T4, z1), -phz[f1 + sx]);
          if (mask[f1] & 2) T4 = f2_add(f2_add(T4, -phz[f1 - sx]), z1);
          if (mask[n + sx] & 2) T4 = f2_add(f2_add(T4, -z0), phz[n + sx]);
          if (m0 & 2) T4 = f2_add(f2_add(T4, phz[n - sx]), -z0);
          F2 qs{0.f, 0.f};
          acc_prod(qs, cq(5), Bx);
          acc_prod(qs, cq(6), By);
          acc_prod(qs, cq(7), Hz);
          acc_prod(qs, cq(8), T3);
          acc_prod(qs, cq(9), T4);
          mh = fmax(mh, fabs(f2_wide(qs)));
        }
      }
    }
  }
  flush();
  const double bw = block_reduce<false>(w);
  if (threadIdx.x == 0) part_w[blockIdx.x] = bw;
  if constexpr (CHARGE) {
    const double be = block_reduce<true>(me);
    const double bh = block_reduce<true>(mh);
    if (threadIdx.x == 0) {
      part_e[blockIdx.x] = be;
      part_h[blockIdx.x] = bh;
    }
  }
}

// balance_items_f32 with per-entry coefficients (material arrays): every
// term of the energy and of Eqs. (35)/(34) is a coefficient of its own entry
// times a sum of float32 values, so each is formed as the product of the
// coefficient as a float32 pair (m: M = 1/M^-1 of the six components; a:
// alpha^2 M^-1 of h_x, h_y, e_x, e_y) and the exact pair of the sum, and the
// products are summed as pairs. Energy: three pair accumulators (sum M v^2,
// sum alpha^2 M^-1 d^2 over the four link differences, the cross term),
// flushed into float64 every kFlush nodes. Charges: the corrected z-fluxes of
// the edge below and of the face above (previous h_z) are carried up the
// column as pairs, each charge is summed as one pair and widened once.
struct MatPairs {
  const float2* m[6];  // M per component
  const float2* a[6];  // alpha^2 M^-1 (entries kHX, kHY, kEX, kEY used)
};
template <bool CHARGE>
__global__ void __launch_bounds__(256, 2)
balance_items_mat_f32(BalanceFields<float> bf, const uint8_t* __restrict__ mask, MatPairs mp, Layout L,
                      WorkView wv, double alpha, const double* qline, int i0, int j0, double* part_w,
                      double* part_e, double* part_h) {
  const float* __restrict__ ex = bf.cur[kEX];
  const float* __restrict__ ey = bf.cur[kEY];
  const float* __restrict__ ez = bf.cur[kEZ];
  const float* __restrict__ hx = bf.cur[kHX];
  const float* __restrict__ hy = bf.cur[kHY];
  const float* __restrict__ hz = bf.cur[kHZ];
  const int item = wv.items ? wv.items[blockIdx.x] : (int)blockIdx.x;
  const ItemCells ic(wv, L, item);
  const long long sx = 1, sy = L.px, sz = L.sz;
  auto M = [&](int c, long long e) { const float2 v = mp.m[c][e]; return F2{v.x, v.y}; };
  auto A = [&](int c, long long e) { const float2 v = mp.a[c][e]; return F2{v.x, v.y}; };
  // d^2 of an exact pair d, as a pair (the dropped d.lo^2 is below 2^-48 of it)
  auto sq2 = [](F2 d) {
    const F2 p = two_prod(d.hi, d.hi);
    return F2{p.hi, fmaf(2.f * d.hi, d.lo, p.lo)};
  };
  auto neg = [](F2 d) { return F2{-d.hi, -d.lo}; };
  F2 accW{0.f, 0.f}, accR{0.f, 0.f}, accL{0.f, 0.f};
  double w = 0.0;
  int cnt = 0;
  double me = 0.0, mh = 0.0;
  auto flush = [&]() {
    w = fma(0.5, f2_wide(accW), w);
    w = fma(-0.5, f2_wide(accR), w);
    w = fma(alpha, f2_wide(accL), w);
    accW = accR = accL = F2{0.f, 0.f};
    cnt = 0;
  };
  // corrected z-flux of edge e (Eq. (35)): M_ez ez - a2 [(t1(e-sy) - t1(e)) +
  // (t2(e-sx) - t2(e))], t1(f) = M^-1_hx(f) (ez(f+sy) - ez(f)), t2 likewise
  // in x; zero on an edge without a field
  auto dz_at = [&](long long e) {
    F2 acc{0.f, 0.f};
    if (!(mask[e] & 4)) return acc;
    const float z = ez[e];
    acc_prod(acc, M(kEZ, e), F2{z, 0.f});
    acc_prod(acc, A(kHX, e - sy), two_sum(ez[e - sy], -z));
    acc_prod(acc, A(kHX, e), two_sum(ez[e + sy], -z));
    acc_prod(acc, A(kHY, e - sx), two_sum(ez[e - sx], -z));
    acc_prod(acc, A(kHY, e), two_sum(ez[e + sx], -z));
    return acc;
  };
  // corrected z-flux of face f of the previous state (Eq. (34)): M_hz hz -
  // a2 [(t3(f+sy) - t3(f)) + (t4(f+sx) - t4(f))], t3(e) = M^-1_ex(e)
  // (hz(e-sy) - hz(e)), t4 likewise in x; zero on a face without a field
  auto bz_at = [&](long long f) {
    F2 acc{0.f, 0.f};
    if (!(mask[f] & 32)) return acc;
    const float* __restrict__ phz = bf.prev[kHZ];
    const float z = phz[f];
    acc_prod(acc, M(kHZ, f), F2{z, 0.f});
    acc_prod(acc, A(kEX, f + sy), two_sum(phz[f + sy], -z));
    acc_prod(acc, A(kEX, f), two_sum(phz[f - sy], -z));
    acc_prod(acc, A(kEY, f + sx), two_sum(phz[f + sx], -z));
    acc_prod(acc, A(kEY, f), two_sum(phz[f - sx], -z));
    return acc;
  };
  for (int c = threadIdx.x; c < ic.tx * ic.ty; c += blockDim.x) {
    const int i = ic.i0 + c % ic.tx, j = ic.j0 + c / ic.tx;
    if (i >= L.nx || j >= L.ny) continue;
    long long n = L.idx(i, j, ic.k0);
    F2 dz_below{0.f, 0.f}, bz_here{0.f, 0.f};
    if constexpr (CHARGE) {
      dz_below = dz_at(n - sz);
      bz_here = bz_at(n);
    }
    for (int k = ic.k0; k < ic.k1; ++k, n += sz) {
      const unsigned m0 = mask[n];
      F2 dz_here{0.f, 0.f}, bz_above{0.f, 0.f};
      if constexpr (CHARGE) {
        dz_here = dz_at(n);
        bz_above = bz_at(n + sz);
      }
      if (m0 != 0) {  // no field object here: every energy term is zero
        const float vex = ex[n], vey = ey[n], vez = ez[n], vhx = hx[n], vhy = hy[n], vhz = hz[n];
        acc_prod(accW, M(kEX, n), two_prod(vex, vex));
        acc_prod(accW, M(kEY, n), two_prod(vey, vey));
        acc_prod(accW, M(kEZ, n), two_prod(vez, vez));
        acc_prod(accW, M(kHX, n), two_prod(vhx, vhx));
        acc_prod(accW, M(kHY, n), two_prod(vhy, vhy));
        acc_prod(accW, M(kHZ, n), two_prod(vhz, vhz));
        acc_prod(accR, A(kHX, n), sq2(two_sum(ez[n + sy], -vez)));
        acc_prod(accR, A(kHY, n), sq2(two_sum(ez[n + sx], -vez)));
        acc_prod(accR, A(kEX, n), sq2(two_sum(hz[n - sy], -vhz)));
        acc_prod(accR, A(kEY, n), sq2(two_sum(hz[n - sx], -vhz)));
        acc_mul2(accL, vhx, two_sum(ey[n + sz], -vey));
        acc_mul2(accL, -vhy, two_sum(ex[n + sz], -vex));
        if (++cnt == kFlush) flush();
      }
      if constexpr (CHARGE) {
        // Eq. (35) at node n: its six incident edges carry a field
        if ((m0 & 7) == 7 && (mask[n - sx] & 1) && (mask[n - sy] & 2) && (mask[n - sz] & 4)) {
          const float* __restrict__ pex = bf.prev[kEX];
          const float* __restrict__ pey = bf.prev[kEY];
          const F2 Sxl = two_sum(0.5f * ex[n - sx], 0.5f * pex[n - sx]);
          const F2 Sxn = two_sum(0.5f * ex[n], 0.5f * pex[n]);
          const F2 Syd = two_sum(0.5f * ey[n - sy], 0.5f * pey[n - sy]);
          const F2 Syn = two_sum(0.5f * ey[n], 0.5f * pey[n]);
          F2 qs{0.f, 0.f};
          acc_prod(qs, M(kEX, n - sx), neg(Sxl));
          acc_prod(qs, M(kEX, n), Sxn);
          acc_prod(qs, M(kEY, n - sy), neg(Syd));
          acc_prod(qs, M(kEY, n), Syn);
          f2_acc(qs, -dz_below.hi, -dz_below.lo);
          f2_acc(qs, dz_here.hi, dz_here.lo);
          double qe = f2_wide(qs);
          if (qline && i == i0 && j == j0) qe -= qline[k];
          me = fmax(me, fabs(qe));
        }
        // Eq. (34) at the cell whose lower node is n: its six faces carry a field
        if ((m0 & 56) == 56 && (mask[n + sx] & 8) && (mask[n + sy] & 16) && (mask[n + sz] & 32)) {
          const float* __restrict__ phx = bf.prev[kHX];
          const float* __restrict__ phy = bf.prev[kHY];
          const F2 Bxr = two_sum(0.5f * hx[n + sx], 0.5f * phx[n + sx]);
          const F2 Bxn = two_sum(0.5f * hx[n], 0.5f * phx[n]);
          const F2 Byu = two_sum(0.5f * hy[n + sy], 0.5f * phy[n + sy]);
          const F2 Byn = two_sum(0.5f * hy[n], 0.5f * phy[n]);
          F2 qs{0.f, 0.f};
          acc_prod(qs, M(kHX, n + sx), Bxr);
          acc_prod(qs, M(kHX, n), neg(Bxn));
          acc_prod(qs, M(kHY, n + sy), Byu);
          acc_prod(qs, M(kHY, n), neg(Byn));
          f2_acc(qs, bz_above.hi, bz_above.lo);
          f2_acc(qs, -bz_here.hi, -bz_here.lo);
          mh = fmax(mh, fabs(f2_wide(qs)));
        }
        dz_below = dz_here;
        bz_here = bz_above;
      }
    }
  }
  flush();
  const double bw = block_reduce<false>(w);
  if (threadIdx.x == 0) part_w[blockIdx.x] = bw;
  if constexpr (CHARGE) {
    const double be = block_reduce<true>(me);
    const double bh = block_reduce<true>(mh);
    if (threadIdx.x == 0) {
      part_e[blockIdx.x] = be;
      part_h[blockIdx.x] = bh;
    }
  }
}

// The three totals of balance_items: sum of the energy partials, maxima of
// the two charge partials.
__global__ void balance_pass2(const double* part_w, const double* part_e, const double* part_h, int n,
                              double* out_w, double* out_e, double* out_h) {
  double w = 0.0, e = 0.0, h = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    w += part_w[q];
    if (part_e) {
      e = fmax(e, part_e[q]);
      h = fmax(h, part_h[q]);
    }
  }
  w = block_reduce<false>(w);
  if (part_e) {
    e = block_reduce<true>(e);
    h = block_reduce<true>(h);
  }
  if (threadIdx.x == 0) {
    *out_w = w;
    if (part_e) {
      *out_e = e;
      *out_h = h;
    }
  }
}

// threads per item: whole warps splitting the tile's columns evenly (224 for
// a 56 x 28 tile)
int balance_threads(const WorkView& wv) {
  const int area = wv.tile_x * wv.tile_y;
  const int rounds = (area + 255) / 256;
  return ((area + rounds - 1) / rounds + 31) / 32 * 32;
}

MinvView make_view(const uint8_t* mask, const double* minv, const double* const minv_a[6],
                   const double* const m_a[6]) {
  MinvView v;
  v.mask = mask;
  for (int c = 0; c < 6; ++c) {
    v.c[c] = minv ? minv[c] : 0.0;
    v.r[c] = (minv && minv[c] != 0.0) ? 1.0 / minv[c] : 0.0;
    v.a[c] = minv_a ? minv_a[c] : nullptr;
    v.ra[c] = m_a ? m_a[c] : nullptr;
  }
  return v;
}


}  // namespace

template <typename T>
cudaError_t launch_energy(const T* const f[6], const uint8_t* mask, const double* minv,
                          const double* const minv_a[6], const double* const m_a[6], const Layout& L, double alpha,
                          const WorkView& wv, const DiagScratch& s, double* result,
                          cudaStream_t st) {
  const int nb = wv.n_items;
  if (nb > s.cap) return cudaErrorInvalidValue;
  if (nb == 0) return cudaMemsetAsync(result, 0, sizeof(double), st);
  energy_items<T><<<nb, kBlock, 0, st>>>(f[0], f[1], f[2], f[3], f[4], f[5],
                                          make_view(mask, minv, minv_a, m_a), L, wv, alpha, s.part);
  reduce_pass2<false><<<1, 1024, 0, st>>>(s.part, nb, result);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_charge(const T* const cur[6], const T* const prev[6], const uint8_t* mask,
                          const double* minv, const double* const minv_a[6], const double* const m_a[6],
                          const Layout& L,
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
  charge_items<T><<<nb, kBlock, 0, st>>>(cf, make_view(mask, minv, minv_a, m_a), L, wv, alpha, qline,
                                          i0, j0, s.part, s.part + nb);
  reduce_pass2<true><<<1, 1024, 0, st>>>(s.part, nb, res_e);
  reduce_pass2<true><<<1, 1024, 0, st>>>(s.part + nb, nb, res_h);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_balances(const T* const cur[6], const T* const prev[6], const uint8_t* mask,
                            const double* minv, const Layout& L, double alpha, const double* qline, int i0,
                            int j0, const WorkView& wv, const DiagScratch& s, double* res_w, double* res_e,
                            double* res_h, cudaStream_t st) {
  const int nb = wv.n_items;
  if (3 * nb > s.cap) return cudaErrorInvalidValue;
  if (nb == 0) {
    cudaError_t e = cudaMemsetAsync(res_w, 0, sizeof(double), st);
    if (e == cudaSuccess && prev) e = cudaMemsetAsync(res_e, 0, sizeof(double), st);
    if (e == cudaSuccess && prev) e = cudaMemsetAsync(res_h, 0, sizeof(double), st);
    return e;
  }
  BalanceFields<T> bf;
  UniformCoef uc;
  for (int c = 0; c < 6; ++c) {
    bf.cur[c] = cur[c];
    bf.prev[c] = prev ? prev[c] : nullptr;
    uc.c[c] = minv[c];
    uc.r[c] = minv[c] != 0.0 ? 1.0 / minv[c] : 0.0;
    uc.half_r[c] = 0.5 * uc.r[c];
  }
  uc.a2c_hx = alpha * alpha * minv[kHX];
  uc.a2c_hy = alpha * alpha * minv[kHY];
  uc.a2c_ex = alpha * alpha * minv[kEX];
  uc.a2c_ey = alpha * alpha * minv[kEY];
  const double qcd[10] = {uc.a2c_hx,       uc.a2c_hy,       -uc.r[kEZ], -uc.half_r[kEY], -uc.half_r[kEX],
                          uc.half_r[kHX], uc.half_r[kHY], uc.r[kHZ],  -uc.a2c_ex,      -uc.a2c_ey};
  for (int q = 0; q < 10; ++q) {
    const float hi = (float)qcd[q];
    uc.qc[q][0] = hi;
    uc.qc[q][1] = (float)(qcd[q] - (double)hi);
  }
  const int nt = balance_threads(wv);
  if constexpr (sizeof(T) == 4) {  // float32 fields: the float32-pipe transformations
    if (prev)
      balance_items_f32<true><<<nb, nt, 0, st>>>(bf, mask, uc, L, wv, alpha, qline, i0, j0, s.part, s.part + nb,
                                                 s.part + 2 * nb);
    else
      balance_items_f32<false><<<nb, nt, 0, st>>>(bf, mask, uc, L, wv, alpha, nullptr, 0, 0, s.part, nullptr,
                                                  nullptr);
    balance_pass2<<<1, 1024, 0, st>>>(s.part, prev ? s.part + nb : nullptr, prev ? s.part + 2 * nb : nullptr, nb,
                                      res_w, res_e, res_h);
    return cudaGetLastError();
  } else {
  if (prev) {
    balance_items<T, true><<<nb, nt, 0, st>>>(bf, mask, uc, L, wv, alpha, qline, i0, j0, s.part, s.part + nb,
                                              s.part + 2 * nb);
    balance_pass2<<<1, 1024, 0, st>>>(s.part, s.part + nb, s.part + 2 * nb, nb, res_w, res_e, res_h);
  } else {
    balance_items<T, false><<<nb, nt, 0, st>>>(bf, mask, uc, L, wv, alpha, nullptr, 0, 0, s.part, nullptr,
                                               nullptr);
    balance_pass2<<<1, 1024, 0, st>>>(s.part, nullptr, nullptr, nb, res_w, nullptr, nullptr);
  }
  return cudaGetLastError();
  }
}
cudaError_t launch_balances_mat_f32(const float* const cur[6], const float* const prev[6], const uint8_t* mask,
                                   const float2* const m[6], const float2* const a[6], const Layout& L,
                                   double alpha, const double* qline, int i0, int j0, const WorkView& wv,
                                   const DiagScratch& s, double* res_w, double* res_e, double* res_h,
                                   cudaStream_t st) {
  const int nb = wv.n_items;
  if (3 * nb > s.cap) return cudaErrorInvalidValue;
  if (nb == 0) {
    cudaError_t e = cudaMemsetAsync(res_w, 0, sizeof(double), st);
    if (e == cudaSuccess && prev) e = cudaMemsetAsync(res_e, 0, sizeof(double), st);
    if (e == cudaSuccess && prev) e = cudaMemsetAsync(res_h, 0, sizeof(double), st);
    return e;
  }
  BalanceFields<float> bf;
  MatPairs mp;
  for (int c = 0; c < 6; ++c) {
    bf.cur[c] = cur[c];
    bf.prev[c] = prev ? prev[c] : nullptr;
    mp.m[c] = m[c];
    mp.a[c] = a[c];
  }
  const int nt = balance_threads(wv);
  if (prev)
    balance_items_mat_f32<true><<<nb, nt, 0, st>>>(bf, mask, mp, L, wv, alpha, qline, i0, j0, s.part,
                                                   s.part + nb, s.part + 2 * nb);
  else
    balance_items_mat_f32<false><<<nb, nt, 0, st>>>(bf, mask, mp, L, wv, alpha, nullptr, 0, 0, s.part, nullptr,
                                                    nullptr);
  balance_pass2<<<1, 1024, 0, st>>>(s.part, prev ? s.part + nb : nullptr, prev ? s.part + 2 * nb : nullptr, nb,
                                    res_w, res_e, res_h);
  return cudaGetLastError();
}

template cudaError_t launch_balances<float>(const float* const[6], const float* const[6], const uint8_t*,
                                            const double*, const Layout&, double, const double*, int, int,
                                            const WorkView&, const DiagScratch&, double*, double*, double*,
                                            cudaStream_t);
template cudaError_t launch_balances<double>(const double* const[6], const double* const[6], const uint8_t*,
                                             const double*, const Layout&, double, const double*, int, int,
                                             const WorkView&, const DiagScratch&, double*, double*, double*,
                                             cudaStream_t);

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

template cudaError_t launch_energy<double>(const double* const[6], const uint8_t*, const double*,
                                           const double* const[6], const double* const[6], const Layout&, double,
                                           const WorkView&, const DiagScratch&, double*,
                                           cudaStream_t);
template cudaError_t launch_charge<double>(const double* const[6], const double* const[6],
                                           const uint8_t*, const double*, const double* const[6], const double* const[6],
                                           const Layout&, double, const double*, int, int,
                                           const WorkView&, const DiagScratch&, double*, double*,
                                           cudaStream_t);

}  // namespace tetm
