// Rotationally symmetric explicit TE/TM scheme (Sec. 4.3, Eq. (24)): a set of
// azimuthal modes advanced together on one (r, z) grid, with a ring bunch and
// the wake of every mode.
//
// Device layout. Fields are stored entry-interleaved: for each mode and each
// row k = -1..nz+1 (plane k of the canonical layout), columns i = -or..pr-or-1
// with the axis i = 0 at column `or`, and per column the six components
// (e_r, e_phi, e_z, h_r, h_phi, h_z) side by side. Entry (mode, comp, i, k) is
// element ((mode * rows + k + 1) * pr + i + or) * 6 + comp. The activity mask
// (one byte per entry, shared by the modes) has the same rows and columns.
// Entries outside 0..nr, 0..nz hold zero and are inactive, so the stencils
// and prefetches read them without bounds checks. Two field sets (ping-pong).
//
// Metric. In the vacuum staircase geometry every coefficient depends on r
// alone: per mode and radial index the kernel keeps alpha*M^-1 of e_r, e_phi,
// h_r, h_phi, 2 alpha*M^-1 of e_z, h_z and the two diagonal factors of (24) in
// registers; the activity byte of an entry says which objects are non-PEC.
//
// Kernel. One warp per (mode, radial tile of 60 entries, z chunk) item. Lane l
// holds the two consecutive entries 2l, 2l+1 of a 64-entry window (2 halo
// entries on each side, which is what the r-differences of the ten updates
// reach), so its six components of both entries are 48 contiguous bytes in
// float32 (three 16-byte loads) and 96 in float64. The warp marches through
// the chunk plane by plane: at plane k it completes the TM stage (h_phi, h_r,
// e_z) with the old e of plane k+1 and then the TE stage (e_phi, e_r, h_z)
// with the new h of planes k-1 and k, so each plane is read once and written
// once; r-neighbours come from the lane's other entry or a shuffle. The TM
// stage of the plane before the chunk is recomputed (not written) to supply
// h^{n+1/2} at k0-1. A plane whose 64 entries are all fully active takes a
// path without the per-object activity selects. Two variants differ in how
// the loads run ahead: a register ring, or asynchronous copies into a
// shared-memory ring.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "tetm_internal.h"
#include "tetm_rz.h"
#include <nvtx3/nvToolsExt.h>

namespace {

using tetm::kC;
using tetm::kEps0;
using tetm::kMu0;

constexpr int kER = TETM_RZ_ER, kEP = TETM_RZ_EPHI, kEZ = TETM_RZ_EZ;
constexpr int kHR = TETM_RZ_HR, kHP = TETM_RZ_HPHI, kHZ = TETM_RZ_HZ;
constexpr double kPi = 3.14159265358979323846;
constexpr int kTile = 60;   // entries a warp owns (64-entry window minus 2 + 2 halo)
constexpr int kTile2 = 56;  // the same for two steps per pass (4 + 4 halo)
// scattered-field form: steps whose sources one launch computes (a power of 2)
constexpr int kSourceSlots = 8;
// scattered-field form: planes per work item of the step kernels over the
// items meeting a source window
constexpr int kSubPlanes = 4;
// planes held ahead: register ring (float32 / float64) and shared-memory ring
template <typename T>
__host__ __device__ constexpr int ring_depth() { return sizeof(T) == 4 ? 3 : 2; }
// resident blocks of 128 threads the register variant is compiled for
template <typename T>
__host__ __device__ constexpr int reg_min_blocks() { return sizeof(T) == 4 ? 4 : 1; }
template <typename T>
__host__ __device__ constexpr int async_depth() { return sizeof(T) == 4 ? 8 : 4; }
// per-mode coefficient rows: alpha M^-1 (er, ephi, hr, hphi), 2 alpha M^-1
// (ez, hz), and the diagonal factors 2 alpha M^-1 / (1 + alpha^2 m^2 M^-1 M^-1)
// of e_z (paired with h_r) and h_z (paired with e_r)
enum { kCoER = 0, kCoEP, kCoEZ, kCoHR, kCoHP, kCoHZ, kCoFEZ, kCoFHZ, kNCo };

struct RzLayout {
  int nr, nz, orr;
  long long pr;     // columns per row
  long long rows;   // nz + 3
  __host__ __device__ __forceinline__ long long col(int i) const { return i + orr; }
  // mask element of entry (i, k)
  __host__ __device__ __forceinline__ long long midx(int i, int k) const {
    return (long long)(k + 1) * pr + i + orr;
  }
  // field element of (mode, comp, i, k)
  __host__ __device__ __forceinline__ long long fidx(int mode, int comp, int i, int k) const {
    return (((long long)mode * rows + k + 1) * pr + i + orr) * 6 + comp;
  }
  __host__ __device__ __forceinline__ long long mode_elems() const { return rows * pr * 6; }
};

RzLayout make_rz_layout(int nr, int nz) {
  RzLayout L;
  L.nr = nr;
  L.nz = nz;
  // a window starts at i = 60 t - 2 (56 t - 4 for two steps per pass); with
  // the axis at column 6 it starts on
  // an even column (16-byte aligned pairs, a 16-byte aligned window of
  // entries) and a 4-byte boundary of the mask; the pitch is a multiple of 16
  // and leaves room for the 80 mask bytes copied for the last window
  L.orr = 6;
  const long long tiles = (nr + 1 + kTile - 1) / kTile;
  const long long tiles2 = (nr + 1 + kTile2 - 1) / kTile2;
  L.pr = (std::max({(long long)L.orr + nr + 3, (long long)kTile * tiles + 24,
                    (long long)kTile2 * tiles2 + 24}) + 15) / 16 * 16;
  L.rows = nz + 3;
  return L;
}

template <typename T>
struct RzArgs {
  const T* in;
  T* out;
  RzLayout L;
  const uint8_t* mask;
  const T* coef;          // one material: [mode][kNCo][pr]; material arrays: [mode][rows][kNCo][pr]
  long long co_mode;      // elements per mode of coef
  long long co_plane;     // elements per plane row of coef (0: the same coefficients on every plane)
  int m_lo, n_modes;
  int tiles, chunk_z;
  int tile_w, halo;       // owned entries per window and halo entries per side (60/2 or 56/4)
  const int* work;        // active (chunk * tiles + tile)
  int n_work;
  int b_on, i0, c0, m_min, nw;
  long long n;            // step being taken (n -> n+1)
  long long kshift;       // static start: the bunch head is at plane n + kshift
  const T* J;             // [mode][2 c0]: share * c * Q_cell / dz
  double* W;              // [mode][nw]
  double inv_q;
  int* err;               // set to 1 when a bounded wait gives up
  // transverse wake at r_{obs+1/2}: WT[mode][w] += tw_er e_r^n + tw_hp h_phi^{n+1/2}
  int obs;
  double tw_er, tw_hp;
  double* WT;
  // scattered-field form: the stored field is the total minus the incident
  // TEM field; S [n mod kSourceSlots][mode][sc_len][pr * 6] is the step's
  // source on planes n + sc_off .. n + sc_off + sc_len - 1 (null otherwise;
  // in the scattered form J holds zeros)
  const T* S;
  long long sc_off;
  int sc_len;
  // work items [sc_lo, sc_hi) meet a source window: the kernels instantiated
  // with SC take exactly those, the plain ones skip them
  int sc_lo, sc_hi;
};

template <typename T>
__device__ __forceinline__ T shfl_dn(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }
template <typename T>
__device__ __forceinline__ T shfl_up(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }

// One lane's two entries of one plane: f[6 * e + comp], activity bytes m
// (low byte: the first entry).
template <typename T>
struct Pair6 {
  T f[12];
  unsigned m;
};

// Loads through the non-coherent path, issued where they are written so the
// scheduler cannot sink them towards their first use.
__device__ __forceinline__ void ld_pair(const float* p, Pair6<float>& d) {
  asm volatile("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(d.f[0]), "=f"(d.f[1]), "=f"(d.f[2]), "=f"(d.f[3]) : "l"(p) : "memory");
  asm volatile("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(d.f[4]), "=f"(d.f[5]), "=f"(d.f[6]), "=f"(d.f[7]) : "l"(p + 4) : "memory");
  asm volatile("ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(d.f[8]), "=f"(d.f[9]), "=f"(d.f[10]), "=f"(d.f[11]) : "l"(p + 8) : "memory");
}
__device__ __forceinline__ void ld_pair(const double* p, Pair6<double>& d) {
#pragma unroll
  for (int q = 0; q < 6; ++q)
    asm volatile("ld.global.nc.v2.f64 {%0,%1}, [%2];"
                 : "=d"(d.f[2 * q]), "=d"(d.f[2 * q + 1]) : "l"(p + 2 * q) : "memory");
}
__device__ __forceinline__ unsigned ld_mask2(const uint8_t* p) {
  unsigned short v;
  asm volatile("ld.global.nc.u16 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_pair(float* p, const float* v) {
  reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
  reinterpret_cast<float4*>(p)[2] = make_float4(v[8], v[9], v[10], v[11]);
}
__device__ __forceinline__ void st_pair(double* p, const double* v) {
#pragma unroll
  for (int q = 0; q < 6; ++q) reinterpret_cast<double2*>(p)[q] = make_double2(v[2 * q], v[2 * q + 1]);
}

// Per-lane constants of a work item.
template <typename T>
struct LaneCo {
  T er[2], ep[2], ez[2], hr[2], hp[2], hz[2], fez[2], fhz[2];
};

// Per-lane state carried from plane to plane: old e_r, e_phi of the current
// plane, new h_r, h_phi of the previous plane.
template <typename T>
struct LaneState {
  T er0[2], ep0[2], hr_p[2], hp_p[2];
};

// Both stages of plane k for the lane's two entries (ten updates of (24)).
// d0: plane k, d1: plane k+1 (only its e_r, e_phi are used). out receives the
// new values in the interleaved order, er_old the e_r of plane k before the
// step. j0/j1: bunch current to subtract at the two e_z entries (zero
// elsewhere).
template <typename T>
__device__ __forceinline__ void rz_plane(const Pair6<T>& d0, const Pair6<T>& d1, const LaneCo<T>& c,
                                         T mm, LaneState<T>& s, T j0, T j1, T* out, T* er_old) {
  const unsigned m = d0.m;
  er_old[0] = s.er0[0];
  er_old[1] = s.er0[1];
  T CER[2], CEP[2], CHR[2], CHP[2], FEZ[2], FHZ[2];
  if (__all_sync(0xffffffffu, m == 0x3F3Fu)) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      CER[e] = c.er[e]; CEP[e] = c.ep[e]; CHR[e] = c.hr[e]; CHP[e] = c.hp[e];
      FEZ[e] = c.fez[e]; FHZ[e] = c.fhz[e];
    }
  } else {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const unsigned b = (m >> (8 * e)) & 0xFFu;
      CER[e] = (b & 1) ? c.er[e] : T(0);
      CEP[e] = (b & 2) ? c.ep[e] : T(0);
      CHR[e] = (b & 8) ? c.hr[e] : T(0);
      CHP[e] = (b & 16) ? c.hp[e] : T(0);
      FEZ[e] = (b & 4) ? ((b & 8) ? c.fez[e] : c.ez[e]) : T(0);
      FHZ[e] = (b & 32) ? ((b & 1) ? c.fhz[e] : c.hz[e]) : T(0);
    }
  }
  T ez[2], hr[2], hp[2], hz[2], der[2], dep[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    ez[e] = d0.f[6 * e + kEZ];
    hr[e] = d0.f[6 * e + kHR];
    hp[e] = d0.f[6 * e + kHP];
    hz[e] = d0.f[6 * e + kHZ];
    der[e] = d1.f[6 * e + kER] - s.er0[e];
    dep[e] = d1.f[6 * e + kEP] - s.ep0[e];
  }
  // TM stage
  const T ezR[2] = {ez[1], shfl_dn(ez[0])};
  T hpa[2], hra[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    hpa[e] = hp[e] + CHP[e] * (der[e] - (ezR[e] - ez[e]));
    hra[e] = hr[e] + CHR[e] * (-dep[e] + mm * ez[e]);
  }
  const T hpaL[2] = {shfl_up(hpa[1]), hpa[0]};
  T ezn[2];
  const T jj[2] = {j0, j1};
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const T cur = ((hpaL[e] - hpa[e]) - mm * hra[e]) - jj[e];
    ezn[e] = ez[e] + FEZ[e] * cur;
  }
  const T eznR[2] = {ezn[1], shfl_dn(ezn[0])};
  T hpn[2], hrn[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    hpn[e] = hpa[e] + CHP[e] * (der[e] - (eznR[e] - ezn[e]));
    hrn[e] = hra[e] + CHR[e] * (-dep[e] + mm * ezn[e]);
  }
  // TE stage
  T dhr[2], dhp[2], epa[2], era[2];
  const T hzL[2] = {shfl_up(hz[1]), hz[0]};
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    dhr[e] = s.hr_p[e] - hrn[e];
    dhp[e] = s.hp_p[e] - hpn[e];
    epa[e] = s.ep0[e] + CEP[e] * (dhr[e] - (hzL[e] - hz[e]));
    era[e] = s.er0[e] + CER[e] * (-dhp[e] + mm * hz[e]);
  }
  const T epaR[2] = {epa[1], shfl_dn(epa[0])};
  T hzn[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) hzn[e] = hz[e] + FHZ[e] * ((epaR[e] - epa[e]) - mm * era[e]);
  const T hznL[2] = {shfl_up(hzn[1]), hzn[0]};
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const T epn = epa[e] + CEP[e] * (dhr[e] - (hznL[e] - hzn[e]));
    const T ern = era[e] + CER[e] * (-dhp[e] + mm * hzn[e]);
    out[6 * e + kER] = ern;
    out[6 * e + kEP] = epn;
    out[6 * e + kEZ] = ezn[e];
    out[6 * e + kHR] = hrn[e];
    out[6 * e + kHP] = hpn[e];
    out[6 * e + kHZ] = hzn[e];
    s.er0[e] = d1.f[6 * e + kER];
    s.ep0[e] = d1.f[6 * e + kEP];
    s.hr_p[e] = hrn[e];
    s.hp_p[e] = hpn[e];
  }
}

// Work-item geometry shared by both variants.
template <typename T>
struct Item {
  int mode, tile, k0, k1, gi;  // gi: radial index of the lane's first entry
  bool own;                    // lanes 1..30 store their two entries
  bool src0, src1;             // the bunch ring is one of the lane's entries
  long long fbase;             // field element of (mode, comp 0, gi, k = -1)
  long long mbase;             // mask element of (gi, k = -1)
};

template <typename T>
__device__ __forceinline__ Item<T> item_of(const RzArgs<T>& a, int witem, int sub = -1) {
  Item<T> it;
  const int lane = threadIdx.x & 31;
  it.mode = witem % a.n_modes;
  const int rest = a.work[witem / a.n_modes];
  it.tile = rest % a.tiles;
  const int chunk = rest / a.tiles;
  it.k0 = chunk * a.chunk_z;
  it.k1 = min(it.k0 + a.chunk_z, a.L.nz);
  if (sub >= 0) {  // planes sub * kSubPlanes .. of the chunk only
    it.k0 += sub * kSubPlanes;
    it.k1 = min(it.k0 + kSubPlanes, it.k1);
  }
  it.gi = it.tile * a.tile_w - a.halo + 2 * lane;
  it.own = 2 * lane >= a.halo && 2 * lane < 64 - a.halo;
  it.src0 = a.b_on && it.gi == a.i0;
  it.src1 = a.b_on && it.gi + 1 == a.i0;
  it.fbase = a.L.fidx(it.mode, 0, it.gi, -1);
  it.mbase = a.L.midx(it.gi, -1);
  return it;
}

// the lane's coefficients of plane k (k = -1 for a solve of one material,
// whose coefficients do not depend on the plane)
template <typename T>
__device__ __forceinline__ LaneCo<T> lane_coefs(const RzArgs<T>& a, const Item<T>& it, int k = -1) {
  LaneCo<T> c;
  const long long PR = a.L.pr;
  const T* co = a.coef + (long long)it.mode * a.co_mode + (long long)(k + 1) * a.co_plane + a.L.col(it.gi);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    c.er[e] = co[kCoER * PR + e];
    c.ep[e] = co[kCoEP * PR + e];
    c.ez[e] = co[kCoEZ * PR + e];
    c.hr[e] = co[kCoHR * PR + e];
    c.hp[e] = co[kCoHP * PR + e];
    c.hz[e] = co[kCoHZ * PR + e];
    c.fez[e] = co[kCoFEZ * PR + e];
    c.fhz[e] = co[kCoFHZ * PR + e];
  }
  return c;
}

// Bunch current at the lane's e_z entry of plane k (zero off the ring) and
// the wake sample of the new e_z.
template <typename T>
__device__ __forceinline__ T current_at(const RzArgs<T>& a, const Item<T>& it, bool src, int k) {
  if (!src || k < 0) return T(0);
  const long long dd = (long long)k - (a.n + a.kshift) + a.c0;
  return (dd >= -a.c0 && dd < a.c0) ? a.J[(long long)it.mode * 2 * a.c0 + dd + a.c0] : T(0);
}
// Scattered-field form: add the step's source to the new values of plane k
// (all lanes; the window of planes is warp-uniform).
template <typename T>
__device__ __forceinline__ void add_source(const RzArgs<T>& a, const Item<T>& it, int k, T* out) {
  if (!a.S) return;
  const long long w = (long long)k - (a.n + a.sc_off);
  if (w < 0 || w >= a.sc_len) return;
  const T* p =
      a.S + ((((a.n & (kSourceSlots - 1)) * a.n_modes + it.mode) * a.sc_len + w) * a.L.pr + a.L.col(it.gi)) * 6;
#pragma unroll
  for (int q = 0; q < 12; ++q) out[q] += p[q];
}

// Wake samples of plane k (Sec. 5): the path s = m dz meets e_z(k+1/2) and
// h_phi(k+1/2) at time n+1/2 and e_r(k) at time n, n = k + m + c0. The
// longitudinal wake takes e_z at the bunch ring; the radial transverse wake
// (E_r - c mu0 H_phi) at r_{obs+1/2}, where per radian h_phi = -r H_phi.
// W and WT are [parity of n][mode][nw]; a wake is the sum of its two halves.
template <typename T>
__device__ __forceinline__ void gather_wake(const RzArgs<T>& a, const Item<T>& it, int k,
                                            const T* out, const T* er_old) {
  if (!it.own || !a.b_on) return;
  const long long w = (a.n + a.kshift) - k - a.c0 - a.m_min;
  if (w < 0 || w >= a.nw) return;
  // even and odd steps accumulate into separate halves: a pass that takes
  // two steps writes step n and step n+1 samples from different work items
  const long long par = (a.n & 1) * (long long)a.n_modes * a.nw;
  const bool s[2] = {it.src0, it.src1};
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    if (s[e]) a.W[par + (long long)it.mode * a.nw + w] -= (double)out[6 * e + kEZ] * a.inv_q;
    if (it.gi + e == a.obs)
      a.WT[par + (long long)it.mode * a.nw + w] += a.tw_er * (double)er_old[e] + a.tw_hp * (double)out[6 * e + kHP];
  }
}

// --- register-ring variant ---------------------------------------------------
// MAT: per-entry material coefficients, read with each plane
template <typename T, bool SC, bool MAT>
__device__ __forceinline__ void rz_item_reg(const RzArgs<T>& a, int witem, int sub) {
  const Item<T> it = item_of(a, witem, sub);
  LaneCo<T> c = lane_coefs(a, it);
  const T mm = T(a.m_lo + it.mode);
  const long long RS = a.L.pr * 6;  // field elements per row
  const long long MS = a.L.pr;      // mask elements per row
  const T* __restrict__ ip = a.in + it.fbase;
  T* __restrict__ op = a.out + it.fbase;
  const uint8_t* __restrict__ mp = a.mask + it.mbase;
  const int kstart = it.k0 - 1;
  auto load = [&](int k, Pair6<T>& d) {
    const int row = min(k, a.L.nz + 1) + 1;
    ld_pair(ip + row * RS, d);
    d.m = ld_mask2(mp + row * MS);
  };
  // ring[u] holds plane k (u = (k - kstart) mod R); a step uses planes k and
  // k+1 and then refills the slot of plane k with plane k + R
  constexpr int R = ring_depth<T>();
  LaneState<T> s;
  Pair6<T> ring[R];
#pragma unroll
  for (int u = 0; u < R; ++u) load(kstart + u, ring[u]);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    s.er0[e] = ring[0].f[6 * e + kER];
    s.ep0[e] = ring[0].f[6 * e + kEP];
    s.hr_p[e] = T(0);
    s.hp_p[e] = T(0);
  }
  for (int kb = kstart; kb < it.k1; kb += R) {
#pragma unroll
    for (int u = 0; u < R; ++u) {
      const int k = kb + u;
      if (k >= it.k1) break;
      T out[12], er_old[2];
      if constexpr (MAT) c = lane_coefs(a, it, k);
      rz_plane(ring[u], ring[(u + 1) % R], c, mm, s, current_at(a, it, it.src0, k),
               current_at(a, it, it.src1, k), out, er_old);
      if (SC) add_source(a, it, k, out);
      if (it.own && k >= it.k0) {
        st_pair(op + (long long)(k + 1) * RS, out);
        gather_wake(a, it, k, out, er_old);
      }
      load(k + R, ring[u]);
    }
  }
}

// SC: the instantiation for the work items [sc_lo, sc_hi) that meet a source
// window of the scattered-field form; the plain one takes all others.
template <typename T, bool SC, bool MAT = false>
__global__ void __launch_bounds__(128, reg_min_blocks<T>()) rz_step_kernel(const RzArgs<T> a) {
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  const int nsub = SC ? (a.chunk_z + kSubPlanes - 1) / kSubPlanes : 1;
  const int hi = SC ? (a.sc_hi - a.sc_lo) * nsub : a.n_work * a.n_modes;
  for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); w < hi; w += nwarps) {
    // plain: every item outside [sc_lo, sc_hi); SC: the items inside, split
    // into runs of kSubPlanes planes (more warps, shorter marches)
    if (!SC && w >= a.sc_lo && w < a.sc_hi) continue;
    const int it_w = SC ? a.sc_lo + w / nsub : w;
    const int sub = SC ? w % nsub : -1;
    if (SC) {
      const int chunk = a.work[it_w / a.n_modes] / a.tiles;
      if (chunk * a.chunk_z + sub * kSubPlanes >= a.L.nz) continue;
    }
    rz_item_reg<T, SC, MAT>(a, it_w, sub);
  }
}

// --- asynchronous-copy variant ------------------------------------------------
// Per warp: a ring of async_depth planes, [slot][lane][12] field words and
// [slot][64] activity bytes, filled with 16-byte cp.async (each lane copies
// and reads back only its own 48 / 96 bytes; lanes 0..15 copy the 64
// activity bytes four at a time, hence the __syncwarp before they are read).
__device__ __forceinline__ void cp_async_16(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_4(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename T>
constexpr size_t rz_async_warp_bytes() {
  return (size_t)async_depth<T>() * 32 * 12 * sizeof(T) + (size_t)async_depth<T>() * 64;
}

template <typename T, bool SC>
__device__ __forceinline__ void rz_item_async(const RzArgs<T>& a, int witem, int sub, unsigned char* wsm) {
  const int lane = threadIdx.x & 31;
  const Item<T> it = item_of(a, witem, sub);
  const LaneCo<T> c = lane_coefs(a, it);
  const T mm = T(a.m_lo + it.mode);
  const long long RS = a.L.pr * 6;
  const long long MS = a.L.pr;
  const T* __restrict__ ip = a.in + it.fbase;
  T* __restrict__ op = a.out + it.fbase;
  // the window's activity bytes: lanes 0..15 copy bytes 4 l .. 4 l + 3
  const uint8_t* __restrict__ mwin = a.mask + a.L.midx(it.tile * a.tile_w - a.halo, -1) + 4 * (lane & 15);
  constexpr int kADepth = async_depth<T>();
  T* ring = reinterpret_cast<T*>(wsm) + lane * 12;
  uint8_t* mring = wsm + (size_t)kADepth * 32 * 12 * sizeof(T);
  const int kstart = it.k0 - 1;
  constexpr int kChunks = 12 * (int)sizeof(T) / 16;  // 16-byte copies per lane and plane

  auto issue = [&](int p) {
    if (p <= it.k1) {
      const int slot = (p - kstart) & (kADepth - 1);
      const T* g = ip + (long long)(p + 1) * RS;
      T* sl = ring + slot * 32 * 12;
#pragma unroll
      for (int q = 0; q < kChunks; ++q) cp_async_16(sl + q * (16 / sizeof(T)), g + q * (16 / sizeof(T)));
      if (lane < 16) cp_async_4(mring + slot * 64 + 4 * lane, mwin + (long long)(p + 1) * MS);
    }
    cp_async_commit();
  };
  auto fetch = [&](int p, Pair6<T>& d) {
    const int slot = (p - kstart) & (kADepth - 1);
    const T* sl = ring + slot * 32 * 12;
#pragma unroll
    for (int q = 0; q < 12; ++q) d.f[q] = sl[q];
    d.m = *reinterpret_cast<const unsigned short*>(mring + slot * 64 + 2 * lane);
  };

  __syncwarp();
#pragma unroll
  for (int p = 0; p < kADepth - 1; ++p) issue(kstart + p);
  LaneState<T> s;
  Pair6<T> d0, d1;
  cp_async_wait<kADepth - 2>();
  __syncwarp();
  fetch(kstart, d0);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    s.er0[e] = d0.f[6 * e + kER];
    s.ep0[e] = d0.f[6 * e + kEP];
    s.hr_p[e] = T(0);
    s.hp_p[e] = T(0);
  }
  for (int k = kstart; k < it.k1; ++k) {
    __syncwarp();
    issue(k + kADepth - 1);
    cp_async_wait<kADepth - 2>();
    __syncwarp();
    fetch(k + 1, d1);
    T out[12], er_old[2];
    rz_plane(d0, d1, c, mm, s, current_at(a, it, it.src0, k), current_at(a, it, it.src1, k), out,
             er_old);
    if (SC) add_source(a, it, k, out);
    if (it.own && k >= it.k0) {
      st_pair(op + (long long)(k + 1) * RS, out);
      gather_wake(a, it, k, out, er_old);
    }
    d0 = d1;
  }
  cp_async_wait<0>();
  __syncwarp();
}

template <typename T, bool SC>
__global__ void __launch_bounds__(128) rz_step_async_kernel(const RzArgs<T> a) {
  extern __shared__ __align__(16) unsigned char rz_smem[];
  unsigned char* wsm = rz_smem + (size_t)(threadIdx.x >> 5) * rz_async_warp_bytes<T>();
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  const int nsub = SC ? (a.chunk_z + kSubPlanes - 1) / kSubPlanes : 1;
  const int hi = SC ? (a.sc_hi - a.sc_lo) * nsub : a.n_work * a.n_modes;
  for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); w < hi; w += nwarps) {
    // plain: every item outside [sc_lo, sc_hi); SC: the items inside, split
    // into runs of kSubPlanes planes (more warps, shorter marches)
    if (!SC && w >= a.sc_lo && w < a.sc_hi) continue;
    const int it_w = SC ? a.sc_lo + w / nsub : w;
    const int sub = SC ? w % nsub : -1;
    if (SC) {
      const int chunk = a.work[it_w / a.n_modes] / a.tiles;
      if (chunk * a.chunk_z + sub * kSubPlanes >= a.L.nz) continue;
    }
    rz_item_async<T, SC>(a, it_w, sub, wsm);
  }
}

// --- bulk-copy variant -------------------------------------------------------
// A warp's window of one plane is one contiguous block of 64 entries x 6
// components (1536 bytes in float32, 3072 in float64), so one bulk copy
// (cp.async.bulk, the TMA engine) per plane fills a ring slot, and a second
// one brings the 80-byte aligned block that holds the window's 64 activity
// bytes. Lane 0 issues both with an mbarrier expecting their byte count;
// every lane waits on the slot's mbarrier phase (bounded: after kMaxPolls
// polls the kernel raises the error word and stops) and reads its own 48 /
// 96 bytes. The ring runs bulk_depth planes ahead without registers.
constexpr int kMaxPolls = TETM_RZ_MAX_POLLS;
constexpr int kMaskBlock = 80;

template <typename T>
__host__ __device__ constexpr int bulk_depth() { return sizeof(T) == 4 ? 8 : 4; }
template <typename T>
__host__ __device__ constexpr int window_bytes() { return 64 * 6 * (int)sizeof(T); }
template <typename T>
constexpr size_t rz_bulk_warp_bytes() {
  return (size_t)bulk_depth<T>() * (window_bytes<T>() + kMaskBlock) + (size_t)bulk_depth<T>() * 8;
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Returns false when the wait gave up.
__device__ __forceinline__ bool mbar_wait_n(uint64_t* bar, unsigned parity, int polls) {
  for (int it = 0; it < polls; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  return mbar_wait_n(bar, parity, kMaxPolls);
}

// Bounded-wait self-test: one warp waits with the step kernels' poll loop on
// an mbarrier that nothing arrives at (a copy that never lands), gives up
// after `polls` polls and raises the error word, as a step kernel would.
__global__ void rz_selftest_wait_kernel(int polls, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncwarp();
  const bool ok = mbar_wait_n(&bar, 0, polls);
  if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) atomicExch(err, 1);
}

template <typename T, bool SC>
__device__ __forceinline__ bool rz_item_bulk(const RzArgs<T>& a, int witem, int sub, unsigned char* wsm,
                                             unsigned& phases) {
  constexpr int D = bulk_depth<T>();
  constexpr int WB = window_bytes<T>();
  const int lane = threadIdx.x & 31;
  const Item<T> it = item_of(a, witem, sub);
  const LaneCo<T> c = lane_coefs(a, it);
  const T mm = T(a.m_lo + it.mode);
  const long long RS = a.L.pr * 6;
  const long long MS = a.L.pr;
  T* __restrict__ op = a.out + it.fbase;
  const int wcol = it.tile * a.tile_w - a.halo + a.L.orr;  // window's first column
  const T* __restrict__ wsrc = a.in + a.L.fidx(it.mode, 0, it.tile * a.tile_w - a.halo, -1);
  const int mcol = wcol & ~15;                              // 16-byte aligned mask block
  const uint8_t* __restrict__ msrc = a.mask + mcol;
  unsigned char* fring = wsm;
  unsigned char* mring = wsm + (size_t)D * WB;
  uint64_t* bars = reinterpret_cast<uint64_t*>(wsm + (size_t)D * (WB + kMaskBlock));
  const int kstart = it.k0 - 1;
  const int moff = wcol - mcol + 2 * lane;                  // lane's activity bytes in a block
  int issued = kstart - 1;                                  // last plane whose copies are queued
  int fetched = kstart - 1;                                 // last plane read

  auto issue = [&](int p) {
    if (p > it.k1) return;
    const int slot = (p - kstart) % D;
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(bars + slot, WB + kMaskBlock);
      bulk_g2s(fring + (size_t)slot * WB, wsrc + (long long)(p + 1) * RS, WB, bars + slot);
      bulk_g2s(mring + (size_t)slot * kMaskBlock, msrc + (long long)(p + 1) * MS, kMaskBlock, bars + slot);
    }
    issued = p;
  };
  bool ok = true;
  auto fetch = [&](int p, Pair6<T>& d) {
    const int slot = (p - kstart) % D;
    if (ok) ok = mbar_wait(bars + slot, (phases >> slot) & 1u);
    if (ok) {
      phases ^= 1u << slot;
      fetched = p;
    }
    const T* src = reinterpret_cast<const T*>(fring + (size_t)slot * WB) + 12 * lane;
#pragma unroll
    for (int q = 0; q < 12; ++q) d.f[q] = src[q];
    d.m = *reinterpret_cast<const unsigned short*>(mring + (size_t)slot * kMaskBlock + moff);
  };

  __syncwarp();
  for (int p = 0; p < D - 1; ++p) issue(kstart + p);
  LaneState<T> s;
  Pair6<T> d0, d1;
  fetch(kstart, d0);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    s.er0[e] = d0.f[6 * e + kER];
    s.ep0[e] = d0.f[6 * e + kEP];
    s.hr_p[e] = T(0);
    s.hp_p[e] = T(0);
  }
  for (int k = kstart; k < it.k1 && __all_sync(0xffffffffu, ok); ++k) {
    __syncwarp();  // every lane is done with the slot refilled next
    issue(k + D - 1);
    fetch(k + 1, d1);
    if (!__all_sync(0xffffffffu, ok)) break;
    T out[12], er_old[2];
    rz_plane(d0, d1, c, mm, s, current_at(a, it, it.src0, k), current_at(a, it, it.src1, k), out,
             er_old);
    if (SC) add_source(a, it, k, out);
    if (it.own && k >= it.k0) {
      st_pair(op + (long long)(k + 1) * RS, out);
      gather_wake(a, it, k, out, er_old);
    }
    d0 = d1;
  }
  if (__all_sync(0xffffffffu, ok)) return true;
  // a wait gave up: raise the error word and drain the copies still queued
  // (each wait bounded again) before the ring's memory is left
  if (lane == 0) atomicExch(a.err, 1);
  for (int p = fetched + 1; p <= issued; ++p) {
    const int slot = (p - kstart) % D;
    mbar_wait(bars + slot, (phases >> slot) & 1u);
    phases ^= 1u << slot;
  }
  return false;
}

template <typename T, bool SC>
__global__ void __launch_bounds__(128) rz_step_bulk_kernel(const RzArgs<T> a) {
  extern __shared__ __align__(128) unsigned char rz_bulk_smem[];
  constexpr int D = bulk_depth<T>();
  unsigned char* wsm = rz_bulk_smem + (size_t)(threadIdx.x >> 5) * rz_bulk_warp_bytes<T>();
  uint64_t* bars = reinterpret_cast<uint64_t*>(wsm + (size_t)D * (window_bytes<T>() + kMaskBlock));
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < D; ++q) mbar_init(bars + q, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncwarp();
  unsigned phases = 0;
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  const int nsub = SC ? (a.chunk_z + kSubPlanes - 1) / kSubPlanes : 1;
  const int hi = SC ? (a.sc_hi - a.sc_lo) * nsub : a.n_work * a.n_modes;
  for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); w < hi; w += nwarps) {
    // plain: every item outside [sc_lo, sc_hi); SC: the items inside, split
    // into runs of kSubPlanes planes (more warps, shorter marches)
    if (!SC && w >= a.sc_lo && w < a.sc_hi) continue;
    const int it_w = SC ? a.sc_lo + w / nsub : w;
    const int sub = SC ? w % nsub : -1;
    if (SC) {
      const int chunk = a.work[it_w / a.n_modes] / a.tiles;
      if (chunk * a.chunk_z + sub * kSubPlanes >= a.L.nz) continue;
    }
    if (!rz_item_bulk<T, SC>(a, it_w, sub, wsm, phases)) return;
  }
}

// --- two steps per pass (temporal blocking) -----------------------------------
// The bulk-copy sweep with a second time step riding one plane behind the
// first: at plane k the warp takes y^n -> y^{n+1} (step 1) as above, then
// y^{n+1} -> y^{n+2} at plane k-1 (step 2) from the step-1 values of planes
// k-1 and k it holds in registers, and stores only y^{n+2}. Each plane of y^n
// is read once and each plane of y^{n+2} written once for two steps. Step 1
// is valid on the window entries 2..61, so step 2 owns 4..59 (56-entry tiles,
// 4 halo entries each side). Step 1 recomputes two planes before the chunk and
// one after; step 2 recomputes one before. Both steps deposit their current;
// each gathers its wake samples on the item's own planes.
template <typename T, bool SC>
__device__ __forceinline__ bool rz_item_bulk2(const RzArgs<T>& a, int witem, int sub, unsigned char* wsm,
                                              unsigned& phases) {
  constexpr int D = bulk_depth<T>();
  constexpr int WB = window_bytes<T>();
  const int lane = threadIdx.x & 31;
  const Item<T> it = item_of(a, witem, sub);
  const LaneCo<T> c = lane_coefs(a, it);
  const T mm = T(a.m_lo + it.mode);
  const long long RS = a.L.pr * 6;
  const long long MS = a.L.pr;
  T* __restrict__ op = a.out + it.fbase;
  const int wcol = it.tile * a.tile_w - a.halo + a.L.orr;
  const T* __restrict__ wsrc = a.in + a.L.fidx(it.mode, 0, it.tile * a.tile_w - a.halo, -1);
  const int mcol = wcol & ~15;
  const uint8_t* __restrict__ msrc = a.mask + mcol;
  unsigned char* fring = wsm;
  unsigned char* mring = wsm + (size_t)D * WB;
  uint64_t* bars = reinterpret_cast<uint64_t*>(wsm + (size_t)D * (WB + kMaskBlock));
  const int kfirst = max(it.k0 - 2, -1);    // first plane of step 1 (plane -1 is all guard)
  const int klast = it.k1;                  // last plane of step 1
  const int moff = wcol - mcol + 2 * lane;
  int issued = kfirst - 1, fetched = kfirst - 1;
  // a second item view for step 2: same geometry, one step later
  RzArgs<T> a2 = a;
  a2.n = a.n + 1;

  auto issue = [&](int p) {
    if (p > klast + 1) return;
    const int slot = (p - kfirst) % D;
    if (lane == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(bars + slot, WB + kMaskBlock);
      bulk_g2s(fring + (size_t)slot * WB, wsrc + (long long)(p + 1) * RS, WB, bars + slot);
      bulk_g2s(mring + (size_t)slot * kMaskBlock, msrc + (long long)(p + 1) * MS, kMaskBlock, bars + slot);
    }
    issued = p;
  };
  bool ok = true;
  auto fetch = [&](int p, Pair6<T>& d) {
    const int slot = (p - kfirst) % D;
    if (ok) ok = mbar_wait(bars + slot, (phases >> slot) & 1u);
    if (ok) {
      phases ^= 1u << slot;
      fetched = p;
    }
    const T* src = reinterpret_cast<const T*>(fring + (size_t)slot * WB) + 12 * lane;
#pragma unroll
    for (int q = 0; q < 12; ++q) d.f[q] = src[q];
    d.m = *reinterpret_cast<const unsigned short*>(mring + (size_t)slot * kMaskBlock + moff);
  };

  __syncwarp();
  for (int p = 0; p < D - 1; ++p) issue(kfirst + p);
  LaneState<T> s1, s2;
  Pair6<T> d0, d1, y1prev;     // y^n of planes k, k+1; y^{n+1} of plane k-1
  fetch(kfirst, d0);
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    s1.er0[e] = d0.f[6 * e + kER];
    s1.ep0[e] = d0.f[6 * e + kEP];
    s1.hr_p[e] = T(0);
    s1.hp_p[e] = T(0);
    s2.hr_p[e] = T(0);
    s2.hp_p[e] = T(0);
    s2.er0[e] = T(0);
    s2.ep0[e] = T(0);
  }
  for (int k = kfirst; k <= klast && __all_sync(0xffffffffu, ok); ++k) {
    __syncwarp();
    issue(k + D - 1);
    fetch(k + 1, d1);
    if (!__all_sync(0xffffffffu, ok)) break;
    // step 1 at plane k
    Pair6<T> y1;
    T er_old[2];
    rz_plane(d0, d1, c, mm, s1, current_at(a, it, it.src0, k), current_at(a, it, it.src1, k), y1.f,
             er_old);
    if (SC) add_source(a, it, k, y1.f);
    y1.m = d0.m;
    if (k >= it.k0 && k < it.k1) gather_wake(a, it, k, y1.f, er_old);
    // step 2 at plane k - 1 (from step-1 planes k-1 and k)
    const int k2 = k - 1;
    if (k2 == it.k0 - 1) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        s2.er0[e] = y1prev.f[6 * e + kER];
        s2.ep0[e] = y1prev.f[6 * e + kEP];
      }
    }
    if (k2 >= it.k0 - 1) {
      T y2[12], er_old2[2];
      rz_plane(y1prev, y1, c, mm, s2, current_at(a2, it, it.src0, k2), current_at(a2, it, it.src1, k2),
               y2, er_old2);
      if (SC) add_source(a2, it, k2, y2);
      if (it.own && k2 >= it.k0) {
        st_pair(op + (long long)(k2 + 1) * RS, y2);
        gather_wake(a2, it, k2, y2, er_old2);
      }
    }
    y1prev = y1;
    d0 = d1;
  }
  if (__all_sync(0xffffffffu, ok)) return true;
  if (lane == 0) atomicExch(a.err, 1);
  for (int p = fetched + 1; p <= issued; ++p) {
    const int slot = (p - kfirst) % D;
    mbar_wait(bars + slot, (phases >> slot) & 1u);
    phases ^= 1u << slot;
  }
  return false;
}

template <typename T, bool SC>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 4 : 1) rz_step_bulk2_kernel(const RzArgs<T> a) {
  extern __shared__ __align__(128) unsigned char rz_bulk2_smem[];
  constexpr int D = bulk_depth<T>();
  unsigned char* wsm = rz_bulk2_smem + (size_t)(threadIdx.x >> 5) * rz_bulk_warp_bytes<T>();
  uint64_t* bars = reinterpret_cast<uint64_t*>(wsm + (size_t)D * (window_bytes<T>() + kMaskBlock));
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < D; ++q) mbar_init(bars + q, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncwarp();
  unsigned phases = 0;
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  const int nsub = SC ? (a.chunk_z + kSubPlanes - 1) / kSubPlanes : 1;
  const int hi = SC ? (a.sc_hi - a.sc_lo) * nsub : a.n_work * a.n_modes;
  for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); w < hi; w += nwarps) {
    // plain: every item outside [sc_lo, sc_hi); SC: the items inside, split
    // into runs of kSubPlanes planes (more warps, shorter marches)
    if (!SC && w >= a.sc_lo && w < a.sc_hi) continue;
    const int it_w = SC ? a.sc_lo + w / nsub : w;
    const int sub = SC ? w % nsub : -1;
    if (SC) {
      const int chunk = a.work[it_w / a.n_modes] / a.tiles;
      if (chunk * a.chunk_z + sub * kSubPlanes >= a.L.nz) continue;
    }
    if (!rz_item_bulk2<T, SC>(a, it_w, sub, wsm, phases)) return;
  }
}

// Scattered-field form. The incident field is the discrete TEM field of the
// ring bunch in the entry pipe (the static start's field), continued along
// the grid and moving one plane per step: at step n it is the static-start
// field shifted by n planes, zero outside planes 0..nz-1. prof [mode][6][pr]
// holds its transverse profile (the entry section's activity, the metric
// zeros and the constant factors folded in; zero for e_z and h_z), G
// [mode][glen] its longitudinal profile: e at plane k takes G[k - n + 1], h
// takes G[k - n + 2]. prof == null: no incident field.
struct RzIncident {
  const double* prof;
  const double* G;
  int glen;
  long long n;
  RzLayout L;
};

__device__ __forceinline__ double inc_value(const RzIncident& x, int mode, int comp, int i, int k) {
  if (!x.prof || k < 0 || k >= x.L.nz || i < 0 || i > x.L.nr || comp == kEZ || comp == kHZ) return 0.0;
  const long long u = (long long)k - x.n + ((comp == kHR || comp == kHP) ? 2 : 1);
  if (u < 0 || u >= x.glen) return 0.0;
  return x.prof[((long long)mode * 6 + comp) * x.L.pr + x.L.col(i)] * x.G[(long long)mode * x.glen + u];
}

// Source of the scattered-field form for steps x.n .. x.n + n_steps - 1 on
// the window planes n + sc_off .. n + sc_off + sc_len - 1. With the stored
// field y = total - x (x^n the incident field) the step is y^{n+1} = F_0(y^n)
// + S^n (F_0: one step of (24) in the grid's geometry without current), where
// S^n = F(x^n) - x^{n+1} and F is the step with the bunch current. The
// incident field solves the step of the continued entry pipe exactly,
// x^{n+1} = F_pipe(x^n), except where the grid ends cut it off (planes 0 and
// nz-1), so on the other planes S^n is evaluated as F(x^n) - F_pipe(x^n):
// both by the step kernels' own per-plane routine, in the field precision, on
// the synthesised incident field, once with the geometry's activity and once
// with the entry section's. The two agree bit for bit wherever the activity
// within the stencil's reach agrees, so S is an exact zero there, and the
// rounding of S scales with the incident field at the wall, not with the
// bunch's near field. One warp per (step, mode, radial tile, group of ch
// planes); the plane before a group is recomputed for the new h of its
// previous plane. A group none of whose rows k0-1..k1-1 differs from the
// entry section within the tile's reach (differs[(k + 1) * s_tiles + tile])
// and that holds no grid end writes zeros.
template <typename T>
__global__ void __launch_bounds__(128) rz_source_kernel(RzArgs<T> a, RzIncident x,
                                                        const uint8_t* differs, int s_tiles, int ch,
                                                        int n_groups, int n_steps, T* S) {
  const int lane = threadIdx.x & 31;
  const int nz = a.L.nz;
  const long long nitems = (long long)n_steps * a.n_modes * s_tiles * n_groups;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < nitems; w += nwarps) {
    long long r = w;
    const int grp = (int)(r % n_groups);
    r /= n_groups;
    const int tile = (int)(r % s_tiles);
    r /= s_tiles;
    const int mode = (int)(r % a.n_modes);
    const long long n = x.n + r / a.n_modes;
    const long long w0 = n + a.sc_off;
    const long long k0l = max(w0 + (long long)grp * ch, 0LL);
    const long long k1l = min(min(w0 + (long long)(grp + 1) * ch, w0 + a.sc_len), (long long)nz);
    if (k0l >= k1l) continue;  // the same for every lane
    const int k0 = (int)k0l, k1 = (int)k1l;
    Item<T> it;
    it.mode = mode;
    it.tile = tile;
    it.k0 = k0;
    it.k1 = k1;
    it.gi = tile * kTile - 2 + 2 * lane;
    it.own = lane >= 1 && lane <= 30;
    it.src0 = it.gi == a.i0;
    it.src1 = it.gi + 1 == a.i0;
    it.fbase = 0;
    it.mbase = 0;
    auto slot = [&](int k) {
      return S + ((((n & (kSourceSlots - 1)) * a.n_modes + mode) * a.sc_len + (k - w0)) * a.L.pr +
                  a.L.col(it.gi)) * 6;
    };
    bool any = k0 == 0 || k1 == nz;
    for (int k = k0 - 1; k < k1; ++k) any = any || differs[(long long)(k + 1) * s_tiles + tile] != 0;
    if (!any) {
      if (it.own)
        for (int k = k0; k < k1; ++k) {
          T* p = slot(k);
#pragma unroll
          for (int q = 0; q < 12; ++q) p[q] = T(0);
        }
      continue;
    }
    const LaneCo<T> c = lane_coefs(a, it);
    const T mm = T(a.m_lo + mode);
    RzArgs<T> an = a;
    an.n = n;
    RzIncident xi = x, xo = x;
    xi.n = n;
    xo.n = n + 1;
    // the entry section's activity bytes of the lane's two entries
    const unsigned m_pipe =
        (unsigned)a.mask[a.L.midx(it.gi, 1)] | ((unsigned)a.mask[a.L.midx(it.gi + 1, 1)] << 8);
    auto synth = [&](int k, Pair6<T>& d) {
#pragma unroll
      for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int comp = 0; comp < 6; ++comp) d.f[6 * e + comp] = (T)inc_value(xi, mode, comp, it.gi + e, k);
      d.m = (unsigned)a.mask[a.L.midx(it.gi, k)] | ((unsigned)a.mask[a.L.midx(it.gi + 1, k)] << 8);
    };
    Pair6<T> d0, d1, p0, p1;
    LaneState<T> sg, sp;
    synth(k0 - 1, d0);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      sg.er0[e] = sp.er0[e] = d0.f[6 * e + kER];
      sg.ep0[e] = sp.ep0[e] = d0.f[6 * e + kEP];
      sg.hr_p[e] = sp.hr_p[e] = T(0);
      sg.hp_p[e] = sp.hp_p[e] = T(0);
    }
    for (int k = k0 - 1; k < k1; ++k) {
      synth(k + 1, d1);
      p0 = d0;
      p0.m = m_pipe;
      p1 = d1;
      p1.m = m_pipe;
      const T j0 = current_at(an, it, it.src0, k), j1 = current_at(an, it, it.src1, k);
      T out[12], ref[12], er_old[2];
      rz_plane(d0, d1, c, mm, sg, j0, j1, out, er_old);
      rz_plane(p0, p1, c, mm, sp, j0, j1, ref, er_old);
      if (it.own && k >= k0) {
        const bool cut = k == 0 || k == nz - 1;  // the incident field cut off by a grid end
        T* p = slot(k);
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
          for (int comp = 0; comp < 6; ++comp) {
            const T next = cut ? (T)inc_value(xo, mode, comp, it.gi + e, k) : ref[6 * e + comp];
            p[6 * e + comp] = out[6 * e + comp] - next;
          }
      }
      d0 = d1;
    }
  }
}

// Scattered-field form: per row (planes -1..nz) and source tile, whether the
// row's activity bytes differ from the entry section's (plane 1) within the
// tile's reach (its 60 entries and 4 more on each side)
__global__ void rz_row_differs(const uint8_t* mask, RzLayout L, int s_tiles, uint8_t* out) {
  const int row = blockIdx.x;
  if (row > L.nz + 1) return;
  for (int tile = 0; tile < s_tiles; ++tile) {
    const long long lo = max((long long)tile * kTile - 4 + L.orr, 0LL);
    const long long hi = min((long long)tile * kTile + kTile + 4 + L.orr, L.pr);
    int d = 0;
    for (long long col = lo + threadIdx.x; col < hi; col += blockDim.x)
      d |= mask[row * L.pr + col] != mask[2 * L.pr + col];
    d = __syncthreads_or(d);
    if (threadIdx.x == 0) out[(long long)row * s_tiles + tile] = (uint8_t)(d != 0);
  }
}

// Scattered-field form: entries of planes 1..nz-1 where the entry section
// (plane 1) has an object that the geometry lacks
__global__ void rz_row_not_covered(const uint8_t* mask, RzLayout L, unsigned long long* out) {
  const long long total = (long long)(L.nz - 1) * L.pr;
  unsigned long long c = 0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long k = 1 + q / L.pr, col = q % L.pr;
    c += (mask[2 * L.pr + col] & ~mask[(k + 1) * L.pr + col]) != 0;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// Add sign times the incident field to a canonical array of one component.
__global__ void rz_canonical_add_inc(double* dst, RzIncident x, int mode, int comp, double sign) {
  const long long n = (long long)(x.L.nr + 1) * (x.L.nz + 1);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % (x.L.nr + 1)), k = (int)(q / (x.L.nr + 1));
    dst[q] += sign * inc_value(x, mode, comp, i, k);
  }
}

// Activity bits from the cell geometry (staircase; the rules of the
// per-radian metric): bit c set <=> object c at entry (i, k) is non-PEC.
__device__ __forceinline__ bool cell_pec(const uint8_t* pec, int nr, int nz, int ci, int ck) {
  if (ci >= nr || ck < 0 || ck >= nz || ci < 0) return true;
  return pec ? pec[ci + (long long)nr * ck] != 0 : false;
}

// Entries that hold a non-zero value where the entry's activity bit is clear
// (the guard rows and columns, PEC objects): the canary of an out-of-place
// write. The six components of a column sit side by side over the mask's entry.
template <typename T>
__global__ void rz_guard_scan(const T* f, const uint8_t* mask, RzLayout L, long long total,
                              unsigned long long* out) {
  const long long per_mode = L.rows * L.pr;
  unsigned long long c = 0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x)
    if (f[q] != T(0) && !((mask[(q / 6) % per_mode] >> (int)(q % 6)) & 1)) ++c;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

__global__ void rz_build_mask(const uint8_t* pec, RzLayout L, uint8_t* mask) {
  const long long total = L.rows * L.pr;
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
__global__ void rz_item_flags(const uint8_t* mask, RzLayout L, int tiles, int tile_w, int chunk_z,
                              int n_chunks, int* flags) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= tiles * n_chunks) return;
  const int tile = q % tiles, chunk = q / tiles;
  const int i_lo = tile * tile_w, i_hi = min(i_lo + tile_w, L.nr + 1);
  const int k_lo = chunk * chunk_z, k_hi = min(k_lo + chunk_z, L.nz);
  int any = 0;
  for (int k = k_lo; k < k_hi && !any; ++k)
    for (int i = i_lo; i < i_hi; ++i)
      if (mask[L.midx(i, k)]) { any = 1; break; }
  flags[q] = any;
}

// Canonical <-> device layout for one component of one mode; inactive
// entries (mask bit clear or the mode's metric zero there) are written as
// zero.
template <typename T>
__global__ void rz_to_canonical(const T* src, RzLayout L, int mode, int comp, double* dst) {
  const long long n = (long long)(L.nr + 1) * (L.nz + 1);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % (L.nr + 1)), k = (int)(q / (L.nr + 1));
    dst[q] = (double)src[L.fidx(mode, comp, i, k)];
  }
}

// (scattered-field form: the stored value is the given total minus the
// incident field x)
// (metric: the component's row, mplane elements apart from plane to plane, 0
// for one material)
template <typename T>
__global__ void rz_from_canonical(const double* src, RzLayout L, const uint8_t* mask, int mode,
                                  int comp, const double* metric, long long mplane, T* dst, RzIncident x) {
  const long long n = (long long)(L.nr + 1) * (L.nz + 1);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % (L.nr + 1)), k = (int)(q / (L.nr + 1));
    const bool act = ((mask[L.midx(i, k)] >> comp) & 1) && metric[(long long)(k + 1) * mplane + i] != 0.0;
    dst[L.fidx(mode, comp, i, k)] = (T)((act ? src[q] : 0.0) - inc_value(x, mode, comp, i, k));
  }
}

// Discrete energy per radian, 0.5 <Q^{e,r} y, y> (Sec. 4.4): the weighted
// squares of all six components, minus alpha^2/2 times the radial part of
// the splitting operator (M_mu_phi^-1 (P_r e_z)^2 and M_eps_phi^-1
// (P_r^T h_z)^2), plus alpha times the longitudinal coupling
// h_phi P_z e_r - h_r P_z e_phi. metric: [6][pr] unscaled M^-1 of the mode
// (zero where the mode has no object), for material arrays one such block per
// plane, mplane elements apart (0 for one material). One partial per block.
constexpr int kEnergyBlocks = 512;
constexpr int kEnergyThreads = 256;
constexpr int kRzRec = 6;  // balance record: step, mode, energy, max |qe - qbunch|, max |qh|, bunch charge scale

template <typename T>
__global__ void __launch_bounds__(kEnergyThreads)
rz_energy_partial(const T* f, RzLayout L, int mode, const uint8_t* mask, const double* metric,
                  long long mplane, double alpha, double* partial, RzIncident x) {
  const long long PR = L.pr;
  const long long n = (long long)(L.nr + 1) * (L.nz + 1);
  double acc = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % (L.nr + 1)), k = (int)(q / (L.nr + 1));
    // the field of entry (i + di, k + dk), plus the incident field in the
    // scattered-field form
    auto v = [&](int comp, int di, int dk) {
      return (double)f[L.fidx(mode, comp, i + di, k + dk)] + inc_value(x, mode, comp, i + di, k + dk);
    };
    const uint8_t m = mask[L.midx(i, k)];
    double w = 0.0;
    double c[6];
    for (int comp = 0; comp < 6; ++comp) {
      c[comp] = ((m >> comp) & 1) ? metric[(long long)(k + 1) * mplane + comp * PR + i] : 0.0;
      if (c[comp] != 0.0) {
        const double val = v(comp, 0, 0);
        w += 0.5 * val * val / c[comp];
      }
    }
    const double ez = v(kEZ, 0, 0), hz = v(kHZ, 0, 0);
    const double t1 = v(kEZ, 1, 0) - ez;
    const double t2 = v(kHZ, -1, 0) - hz;
    const double r = c[kHP] * t1 * t1 + c[kEP] * t2 * t2;
    const double l = v(kHP, 0, 0) * (v(kER, 0, 1) - v(kER, 0, 0)) -
                     v(kHR, 0, 0) * (v(kEP, 0, 1) - v(kEP, 0, 0));
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

// Charges of mode m (the analogue of Eqs. (35) and (34) for scheme (24)):
// at node (i, k), qe = -P_r^T dr - m dphi - P_z^T dz~ with dr, dphi the e_r,
// e_phi fluxes averaged over the two states and dz~ = M_ez ez - alpha^2
// P_r^T M_hphi^-1 P_r ez; at the cell of lower node (i, k), qh = m bphi +
// P_r br + P_z bz~ with bz~ = M_hz hz - alpha^2 P_r M_ephi^-1 P_r^T hz of the
// previous state (the m-part of the splitting operator stays in B^{e,r}). A
// node (cell) counts when every edge (face) it touches carries a field; at
// the bunch ring the node charge is compared with the bunch's share of the
// node charge qline. fc, fp: the current and the previous state (the
// incident field added in the scattered-field form). One max per block.
template <typename T>
__global__ void __launch_bounds__(kEnergyThreads)
rz_charge_partial(const T* fc, const T* fp, RzLayout L, int mode, double mm, const uint8_t* mask,
                  const double* metric, long long mplane, double a2, RzIncident xc, RzIncident xp,
                  const double* qline, double share, int i0, double* part_e, double* part_h) {
  const long long PR = L.pr;
  const long long n = (long long)(L.nr + 1) * (L.nz + 1);
  double me = 0.0, mh = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % (L.nr + 1)), k = (int)(q / (L.nr + 1));
    auto C = [&](int comp, int ii, int kk) -> double {  // M^-1 of the entry, 0 where it has no object
      if (ii < 0 || ii > L.nr || kk < -1 || kk > L.nz + 1) return 0.0;
      return ((mask[L.midx(ii, kk)] >> comp) & 1) ? metric[(long long)(kk + 1) * mplane + comp * PR + ii] : 0.0;
    };
    auto vc = [&](int comp, int ii, int kk) {
      return (double)fc[L.fidx(mode, comp, ii, kk)] + inc_value(xc, mode, comp, ii, kk);
    };
    auto vp = [&](int comp, int ii, int kk) {
      return (double)fp[L.fidx(mode, comp, ii, kk)] + inc_value(xp, mode, comp, ii, kk);
    };
    // Eq. (35) at node (i, k)
    const double cep = C(kEP, i, k);
    if (C(kEZ, i, k) != 0.0 && C(kEZ, i, k - 1) != 0.0 && C(kER, i, k) != 0.0 &&
        (i == 0 || C(kER, i - 1, k) != 0.0) && (mm == 0.0 || cep != 0.0)) {
      auto dr = [&](int ii) {
        const double c = C(kER, ii, k);
        return c != 0.0 ? 0.5 * (vc(kER, ii, k) + vp(kER, ii, k)) / c : 0.0;
      };
      auto dzt = [&](int kk) {
        const double z = vc(kEZ, i, kk), zl = vc(kEZ, i - 1, kk), zr = vc(kEZ, i + 1, kk);
        const double r = (i > 0 ? C(kHP, i - 1, kk) * (z - zl) : 0.0) - C(kHP, i, kk) * (zr - z);
        return z / C(kEZ, i, kk) - a2 * r;
      };
      const double dp = cep != 0.0 ? 0.5 * (vc(kEP, i, k) + vp(kEP, i, k)) / cep : 0.0;
      double qe = -((i > 0 ? dr(i - 1) : 0.0) - dr(i)) - mm * dp - (dzt(k - 1) - dzt(k));
      if (qline && i == i0) qe -= share * qline[k];
      me = fmax(me, fabs(qe));
    }
    // Eq. (34) at the cell of lower node (i, k)
    const double chp = C(kHP, i, k);
    if (C(kHZ, i, k) != 0.0 && C(kHZ, i, k + 1) != 0.0 && C(kHR, i + 1, k) != 0.0 &&
        (i == 0 || C(kHR, i, k) != 0.0) && (mm == 0.0 || chp != 0.0)) {
      auto br = [&](int ii) {
        const double c = C(kHR, ii, k);
        return c != 0.0 ? 0.5 * (vc(kHR, ii, k) + vp(kHR, ii, k)) / c : 0.0;
      };
      auto bzt = [&](int kk) {
        const double z = vp(kHZ, i, kk), zl = vp(kHZ, i - 1, kk), zr = vp(kHZ, i + 1, kk);
        const double r = C(kEP, i + 1, kk) * (z - zr) - C(kEP, i, kk) * (zl - z);
        return z / C(kHZ, i, kk) - a2 * r;
      };
      const double bp = chp != 0.0 ? 0.5 * (vc(kHP, i, k) + vp(kHP, i, k)) / chp : 0.0;
      const double qh = mm * bp + (br(i + 1) - br(i)) + (bzt(k + 1) - bzt(k));
      mh = fmax(mh, fabs(qh));
    }
  }
  __shared__ double sh[2][kEnergyThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    me = fmax(me, __shfl_down_sync(0xffffffffu, me, o));
    mh = fmax(mh, __shfl_down_sync(0xffffffffu, mh, o));
  }
  if ((threadIdx.x & 31) == 0) {
    sh[0][threadIdx.x >> 5] = me;
    sh[1][threadIdx.x >> 5] = mh;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double a = threadIdx.x < kEnergyThreads / 32 ? sh[0][threadIdx.x] : 0.0;
    double b = threadIdx.x < kEnergyThreads / 32 ? sh[1][threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
      b = fmax(b, __shfl_down_sync(0xffffffffu, b, o));
    }
    if (threadIdx.x == 0) {
      part_e[blockIdx.x] = a;
      part_h[blockIdx.x] = b;
    }
  }
}

// the maxima of the charge partials and the record's step, mode and charge
// scale: rec = {n, m, W (written before), max_e, max_h, share * qmax}
__global__ void rz_balance_record(const double* part_e, const double* part_h, int nblocks, double n, double m,
                                  double share, const double* qmax, double* rec) {
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nblocks; q += 32) {
    a = fmax(a, part_e[q]);
    b = fmax(b, part_h[q]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_down_sync(0xffffffffu, b, o));
  }
  if (threadIdx.x == 0) {
    rec[0] = n;
    rec[1] = m;
    rec[3] = a;
    rec[4] = b;
    rec[5] = qmax ? share * *qmax : 0.0;
  }
}

// Static start: number of activity bytes of rows 2..K that differ from row 1
__global__ void rz_row_mismatch(const uint8_t* mask, RzLayout L, int K, unsigned long long* out) {
  const long long total = (long long)(K - 1) * L.pr;
  unsigned long long c = 0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long k = 2 + q / L.pr, col = q % L.pr;
    c += mask[(k + 1) * L.pr + col] != mask[2 * L.pr + col];
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// Static start: the TEM field of every mode on planes 0..K+1 (see
// tetm_rz_set_bunch_static); psi [mode][nr+1], G [mode][K+4] (G[u+1]),
// metric [mode][6][pr] (column orr = axis).
template <typename T>
__global__ void rz_write_tem(T* f, RzLayout L, const uint8_t* mask, const double* metric, int m_lo,
                             int n_modes, const double* psi, const double* G, int K, double dr,
                             double eta0) {
  const long long per_mode = (long long)(L.nr + 1) * (K + 2);
  const long long total = per_mode * n_modes;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int mode = (int)(q / per_mode);
    const long long t = q % per_mode;
    const int i = (int)(t % (L.nr + 1)), k = (int)(t / (L.nr + 1));
    const uint8_t b = mask[L.midx(i, k)];
    const double* me = metric + (long long)mode * 6 * L.pr + L.orr + i;
    auto act = [&](int c) { return ((b >> c) & 1) && me[c * L.pr] != 0.0; };
    const double* ps = psi + (long long)mode * (L.nr + 1);
    const double* g = G + (long long)mode * (K + 4);
    const double g0 = g[k + 1], g1 = g[k + 2];
    const double m = (double)(m_lo + mode);
    const double prp = i < L.nr ? ps[i + 1] - ps[i] : 0.0;
    T* e = f + L.fidx(mode, 0, i, k);
    e[kER] = act(kER) ? (T)(-prp * g0) : T(0);
    e[kEP] = act(kEP) ? (T)(-m * ps[i] * g0) : T(0);
    e[kEZ] = T(0);
    e[kHP] = act(kHP) ? (T)(((i + 0.5) * dr / (dr * eta0)) * prp * g1) : T(0);
    e[kHR] = (act(kHR) && i > 0) ? (T)(-(dr / (i * dr * eta0)) * m * ps[i] * g1) : T(0);
    e[kHZ] = T(0);
  }
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
  void* coef = nullptr;          // [mode][kNCo][pr], T (material arrays: [mode][rows][kNCo][pr])
  double* metric = nullptr;      // [mode][6][pr] (material arrays: [mode][rows][6][pr])
  bool mat = false;              // per-cell eps_r / mu_r: coefficients per entry
  long long co_mode = 0, co_plane = 0;  // strides of coef per mode and per plane row (0: one row for all)
  long long me_mode = 0, me_plane = 0;  // the same for metric
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
  // the source-window launch of a scattered-form pass runs on a side stream,
  // beside the plain launch (their items are disjoint), joined before the next pass
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int resident = 0;
  int kernel = TETM_RZ_KERNEL_ASYNC;
  int* err = nullptr;            // device error word of the bulk-copy kernel
  int obs = 0;                   // transverse wake at r_{obs+1/2}
  long long kshift = 0;          // static start: head at plane step + kshift
  int tile_w = kTile;            // owned entries per window of the current work list
  double* WT = nullptr;          // [mode][nw]
  // scattered-field form (tetm_rz_set_bunch_scattered)
  bool scattered = false;
  double* inc_prof = nullptr;    // [mode][6][pr]
  double* inc_G = nullptr;       // [mode][inc_glen]
  int inc_glen = 0;
  void* S = nullptr;             // [kSourceSlots][mode][sc_len][pr * 6], field precision
  long long sc_until = 0;        // sources are ready for steps below this one
  std::vector<int> chunk_first;  // [n_chunks + 1]: first work-list entry of each chunk
  void* Jzero = nullptr;         // the step kernels' current in the scattered form (zeros)
  uint8_t* differs = nullptr;    // [nz + 2][s_tiles]: row k + 1 differs from the entry section
  long long sc_off = 0;          // source window: planes n + sc_off .. + sc_len - 1
  int sc_len = 0;
  int s_tiles = 0;               // radial tiles (of 60 entries) the source covers
  // balances (energy of Sec. 4.4, charges of Sec. 4.5) of every mode
  bool prev_valid = false;       // set[cur ^ 1] holds the state one step before set[cur]
  int bal_every = 0;
  double* hist = nullptr;        // [hist_cap][n_modes][kRzRec] records
  int hist_cap = 0;
  long long hist_count = 0;
  double* cpart = nullptr;       // charge partials [2][kEnergyBlocks], the bunch line [nz + 1] and its max
  double* rec1 = nullptr;        // [n_modes][kRzRec]: the records of tetm_rz_charge_residual
};

namespace {

RzIncident rz_incident(const tetm_rz* s, long long n) {
  RzIncident x;
  x.prof = s->scattered ? s->inc_prof : nullptr;
  x.G = s->inc_G;
  x.glen = s->inc_glen;
  x.n = n;
  x.L = s->L;
  return x;
}

constexpr int kSourcePlanes = 2;  // planes per source work item

// Sources of the scattered-field form for steps s->step .. s->step + n_steps - 1.
template <typename T>
cudaError_t rz_launch_source(tetm_rz* s, int n_steps) {
  RzArgs<T> a{};
  a.L = s->L;
  a.mask = s->mask;
  a.coef = static_cast<const T*>(s->coef);
  a.co_mode = s->co_mode;
  a.co_plane = s->co_plane;
  a.m_lo = s->g.m_lo;
  a.n_modes = s->n_modes;
  a.b_on = 1;
  a.i0 = s->i0;
  a.c0 = s->c0;
  a.J = static_cast<const T*>(s->J);
  a.kshift = s->kshift;
  a.sc_off = s->sc_off;
  a.sc_len = s->sc_len;
  const int n_groups = (s->sc_len + kSourcePlanes - 1) / kSourcePlanes;
  const long long items = (long long)n_steps * s->n_modes * s->s_tiles * n_groups;
  const int blocks = (int)std::max(1LL, std::min((items + 3) / 4, (long long)4 * s->resident));
  rz_source_kernel<T><<<blocks, 128, 0, s->st>>>(a, rz_incident(s, s->step), s->differs, s->s_tiles,
                                                  kSourcePlanes, n_groups, n_steps, static_cast<T*>(s->S));
  return cudaGetLastError();
}

// Queues the balances of every mode for the state just reached into rec
// (kRzRec doubles per mode): energy, charges against the bunch (its node
// charges for the centre of the last step, as in the Cartesian solver).
template <typename T>
int rz_queue_balances(tetm_rz* s, double* rec) {
  if (!s->cpart) {
    cudaError_t e = cudaMalloc(&s->cpart, sizeof(double) * (2 * kEnergyBlocks + s->g.nz + 2));
    if (e != cudaSuccess) return rz_fail(e);
  }
  double* pe = s->cpart;
  double* ph = s->cpart + kEnergyBlocks;
  double* ql = s->cpart + 2 * kEnergyBlocks;
  double* qmax = ql + s->g.nz + 1;
  const double zc = ((double)(s->step + s->kshift - 1) + 0.5 - s->c0) * s->g.dz;
  cudaError_t e = tetm::launch_bunch_charge(s->bunch ? s->q : 0.0, s->bunch ? s->sigma : 1.0, s->g.dz, zc, s->g.nz, ql,
                                      qmax, 0.0, nullptr, s->st);
  const T* fc = static_cast<const T*>(s->set[s->cur]);
  const T* fp = static_cast<const T*>(s->set[s->cur ^ 1]);
  for (int mi = 0; mi < s->n_modes && e == cudaSuccess; ++mi) {
    const int m = s->g.m_lo + mi;
    const double share = (m == 0 ? 1.0 : 2.0) / (2.0 * kPi);
    double* r = rec + (size_t)mi * kRzRec;
    const double* me = s->metric + (size_t)mi * s->me_mode + s->L.orr;
    rz_energy_partial<T><<<kEnergyBlocks, kEnergyThreads, 0, s->st>>>(fc, s->L, mi, s->mask, me, s->me_plane,
                                                                       s->alpha, s->partial, rz_incident(s, s->step));
    rz_energy_final<<<1, 32, 0, s->st>>>(s->partial, kEnergyBlocks, r + 2);
    rz_charge_partial<T><<<kEnergyBlocks, kEnergyThreads, 0, s->st>>>(
        fc, fp, s->L, mi, (double)m, s->mask, me, s->me_plane, s->alpha * s->alpha, rz_incident(s, s->step),
        rz_incident(s, s->step - 1), s->bunch ? ql : nullptr, share, s->i0, pe, ph);
    rz_balance_record<<<1, 32, 0, s->st>>>(pe, ph, kEnergyBlocks, (double)s->step, (double)m, share,
                                           s->bunch ? qmax : nullptr, r);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? TETM_OK : rz_fail(e);
}

template <typename T>
int rz_launch_steps(tetm_rz* s, long long n) {
  RzArgs<T> a;
  a.L = s->L;
  a.mask = s->mask;
  a.coef = static_cast<const T*>(s->coef);
  a.co_mode = s->co_mode;
  a.co_plane = s->co_plane;
  a.m_lo = s->g.m_lo;
  a.n_modes = s->n_modes;
  a.tiles = s->tiles;
  a.chunk_z = s->chunk_z;
  a.tile_w = s->tile_w;
  a.halo = s->tile_w == kTile2 ? 4 : 2;
  a.work = s->work;
  a.n_work = s->n_work;
  a.b_on = s->bunch ? 1 : 0;
  a.i0 = s->i0;
  a.c0 = s->c0;
  a.m_min = s->m_min;
  a.nw = s->nw;
  a.J = static_cast<const T*>(s->scattered ? s->Jzero : s->J);
  a.S = s->scattered ? static_cast<const T*>(s->S) : nullptr;
  a.sc_off = s->sc_off;
  a.sc_len = s->sc_len;
  a.W = s->W;
  a.inv_q = s->bunch ? 1.0 / s->q : 0.0;
  a.err = s->err;
  a.kshift = s->kshift;
  a.obs = s->obs;
  a.WT = s->WT;
  if (s->bunch) {
    const double rh = (s->obs + 0.5) * s->g.dr;
    a.tw_er = s->g.dz / (s->q * s->g.dr);
    a.tw_hp = kMu0 * kC * s->g.dz / (s->q * rh);
  } else {
    a.tw_er = a.tw_hp = 0.0;
  }
  const int items = s->n_work * s->n_modes;
  const int blocks = std::max(1, std::min(s->resident, (items + 3) / 4));
  // launches one step kernel over the plain items (SC = false) or over the
  // items meeting a source window (SC = true)
  auto launch = [&](bool sc, int steps, int nblocks, cudaStream_t st) {
    if (steps == 2) {
      if (sc) rz_step_bulk2_kernel<T, true><<<nblocks, 128, 4 * rz_bulk_warp_bytes<T>(), st>>>(a);
      else rz_step_bulk2_kernel<T, false><<<nblocks, 128, 4 * rz_bulk_warp_bytes<T>(), st>>>(a);
    } else if (s->kernel == TETM_RZ_KERNEL_BULK || s->kernel == TETM_RZ_KERNEL_BULK2) {
      if (sc) rz_step_bulk_kernel<T, true><<<nblocks, 128, 4 * rz_bulk_warp_bytes<T>(), st>>>(a);
      else rz_step_bulk_kernel<T, false><<<nblocks, 128, 4 * rz_bulk_warp_bytes<T>(), st>>>(a);
    } else if (s->kernel == TETM_RZ_KERNEL_ASYNC) {
      if (sc) rz_step_async_kernel<T, true><<<nblocks, 128, 4 * rz_async_warp_bytes<T>(), st>>>(a);
      else rz_step_async_kernel<T, false><<<nblocks, 128, 4 * rz_async_warp_bytes<T>(), st>>>(a);
    } else if (s->mat) {  // material arrays: the register kernel, coefficients per plane
      rz_step_kernel<T, false, true><<<nblocks, 128, 0, st>>>(a);
    } else {
      if (sc) rz_step_kernel<T, true><<<nblocks, 128, 0, st>>>(a);
      else rz_step_kernel<T, false><<<nblocks, 128, 0, st>>>(a);
    }
    return cudaGetLastError();
  };
  for (long long t = 0; t < n; ++t) {
    a.in = static_cast<const T*>(s->set[s->cur]);
    a.out = static_cast<T*>(s->set[s->cur ^ 1]);
    a.n = s->step;
    // steps in this pass: two with the two-step kernel, except past or into
    // a step that carries balances (they need the state one step before it)
    int p = (s->kernel == TETM_RZ_KERNEL_BULK2 && t + 1 < n) ? 2 : 1;
    if (p == 2 && s->bal_every > 0 &&
        ((s->step + 1) % s->bal_every == 0 || (s->step + 2) % s->bal_every == 0))
      p = 1;
    a.sc_lo = a.sc_hi = 0;
    if (s->scattered) {
      if (s->step + p > s->sc_until) {
        // the sources of the next kSourceSlots steps in one launch (their
        // slots were last read by passes queued before it)
        cudaError_t e = rz_launch_source<T>(s, kSourceSlots);
        if (e != cudaSuccess) return rz_fail(e);
        s->sc_until = s->step + kSourceSlots;
      }
      // the items whose planes (with the recomputed ones: k0-2 .. k1) meet
      // the windows [lo, hi) of this pass's steps: chunks c with
      // (c+1) cz + 1 > lo and c cz - 2 < hi, a contiguous run of the work
      // list (ordered by chunk)
      const long long lo = s->step + s->sc_off, hi = s->step + p - 1 + s->sc_off + s->sc_len;
      const long long cz = s->chunk_z;
      const long long c_lo = lo >= 1 ? (lo - 1) / cz : 0;
      const long long c_hi = std::min((long long)s->n_chunks, hi + 2 > 0 ? (hi + 2 + cz - 1) / cz : 0LL);
      if (c_lo < c_hi) {
        a.sc_lo = s->chunk_first[(size_t)c_lo] * s->n_modes;
        a.sc_hi = s->chunk_first[(size_t)c_hi] * s->n_modes;
      }
    }
    if (items > 0) {
      const bool win = a.sc_hi > a.sc_lo;
      if (win && !s->side) {  // the side stream and its two events, once
        if (cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess)
          return rz_fail(cudaGetLastError());
      }
      if (win) {
        // fork: the window items (whose sources were queued on the main stream
        // before) on the side stream, the plain items on the main stream
        const int nsub = (s->chunk_z + kSubPlanes - 1) / kSubPlanes;
        cudaError_t e = cudaEventRecord(s->ev_fork, s->st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s->side, s->ev_fork, 0);
        if (e == cudaSuccess)
          e = launch(true, p, std::max(1, std::min(blocks, ((a.sc_hi - a.sc_lo) * nsub + 3) / 4)), s->side);
        if (e == cudaSuccess) e = cudaEventRecord(s->ev_join, s->side);
        if (e != cudaSuccess) return rz_fail(e);
      }
      cudaError_t e = launch(false, p, blocks, s->st);
      if (e == cudaSuccess && win) e = cudaStreamWaitEvent(s->st, s->ev_join, 0);  // join
      if (e != cudaSuccess) return rz_fail(e);
    }
    s->cur ^= 1;
    s->step += p;
    s->prev_valid = p == 1;
    t += p - 1;
    if (s->bal_every > 0 && s->step % s->bal_every == 0) {
      double* rec = s->hist + (size_t)(s->hist_count % s->hist_cap) * s->n_modes * kRzRec;
      const int rc = rz_queue_balances<T>(s, rec);
      if (rc) return rc;
      s->hist_count += 1;
    }
  }
  return TETM_OK;
}

// Blocks of 4 warps the step kernel keeps resident on the whole device.
template <typename T>
int rz_occupancy(tetm_rz* s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t smem = 4 * rz_async_warp_bytes<T>();
  if (e == cudaSuccess && smem > 48 * 1024)
    e = cudaFuncSetAttribute(rz_step_async_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  if (e == cudaSuccess && smem > 48 * 1024)
    e = cudaFuncSetAttribute(rz_step_async_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  const size_t bsmem = 4 * rz_bulk_warp_bytes<T>();
  if (e == cudaSuccess && bsmem > 48 * 1024)
    e = cudaFuncSetAttribute(rz_step_bulk_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bsmem);
  if (e == cudaSuccess && bsmem > 48 * 1024)
    e = cudaFuncSetAttribute(rz_step_bulk_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bsmem);
  if (e == cudaSuccess && bsmem > 48 * 1024)
    e = cudaFuncSetAttribute(rz_step_bulk2_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bsmem);
  if (e == cudaSuccess && bsmem > 48 * 1024)
    e = cudaFuncSetAttribute(rz_step_bulk2_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bsmem);
  if (e == cudaSuccess) {
    if (s->kernel == TETM_RZ_KERNEL_BULK2)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rz_step_bulk2_kernel<T, false>, 128, bsmem);
    else if (s->kernel == TETM_RZ_KERNEL_BULK)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rz_step_bulk_kernel<T, false>, 128, bsmem);
    else if (s->kernel == TETM_RZ_KERNEL_ASYNC)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rz_step_async_kernel<T, false>, 128, smem);
    else
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rz_step_kernel<T, false>, 128, 0);
  }
  if (e != cudaSuccess) return rz_fail(e);
  s->resident = std::max(1, sms * per_sm);
  return TETM_OK;
}

int rz_rebuild_work(tetm_rz* s) {
  const RzLayout& L = s->L;
  const int tw = s->kernel == TETM_RZ_KERNEL_BULK2 ? kTile2 : kTile;
  s->tile_w = tw;
  s->tiles = (L.nr + 1 + tw - 1) / tw;
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
  rz_item_flags<<<(nf + 255) / 256, 256, 0, s->st>>>(s->mask, L, s->tiles, tw, s->chunk_z,
                                                      s->n_chunks, s->flags);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rz_fail(e);
  std::vector<int> fl((size_t)nf);
  e = cudaMemcpyAsync(fl.data(), s->flags, sizeof(int) * (size_t)nf, cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return rz_fail(e);
  std::vector<int> w;
  long long processed = 0;
  s->chunk_first.assign((size_t)s->n_chunks + 1, 0);
  for (int q = 0; q < nf; ++q) {
    if (q % s->tiles == 0) s->chunk_first[(size_t)(q / s->tiles)] = (int)w.size();
    if (!fl[(size_t)q]) continue;
    w.push_back(q);
    const int tile = q % s->tiles, chunk = q / s->tiles;
    const int width = std::min(tw, L.nr + 1 - tile * tw);
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
  s->chunk_first[(size_t)s->n_chunks] = s->n_work;
  s->processed = processed * s->n_modes;
  s->work_dirty = false;
  return TETM_OK;
}

// Per-radian metric of one mode at radial index i (unscaled M^-1; zero where
// the mode has no object) and the update coefficients derived from it.
__host__ __device__ inline void rz_metric_at(double dr, double dz, int nr, int m, int i, double out[6]) {
  const double ri = i * dr, rh = (i + 0.5) * dr;
  out[kER] = i < nr ? dr / (kEps0 * rh * dz) : 0.0;
  out[kEP] = (i > 0 && i < nr) ? ri / (kEps0 * dr * dz) : 0.0;
  if (i == 0) out[kEZ] = m == 0 ? dz / (kEps0 * dr * dr / 4.0) : 0.0;
  else out[kEZ] = i < nr ? dz / (kEps0 * ri * dr) : 0.0;
  out[kHR] = (i > 0 && i < nr) ? dr / (kMu0 * ri * dz) : 0.0;
  out[kHP] = i < nr ? rh / (kMu0 * dr * dz) : 0.0;
  out[kHZ] = i < nr ? dz / (kMu0 * rh * dr) : 0.0;
}
void rz_metric_row(const tetm_rz_grid& g, int m, int i, double out[6]) { rz_metric_at(g.dr, g.dz, g.nr, m, i, out); }

// Material arrays (per cell, eps_r / mu_r at ci + nr ck, nullptr = 1): the
// metric and coefficients of every entry (i, k), k = -1 .. nz+1, of every
// mode. The column's metric is divided by the staircase mean of eps_r over
// the cells an edge touches (e_r, e_z two, e_phi four; the axis e_z its one
// cell) and multiplied by the mean of 1/mu_r over the cells a face touches
// (h_phi its cell, h_r and h_z two), as in the 3D material matrices (Sec. 2).
// A cell outside the grid counts as vacuum: an object that touches one lies
// in the PEC wall, carries no field and its value is never read.
template <typename T>
__global__ void rz_material_coefs(const double* eps, const double* mu, RzLayout L, double dr, double dz,
                                  int m_lo, int n_modes, double alpha, T* coef, double* metric) {
  const int nr = L.nr, nz = L.nz;
  const long long PR = L.pr;
  const long long n = L.rows * (long long)(nr + 1);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % (nr + 1)), row = (int)(q / (nr + 1)), k = row - 1;
    auto inside = [&](int ci, int ck) { return ci >= 0 && ci < nr && ck >= 0 && ck < nz; };
    auto E = [&](int ci, int ck) { return eps && inside(ci, ck) ? eps[ci + (long long)nr * ck] : 1.0; };
    auto IM = [&](int ci, int ck) { return mu && inside(ci, ck) ? 1.0 / mu[ci + (long long)nr * ck] : 1.0; };
    double f[6];
    f[kER] = 1.0 / (0.5 * (E(i, k - 1) + E(i, k)));
    f[kEP] = 1.0 / ((E(i - 1, k - 1) + E(i - 1, k) + E(i, k - 1) + E(i, k)) / 4.0);
    f[kEZ] = i == 0 ? 1.0 / E(0, k) : 1.0 / (0.5 * (E(i - 1, k) + E(i, k)));
    f[kHP] = IM(i, k);
    f[kHR] = 0.5 * (IM(i - 1, k) + IM(i, k));
    f[kHZ] = 0.5 * (IM(i, k - 1) + IM(i, k));
    for (int mi = 0; mi < n_modes; ++mi) {
      const int m = m_lo + mi;
      double c[6];
      rz_metric_at(dr, dz, nr, m, i, c);
      for (int comp = 0; comp < 6; ++comp) c[comp] *= f[comp];
      const long long col = i + L.orr;
      double* me = metric + (((long long)mi * L.rows + row) * 6) * PR + col;
      for (int comp = 0; comp < 6; ++comp) me[comp * PR] = c[comp];
      T* co = coef + (((long long)mi * L.rows + row) * kNCo) * PR + col;
      const double mm = (double)m * m;
      co[kCoER * PR] = (T)(alpha * c[kER]);
      co[kCoEP * PR] = (T)(alpha * c[kEP]);
      co[kCoHR * PR] = (T)(alpha * c[kHR]);
      co[kCoHP * PR] = (T)(alpha * c[kHP]);
      co[kCoEZ * PR] = (T)(2.0 * alpha * c[kEZ]);
      co[kCoHZ * PR] = (T)(2.0 * alpha * c[kHZ]);
      co[kCoFEZ * PR] = (T)(2.0 * alpha * c[kEZ] / (1.0 + alpha * alpha * mm * c[kEZ] * c[kHR]));
      co[kCoFHZ * PR] = (T)(2.0 * alpha * c[kHZ] / (1.0 + alpha * alpha * mm * c[kHZ] * c[kER]));
    }
  }
}

// uploads the material arrays and fills coef and metric on the device
template <typename T>
int rz_material_setup(tetm_rz* s, const double* eps_r, const double* mu_r) {
  const size_t nc = (size_t)s->g.nr * s->g.nz;
  double *deps = nullptr, *dmu = nullptr;
  cudaError_t e = cudaSuccess;
  if (eps_r) e = cudaMalloc(&deps, sizeof(double) * nc);
  if (e == cudaSuccess && mu_r) e = cudaMalloc(&dmu, sizeof(double) * nc);
  if (e == cudaSuccess && eps_r) e = cudaMemcpyAsync(deps, eps_r, sizeof(double) * nc, cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess && mu_r) e = cudaMemcpyAsync(dmu, mu_r, sizeof(double) * nc, cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess) {
    rz_material_coefs<T><<<1024, 256, 0, s->st>>>(deps, dmu, s->L, s->g.dr, s->g.dz, s->g.m_lo, s->n_modes, s->alpha,
                                                  static_cast<T*>(s->coef), s->metric);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  cudaFree(deps);
  cudaFree(dmu);
  return e == cudaSuccess ? TETM_OK : rz_fail(e);
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
  return (size_t)n_modes * (size_t)L.mode_elems() * (size_t)esz;
}

bool rz_mode_ok(const tetm_rz* s, int mode) { return s && mode >= 0 && mode < s->n_modes; }

// a wake of one mode: the sum of its even-step and odd-step halves
int rz_read_wake(tetm_rz* s, const double* W, int mode, double* out) {
  std::vector<double> h((size_t)2 * s->nw);
  const size_t half = (size_t)s->n_modes * s->nw;
  cudaError_t e = cudaMemcpyAsync(h.data(), W + (size_t)mode * s->nw, sizeof(double) * s->nw,
                                  cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data() + s->nw, W + half + (size_t)mode * s->nw, sizeof(double) * s->nw,
                        cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return rz_fail(e);
  for (int q = 0; q < s->nw; ++q) out[q] = h[(size_t)q] + h[(size_t)(s->nw + q)];
  return TETM_OK;
}

}  // namespace

extern "C" {

int64_t tetm_rz_bytes_needed(const tetm_rz_grid* g) {
  if (!rz_grid_ok(g)) return 0;
  const int esz = g->precision == TETM_FP64 ? 8 : 4;
  const int nm = g->m_hi - g->m_lo + 1;
  const RzLayout L = make_rz_layout(g->nr, g->nz);
  return (int64_t)(2 * rz_field_bytes(L, esz, nm) + (size_t)(L.rows * L.pr) +
                   (size_t)nm * L.pr * (kNCo * esz + 6 * 8)) + (int64_t)(1 << 20);
}

int tetm_rz_create(const tetm_rz_grid* g, const double* eps_r, const double* mu_r,
                   const uint8_t* pec, tetm_rz** out) {
  if (!out) return TETM_E_ARG;
  *out = nullptr;
  if (!rz_grid_ok(g)) return TETM_E_ARG;
  // material arrays: physical (>= 1) and finite; all ones is the vacuum
  bool mat = false;
  const long long ncell = (long long)g->nr * g->nz;
  for (const double* a : {eps_r, mu_r}) {
    if (!a) continue;
    for (long long q = 0; q < ncell; ++q) {
      if (!(a[q] >= 1.0) || !isfinite(a[q])) return TETM_E_ARG;
      if (a[q] != 1.0) mat = true;
    }
  }
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
  s->L = make_rz_layout(g->nr, g->nz);
  s->mat = mat;
  const long long prows = mat ? s->L.rows : 1;  // coefficient rows per mode
  s->co_plane = mat ? (long long)kNCo * s->L.pr : 0;
  s->co_mode = prows * kNCo * s->L.pr;
  s->me_plane = mat ? 6LL * s->L.pr : 0;
  s->me_mode = prows * 6 * s->L.pr;
  if (mat) s->kernel = TETM_RZ_KERNEL_REGISTER;  // the kernel that reads coefficients per plane
  int rc = TETM_OK;
  uint8_t* dpec = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete s;
    return rz_fail(e);
  }
  s->st = s->own;
  const size_t fb = rz_field_bytes(s->L, s->esz, s->n_modes);
  const size_t cob = (size_t)s->n_modes * s->co_mode * s->esz;
  const size_t meb = (size_t)s->n_modes * s->me_mode * sizeof(double);
  do {
    if ((e = cudaMalloc(&s->set[0], fb)) != cudaSuccess) break;
    if ((e = cudaMalloc(&s->set[1], fb)) != cudaSuccess) break;
    if ((e = cudaMalloc(&s->mask, (size_t)(s->L.rows * s->L.pr))) != cudaSuccess) break;
    if ((e = cudaMalloc(&s->coef, cob)) != cudaSuccess) break;
    if ((e = cudaMalloc(&s->metric, meb)) != cudaSuccess) break;
    if ((e = cudaMalloc(&s->partial, sizeof(double) * (kEnergyBlocks + 1))) != cudaSuccess) break;
    if ((e = cudaMalloc(&s->err, sizeof(int))) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(s->err, 0, sizeof(int), s->st)) != cudaSuccess) break;
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
  if (rc == TETM_OK && mat) {
    if (cudaMemsetAsync(s->coef, 0, cob, s->st) != cudaSuccess || cudaMemsetAsync(s->metric, 0, meb, s->st) != cudaSuccess)
      rc = TETM_E_CUDA;
    if (rc == TETM_OK)
      rc = s->esz == 8 ? rz_material_setup<double>(s, eps_r, mu_r) : rz_material_setup<float>(s, eps_r, mu_r);
  } else if (rc == TETM_OK) {
    rc = s->esz == 8 ? rz_upload_coefs<double>(s) : rz_upload_coefs<float>(s);
  }
  if (rc == TETM_OK) rc = s->esz == 8 ? rz_occupancy<double>(s) : rz_occupancy<float>(s);
  if (rc == TETM_OK) rc = rz_rebuild_work(s);
  if (rc != TETM_OK) {
    tetm_rz_destroy(s);
    return rc;
  }
  s->device_bytes = (long long)(2 * fb + (size_t)(s->L.rows * s->L.pr) + cob + meb);
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
  double *W = nullptr, *WT = nullptr;
  cudaError_t e = cudaMalloc(&J, (size_t)s->esz * nj);
  if (e == cudaSuccess) e = cudaMalloc(&W, 2 * sizeof(double) * (size_t)s->n_modes * nw);
  if (e == cudaSuccess) e = cudaMalloc(&WT, 2 * sizeof(double) * (size_t)s->n_modes * nw);
  if (e == cudaSuccess) e = cudaMemset(WT, 0, 2 * sizeof(double) * (size_t)s->n_modes * nw);
  if (e == cudaSuccess)
    e = cudaMemcpy(J, s->esz == 8 ? (const void*)jd.data() : (const void*)jf.data(),
                   (size_t)s->esz * nj, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(W, 0, 2 * sizeof(double) * (size_t)s->n_modes * nw);
  if (e != cudaSuccess) {
    cudaFree(J);
    cudaFree(W);
    cudaFree(WT);
    return rz_fail(e);
  }
  s->J = J;
  s->W = W;
  s->WT = WT;
  s->obs = i0 < s->g.nr - 1 ? i0 : s->g.nr - 2;
  s->bunch = true;
  s->i0 = i0;
  s->c0 = c0;
  s->m_min = -c0 - 1;
  s->m_max = m_max;
  s->nw = nw;
  s->q = q;
  s->sigma = sigma;
  s->device_bytes += (long long)((size_t)s->esz * nj + 4 * sizeof(double) * (size_t)s->n_modes * nw);
  return TETM_OK;
}

int tetm_rz_step(tetm_rz* s, int64_t n) {
  if (!s || n < 0) return TETM_E_ARG;
  if (s->work_dirty) {
    int rc = rz_rebuild_work(s);
    if (rc) return rc;
  }
  nvtxRangePushA("tetm_rz_step");
  const int rc = s->esz == 8 ? rz_launch_steps<double>(s, n) : rz_launch_steps<float>(s, n);
  nvtxRangePop();
  return rc;
}

int tetm_rz_sync(tetm_rz* s) {
  if (!s) return TETM_E_ARG;
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return rz_fail(e);
  return flag ? TETM_E_TIMEOUT : TETM_OK;
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
  return rz_read_wake(s, s->W, mode, out);
}

}  // extern "C"

namespace {

// The entry pipe's TEM field of the ring bunch (static start and scattered
// form): checks the arguments and that planes 1..K carry the activity bytes of
// plane 1 (row: those bytes), solves every mode's radial potential psi
// [mode][nr+1] and the longitudinal profile G [mode][K+4] (G[u+1]).
int rz_tem_setup(tetm_rz* s, double sigma, double q, int i0, int k_head, std::vector<uint8_t>& row,
                 std::vector<double>& psi, std::vector<double>& G) {
  if (!s) return TETM_E_ARG;
  if (s->mat) return TETM_E_UNSUPPORTED;  // the static start's entry section is vacuum
  if (s->step != 0 || s->bunch) return TETM_E_STATE;
  if (!(sigma > 0) || !isfinite(sigma)) return TETM_E_ARG;
  const double dz = s->g.dz, dr = s->g.dr;
  const int c0 = (int)ceil(5.0 * sigma / dz - 1e-12);
  const int K = k_head;
  if (K < 2 * c0 + 2 || K > s->g.nz || i0 < 0 || i0 >= s->g.nr) return TETM_E_ARG;
  const RzLayout& L = s->L;
  // the entry section: rows 2..K carry the activity bytes of row 1
  unsigned long long* dcount = nullptr;
  cudaError_t e = cudaMalloc(&dcount, sizeof(unsigned long long));
  if (e != cudaSuccess) return rz_fail(e);
  unsigned long long mism = 0;
  row.assign((size_t)L.pr, 0);
  e = cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), s->st);
  if (e == cudaSuccess) {
    rz_row_mismatch<<<256, 256, 0, s->st>>>(s->mask, L, K, dcount);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&mism, dcount, sizeof(mism), cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(row.data(), s->mask + 2 * L.pr, (size_t)L.pr, cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  cudaFree(dcount);
  if (e != cudaSuccess) return rz_fail(e);
  if (mism) return TETM_E_ARG;
  // per mode: the radial potential (tridiagonal, symmetric positive definite,
  // eliminated without pivoting) and the longitudinal profile
  const int nn = s->g.nr + 1;
  const double eta0 = kMu0 * kC;
  psi.assign((size_t)s->n_modes * nn, 0.0);
  G.assign((size_t)s->n_modes * (K + 4), 0.0);
  std::vector<double> qc((size_t)(2 * c0));
  for (int d = -c0; d < c0; ++d) {
    const double lo = std::max((double)d * dz, -5.0 * sigma);
    const double hi = std::min((double)(d + 1) * dz, 5.0 * sigma);
    qc[(size_t)(d + c0)] = hi > lo ? q * (rz_phi(hi / sigma) - rz_phi(lo / sigma)) : 0.0;
  }
  for (int mi = 0; mi < s->n_modes; ++mi) {
    const int m = s->g.m_lo + mi;
    std::vector<int> unk((size_t)nn);
    for (int i = 0; i < nn; ++i) {
      double c[6];
      rz_metric_row(s->g, m, i, c);
      unk[(size_t)i] = ((row[(size_t)L.col(i)] >> kEZ) & 1) && c[kEZ] != 0.0;
    }
    if (!unk[(size_t)i0]) return TETM_E_ARG;   // the axis carries only m = 0
    std::vector<double> a((size_t)nn, 0.0), b((size_t)nn, 0.0), cc((size_t)nn, 0.0), r((size_t)nn, 0.0);
    auto er_on = [&](int i) { return i >= 0 && i < s->g.nr && ((row[(size_t)L.col(i)] >> kER) & 1); };
    for (int i = 0; i < nn; ++i) {
      if (!unk[(size_t)i]) { b[(size_t)i] = 1.0; continue; }
      if (i + 1 < nn && er_on(i)) {
        const double w = (i + 0.5) * dr / dr;
        b[(size_t)i] += w;
        if (unk[(size_t)i + 1]) cc[(size_t)i] = -w;
      }
      if (i >= 1 && er_on(i - 1)) {
        const double w = (i - 0.5) * dr / dr;
        b[(size_t)i] += w;
        if (unk[(size_t)i - 1]) a[(size_t)i] = -w;
      }
      if (i >= 1) b[(size_t)i] += (double)m * m * dr / (i * dr);
    }
    r[(size_t)i0] = 1.0;
    for (int i = 1; i < nn; ++i) {
      const double f = a[(size_t)i] / b[(size_t)i - 1];
      b[(size_t)i] -= f * cc[(size_t)i - 1];
      r[(size_t)i] -= f * r[(size_t)i - 1];
    }
    double* ps = psi.data() + (size_t)mi * nn;
    ps[nn - 1] = r[(size_t)nn - 1] / b[(size_t)nn - 1];
    for (int i = nn - 2; i >= 0; --i) ps[i] = (r[(size_t)i] - cc[(size_t)i] * ps[i + 1]) / b[(size_t)i];
    for (int i = 0; i < nn; ++i) if (!unk[(size_t)i]) ps[i] = 0.0;
    const double share = (m == 0 ? 1.0 : 2.0) / (2.0 * kPi);
    double* g = G.data() + (size_t)mi * (K + 4);
    for (int u = K - 1; u >= K - 2 * c0; --u)
      g[u + 1] = 2.0 * eta0 * (share * kC * qc[(size_t)(u - K + 2 * c0)] / dz) - g[u + 2];
  }
  return TETM_OK;
}

}  // namespace

extern "C" {

int tetm_rz_set_bunch_static(tetm_rz* s, double sigma, double q, int32_t i0, int32_t k_head) {
  if (!s) return TETM_E_ARG;
  if (s->step != 0 || s->bunch) return TETM_E_STATE;
  std::vector<uint8_t> row;
  std::vector<double> psi, G;
  int rc = rz_tem_setup(s, sigma, q, i0, k_head, row, psi, G);
  if (rc != TETM_OK) return rc;
  const RzLayout& L = s->L;
  const int K = k_head;
  const double dr = s->g.dr, eta0 = kMu0 * kC;
  cudaError_t e = cudaSuccess;
  rc = tetm_rz_set_bunch(s, sigma, q, i0);
  if (rc != TETM_OK) return rc;
  double *dpsi = nullptr, *dg = nullptr;
  e = cudaMalloc(&dpsi, sizeof(double) * psi.size());
  if (e == cudaSuccess) e = cudaMalloc(&dg, sizeof(double) * G.size());
  if (e == cudaSuccess) e = cudaMemcpyAsync(dpsi, psi.data(), sizeof(double) * psi.size(), cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dg, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess) {
    if (s->esz == 8)
      rz_write_tem<double><<<512, 256, 0, s->st>>>(static_cast<double*>(s->set[s->cur]), L, s->mask,
                                                   s->metric, s->g.m_lo, s->n_modes, dpsi, dg, K, dr, eta0);
    else
      rz_write_tem<float><<<512, 256, 0, s->st>>>(static_cast<float*>(s->set[s->cur]), L, s->mask,
                                                  s->metric, s->g.m_lo, s->n_modes, dpsi, dg, K, dr, eta0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  cudaFree(dpsi);
  cudaFree(dg);
  if (e != cudaSuccess) return rz_fail(e);
  s->kshift = K;
  return TETM_OK;
}

int tetm_rz_set_bunch_scattered(tetm_rz* s, double sigma, double q, int32_t i0, int32_t k_head) {
  if (!s) return TETM_E_ARG;
  if (s->step != 0 || s->bunch) return TETM_E_STATE;
  std::vector<uint8_t> row;
  std::vector<double> psi, G;
  int rc = rz_tem_setup(s, sigma, q, i0, k_head, row, psi, G);
  if (rc != TETM_OK) return rc;
  const RzLayout& L = s->L;
  const int K = k_head;
  const int nr = s->g.nr, nn = nr + 1;
  const double dr = s->g.dr, eta0 = kMu0 * kC;
  // the geometry holds every object of the entry section on planes 1..nz-1
  // (the incident field then vanishes wherever the geometry is PEC)
  unsigned long long* dcount = nullptr;
  unsigned long long uncovered = 0;
  cudaError_t e = cudaMalloc(&dcount, sizeof(unsigned long long));
  if (e != cudaSuccess) return rz_fail(e);
  e = cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), s->st);
  if (e == cudaSuccess) {
    rz_row_not_covered<<<256, 256, 0, s->st>>>(s->mask, L, dcount);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&uncovered, dcount, sizeof(uncovered), cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  cudaFree(dcount);
  if (e != cudaSuccess) return rz_fail(e);
  if (uncovered) return TETM_E_ARG;
  // the incident field's transverse profile (as the static start writes it)
  const long long PR = L.pr;
  std::vector<double> prof((size_t)s->n_modes * 6 * PR, 0.0);
  int i_top = 0;
  for (int mi = 0; mi < s->n_modes; ++mi) {
    const int m = s->g.m_lo + mi;
    const double* ps = psi.data() + (size_t)mi * nn;
    for (int i = 0; i <= nr; ++i) {
      double c[6];
      rz_metric_row(s->g, m, i, c);
      const uint8_t b = row[(size_t)L.col(i)];
      auto act = [&](int comp) { return ((b >> comp) & 1) && c[comp] != 0.0; };
      const double prp = i < nr ? ps[i + 1] - ps[i] : 0.0;
      double* pr = prof.data() + (size_t)mi * 6 * PR + L.col(i);
      pr[kER * PR] = act(kER) ? -prp : 0.0;
      pr[kEP * PR] = act(kEP) ? -m * ps[i] : 0.0;
      pr[kHP * PR] = act(kHP) ? ((i + 0.5) * dr / (dr * eta0)) * prp : 0.0;
      pr[kHR * PR] = (act(kHR) && i > 0) ? -(dr / (i * dr * eta0)) * m * ps[i] : 0.0;
      for (int comp = 0; comp < 6; ++comp)
        if (pr[comp * PR] != 0.0) i_top = std::max(i_top, i);
    }
  }
  const int c0 = (int)ceil(5.0 * sigma / s->g.dz - 1e-12);  // as tetm_rz_set_bunch
  const int tiles60 = (nr + 1 + kTile - 1) / kTile;
  const int s_tiles = std::min(tiles60, (i_top + 3 + kTile - 1) / kTile);  // the step reaches 2 entries out
  const int sc_len = 2 * c0 + 3;
  const size_t sbytes = (size_t)kSourceSlots * s->n_modes * sc_len * PR * 6 * s->esz;
  const size_t dbytes = (size_t)(s->g.nz + 2) * s_tiles;
  double *dprof = nullptr, *dG = nullptr;
  void *dS = nullptr, *dJ0 = nullptr;
  uint8_t* ddiff = nullptr;
  const size_t jbytes = (size_t)s->n_modes * 2 * c0 * s->esz;
  e = cudaMalloc(&dprof, sizeof(double) * prof.size());
  if (e == cudaSuccess) e = cudaMalloc(&dG, sizeof(double) * G.size());
  if (e == cudaSuccess) e = cudaMalloc(&dS, sbytes);
  if (e == cudaSuccess) e = cudaMalloc(&ddiff, dbytes);
  if (e == cudaSuccess) e = cudaMalloc(&dJ0, jbytes);
  if (e == cudaSuccess) e = cudaMemsetAsync(dJ0, 0, jbytes, s->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dS, 0, sbytes, s->st);
  if (e == cudaSuccess) {
    rz_row_differs<<<s->g.nz + 2, 256, 0, s->st>>>(s->mask, L, s_tiles, ddiff);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dprof, prof.data(), sizeof(double) * prof.size(), cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dG, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  rc = e == cudaSuccess ? tetm_rz_set_bunch(s, sigma, q, i0) : rz_fail(e);
  if (rc != TETM_OK) {
    cudaFree(dprof);
    cudaFree(dG);
    cudaFree(dS);
    cudaFree(ddiff);
    cudaFree(dJ0);
    return rc;
  }
  s->inc_prof = dprof;
  s->inc_G = dG;
  s->S = dS;
  s->differs = ddiff;
  s->Jzero = dJ0;
  s->s_tiles = s_tiles;
  s->sc_off = (long long)K - 2 * c0 - 2;
  s->sc_len = sc_len;
  s->inc_glen = K + 4;
  s->device_bytes += (long long)(sizeof(double) * (prof.size() + G.size()) + sbytes + dbytes + jbytes);
  s->kshift = K;
  s->scattered = true;
  return TETM_OK;
}

int tetm_rz_selftest_wait(int32_t polls) {
  if (polls < 1 || polls > (1 << 26)) return TETM_E_ARG;
  int* err = nullptr;
  cudaError_t e = cudaMalloc(&err, sizeof(int));
  if (e != cudaSuccess) return rz_fail(e);
  int flag = 0;
  e = cudaMemset(err, 0, sizeof(int));
  if (e == cudaSuccess) {
    rz_selftest_wait_kernel<<<1, 32>>>(polls, err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&flag, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(err);
  if (e != cudaSuccess) return rz_fail(e);
  return flag ? TETM_E_TIMEOUT : TETM_OK;
}

int tetm_rz_set_observer(tetm_rz* s, int32_t obs) {
  if (!s || obs < 0 || obs >= s->g.nr - 1) return TETM_E_ARG;
  if (!s->bunch || s->step != 0) return TETM_E_STATE;
  s->obs = obs;
  return TETM_OK;
}

int tetm_rz_transverse_wake(tetm_rz* s, int32_t mode, double* out, int32_t cap, int32_t* n_out,
                            double* s0, double* ds) {
  if (!rz_mode_ok(s, mode)) return TETM_E_ARG;
  if (!s->bunch) return TETM_E_STATE;
  if (n_out) *n_out = s->nw;
  if (s0) *s0 = s->m_min * s->g.dz;
  if (ds) *ds = s->g.dz;
  if (!out) return TETM_OK;
  if (cap < s->nw) return TETM_E_ARG;
  return rz_read_wake(s, s->WT, mode, out);
}

int tetm_rz_energy(tetm_rz* s, int32_t mode, double* w) {
  if (!rz_mode_ok(s, mode) || !w) return TETM_E_ARG;
  const void* f = s->set[s->cur];
  const double* me = s->metric + (size_t)mode * s->me_mode + s->L.orr;
  if (s->esz == 8)
    rz_energy_partial<double><<<kEnergyBlocks, kEnergyThreads, 0, s->st>>>(
        static_cast<const double*>(f), s->L, mode, s->mask, me, s->me_plane, s->alpha, s->partial,
        rz_incident(s, s->step));
  else
    rz_energy_partial<float><<<kEnergyBlocks, kEnergyThreads, 0, s->st>>>(
        static_cast<const float*>(f), s->L, mode, s->mask, me, s->me_plane, s->alpha, s->partial,
        rz_incident(s, s->step));
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
  const void* f = s->set[s->cur];
  if (s->esz == 8)
    rz_to_canonical<double><<<512, 256, 0, s->st>>>(static_cast<const double*>(f), s->L, mode, comp, tmp);
  else
    rz_to_canonical<float><<<512, 256, 0, s->st>>>(static_cast<const float*>(f), s->L, mode, comp, tmp);
  if (s->scattered) rz_canonical_add_inc<<<512, 256, 0, s->st>>>(tmp, rz_incident(s, s->step), mode, comp, 1.0);
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
  void* f = s->set[s->cur];
  const double* me = s->metric + (size_t)mode * s->me_mode + (size_t)comp * s->L.pr + s->L.orr;
  if (e == cudaSuccess) {
    if (s->esz == 8)
      rz_from_canonical<double><<<512, 256, 0, s->st>>>(tmp, s->L, s->mask, mode, comp, me, s->me_plane,
                                                        static_cast<double*>(f), rz_incident(s, s->step));
    else
      rz_from_canonical<float><<<512, 256, 0, s->st>>>(tmp, s->L, s->mask, mode, comp, me, s->me_plane,
                                                       static_cast<float*>(f), rz_incident(s, s->step));
    e = cudaGetLastError();
  }
  cudaFreeAsync(tmp, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  s->prev_valid = false;
  return e == cudaSuccess ? TETM_OK : rz_fail(e);
}

int tetm_rz_set_tiling(tetm_rz* s, int32_t chunk_z) {
  if (!s || chunk_z < 4 || chunk_z > (1 << 20)) return TETM_E_ARG;
  s->chunk_z = chunk_z;
  s->work_dirty = true;
  return rz_rebuild_work(s);
}

int tetm_rz_set_kernel(tetm_rz* s, int32_t kernel) {
  if (!s || (kernel != TETM_RZ_KERNEL_REGISTER && kernel != TETM_RZ_KERNEL_ASYNC &&
             kernel != TETM_RZ_KERNEL_BULK && kernel != TETM_RZ_KERNEL_BULK2))
    return TETM_E_ARG;
  if (s->mat && kernel != TETM_RZ_KERNEL_REGISTER) return TETM_E_UNSUPPORTED;  // per-plane coefficients
  const bool retile = (kernel == TETM_RZ_KERNEL_BULK2) != (s->kernel == TETM_RZ_KERNEL_BULK2);
  s->kernel = kernel;
  int rc = s->esz == 8 ? rz_occupancy<double>(s) : rz_occupancy<float>(s);
  if (rc == TETM_OK && retile) rc = rz_rebuild_work(s);
  return rc;
}

int tetm_rz_set_stream(tetm_rz* s, void* cuda_stream) {
  if (!s) return TETM_E_ARG;
  s->st = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : s->own;
  return TETM_OK;
}

int tetm_rz_check_guards(tetm_rz* s, int64_t* violations) {
  if (!s || !violations) return TETM_E_ARG;
  unsigned long long* cnt = nullptr;
  unsigned long long h = 0;
  cudaError_t e = cudaMalloc(&cnt, sizeof(*cnt));
  if (e != cudaSuccess) return rz_fail(e);
  e = cudaMemsetAsync(cnt, 0, sizeof(*cnt), s->st);
  const long long total = (long long)s->n_modes * s->L.mode_elems();
  for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
    if (s->esz == 8)
      rz_guard_scan<double><<<1024, 256, 0, s->st>>>(static_cast<const double*>(s->set[b]), s->mask, s->L, total, cnt);
    else
      rz_guard_scan<float><<<1024, 256, 0, s->st>>>(static_cast<const float*>(s->set[b]), s->mask, s->L, total, cnt);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  cudaFree(cnt);
  if (e != cudaSuccess) return rz_fail(e);
  *violations = (int64_t)h;
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
  info->kernel = s->kernel;
  return TETM_OK;
}

int tetm_rz_charge_residual(tetm_rz* s, int32_t mode, double* max_e, double* max_h, double* q_scale) {
  if (!rz_mode_ok(s, mode)) return TETM_E_ARG;
  if (!s->prev_valid || s->step < 1) return TETM_E_STATE;
  if (!s->rec1) {
    cudaError_t e = cudaMalloc(&s->rec1, sizeof(double) * (size_t)s->n_modes * kRzRec);
    if (e != cudaSuccess) return rz_fail(e);
  }
  const int rc = s->esz == 8 ? rz_queue_balances<double>(s, s->rec1) : rz_queue_balances<float>(s, s->rec1);
  if (rc) return rc;
  double h[kRzRec];
  cudaError_t e = cudaMemcpyAsync(h, s->rec1 + (size_t)mode * kRzRec, sizeof(h), cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return rz_fail(e);
  if (max_e) *max_e = h[3];
  if (max_h) *max_h = h[4];
  if (q_scale) *q_scale = h[5];
  return TETM_OK;
}

int tetm_rz_set_balance_every(tetm_rz* s, int32_t every) {
  if (!s || every < 0) return TETM_E_ARG;
  if (every > 0 && !s->hist) {
    const int cap = 1024;
    cudaError_t e = cudaMalloc(&s->hist, sizeof(double) * (size_t)cap * s->n_modes * kRzRec);
    if (e != cudaSuccess) return rz_fail(e);
    s->hist_cap = cap;
    s->device_bytes += (long long)(sizeof(double) * (size_t)cap * s->n_modes * kRzRec);
  }
  s->bal_every = every;
  return TETM_OK;
}

int tetm_rz_balance_history(tetm_rz* s, double* out, int32_t cap, int32_t* n_out) {
  if (!s) return TETM_E_ARG;
  const long long nrec = std::min<long long>(s->hist_count, s->hist_cap);
  const long long rows = nrec * s->n_modes;
  if (n_out) *n_out = (int32_t)rows;
  cudaError_t e = cudaSuccess;
  if (out && rows > 0) {
    if (cap < rows) return TETM_E_ARG;
    std::vector<double> h((size_t)s->hist_cap * s->n_modes * kRzRec);
    e = cudaMemcpyAsync(h.data(), s->hist, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) return rz_fail(e);
    const long long first = s->hist_count - nrec;
    const size_t rec = (size_t)s->n_modes * kRzRec;
    for (long long r = 0; r < nrec; ++r)
      memcpy(out + (size_t)r * rec, h.data() + (size_t)((first + r) % s->hist_cap) * rec, sizeof(double) * rec);
  } else {
    e = cudaStreamSynchronize(s->st);
  }
  return e == cudaSuccess ? TETM_OK : rz_fail(e);
}

namespace {
// Checkpoint of a rotationally symmetric solve: header, the current state of
// every mode in the device layout, then the wake accumulators (longitudinal
// and transverse, even and odd halves).
struct RzCkpt {
  char magic[8];
  int32_t nr, nz, m_lo, m_hi, precision, bunch, nw, obs, scattered, kernel_pairs;
  double dr, dz, cdt;
  int64_t step, kshift, elems;
};
size_t rz_ckpt_bytes(const tetm_rz* s) {
  return sizeof(RzCkpt) + rz_field_bytes(s->L, s->esz, s->n_modes) +
         (s->bunch ? 4 * sizeof(double) * (size_t)s->n_modes * s->nw : 0);
}
}  // namespace

int tetm_rz_save(tetm_rz* s, void* buf, size_t cap, size_t* used) {
  if (!s) return TETM_E_ARG;
  const size_t need = rz_ckpt_bytes(s);
  if (used) *used = need;
  if (!buf) return TETM_OK;
  if (cap < need) return TETM_E_ARG;
  RzCkpt h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, "TETMRZC1", 8);
  h.nr = s->g.nr; h.nz = s->g.nz; h.m_lo = s->g.m_lo; h.m_hi = s->g.m_hi; h.precision = s->g.precision;
  h.bunch = s->bunch; h.nw = s->bunch ? s->nw : 0; h.obs = s->obs; h.scattered = s->scattered;
  h.dr = s->g.dr; h.dz = s->g.dz; h.cdt = s->cdt;
  h.step = s->step; h.kshift = s->kshift;
  h.elems = (int64_t)s->n_modes * s->L.mode_elems();
  char* p = static_cast<char*>(buf);
  memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  const size_t fb = rz_field_bytes(s->L, s->esz, s->n_modes);
  cudaError_t e = cudaMemcpyAsync(p, s->set[s->cur], fb, cudaMemcpyDeviceToHost, s->st);
  p += fb;
  const size_t wb = 2 * sizeof(double) * (size_t)s->n_modes * s->nw;
  if (e == cudaSuccess && s->bunch) e = cudaMemcpyAsync(p, s->W, wb, cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess && s->bunch) e = cudaMemcpyAsync(p + wb, s->WT, wb, cudaMemcpyDeviceToHost, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  return e == cudaSuccess ? TETM_OK : rz_fail(e);
}

int tetm_rz_load(tetm_rz* s, const void* buf, size_t size) {
  if (!s || !buf || size < sizeof(RzCkpt)) return TETM_E_ARG;
  RzCkpt h;
  memcpy(&h, buf, sizeof(h));
  if (memcmp(h.magic, "TETMRZC1", 8) != 0 || h.nr != s->g.nr || h.nz != s->g.nz || h.m_lo != s->g.m_lo ||
      h.m_hi != s->g.m_hi || h.precision != s->g.precision || h.bunch != (int)s->bunch ||
      h.nw != (s->bunch ? s->nw : 0) || h.obs != s->obs || h.scattered != (int)s->scattered || h.dr != s->g.dr ||
      h.dz != s->g.dz || h.cdt != s->cdt || h.kshift != s->kshift ||
      h.elems != (int64_t)s->n_modes * s->L.mode_elems() || size < rz_ckpt_bytes(s))
    return TETM_E_ARG;
  const char* p = static_cast<const char*>(buf) + sizeof(h);
  const size_t fb = rz_field_bytes(s->L, s->esz, s->n_modes);
  cudaError_t e = cudaMemcpyAsync(s->set[s->cur], p, fb, cudaMemcpyHostToDevice, s->st);
  p += fb;
  const size_t wb = 2 * sizeof(double) * (size_t)s->n_modes * s->nw;
  if (e == cudaSuccess && s->bunch) e = cudaMemcpyAsync(s->W, p, wb, cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess && s->bunch) e = cudaMemcpyAsync(s->WT, p + wb, wb, cudaMemcpyHostToDevice, s->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
  if (e != cudaSuccess) return rz_fail(e);
  s->step = h.step;
  s->prev_valid = false;
  s->sc_until = 0;  // the scattered form's sources are recomputed from the loaded step on
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
  cudaFree(s->WT);
  cudaFree(s->partial);
  cudaFree(s->err);
  cudaFree(s->inc_prof);
  cudaFree(s->inc_G);
  cudaFree(s->S);
  cudaFree(s->differs);
  cudaFree(s->Jzero);
  cudaFree(s->hist);
  cudaFree(s->cpart);
  cudaFree(s->rec1);
  if (s->side) {
    cudaStreamSynchronize(s->side);
    cudaStreamDestroy(s->side);
  }
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  if (s->own) cudaStreamDestroy(s->own);
  cudaGetLastError();
  delete s;
  return TETM_OK;
}

}  // extern "C"
