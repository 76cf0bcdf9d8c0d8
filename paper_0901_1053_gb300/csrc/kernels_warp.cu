// Warp-tiled fused step of the explicit TE/TM scheme (Sec. 4.2, Eq. (23)).
//
// One warp owns a work item: a transverse tile of 28 x TY nodes and a chunk
// of z-planes. Its 32 lanes are 32 consecutive x-columns (2 halo columns on
// each side of the 28 it stores); inside a plane the warp sweeps the TY + 4
// rows of its tile (2 halo rows per side) in increasing y as a software
// pipeline:
//   row r: TM  U1 hx_a(r), U2 hy_a(r), U3 ez'(r) (+ bunch current),
//              U5 hy'(r), U4 hx'(r-1)
//          TE  U6 ex_a(r-1), U7 ey_a(r-1), U8 hz'(r-2), U9 ex'(r-2), U10 ey'(r-2)
// (the lags follow the y-stencil: hx' needs ez' one row up, hz' needs ex_a
// one row up, ex' needs hz' one row down). x-neighbours come from lane
// shuffles and y-neighbours from the previous rows' registers; the new hx, hy
// of a plane, which the TE stage of the next plane reads, stay per row in
// lane-private shared memory. No block barriers: warps are independent and
// persistent (each strides over the work items).
//
// Two variants differ in how the loads run ahead of the sweep (the row stream
// continues from the last row of a plane into the first of the next):
//   fused_step_warp      asynchronous copies (cp.async) into an 8-row
//                        shared-memory ring; used for float64, where deep
//                        prefetch without register cost pays;
//   fused_step_warp_reg  a 4-row register ring; fewer instructions per row,
//                        used for float32.
//
// As in the block-tiled kernel, the state is read from one field set and
// written to the other (y^n -> y^{n+1}), so a chunk starting at plane k0 also
// runs the TM stage of plane k0-1 (without storing it) for its first TE plane.
#include <algorithm>

#include "tetm_internal.h"

namespace tetm {
namespace {

constexpr int kWarpTileX = 28;  // stored columns per warp (32 lanes - 2*2 halo)

template <typename T>
__device__ __forceinline__ T shfl_dn(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }
template <typename T>
__device__ __forceinline__ T shfl_up1(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }


// Asynchronous copies into the warp's shared-memory ring (lane-private words:
// each lane copies and later reads only its own column, so no barrier is
// needed beyond the lane's own wait_group).
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int kDepth = 8;   // rows of loads in flight ahead of the sweep
constexpr int kArrs = 8;    // ez hx hy hz (plane k), ex ey (plane k), ex ey (plane k+1)

template <typename T, int TY>
__device__ __forceinline__ void fused_step_warp_item(const StepArgs<T>& a, int item,
                                                unsigned char* smem_raw) {

  constexpr int RH = TY + 4;
  static_assert(RH % kDepth == 0, "rows per tile must be a multiple of the ring depth");
  // per warp: the load ring [kDepth][kArrs][32] and the per-row state carried
  // to the next plane (new hx, hy of this plane) [2][RH][32]; the activity
  // bytes of the ring rows stay in registers
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  T* wbase = reinterpret_cast<T*>(smem_raw) + (size_t)wib * (kDepth * kArrs + 2 * RH) * 32;
  T* ring = wbase;
  T* sHXP = wbase + kDepth * kArrs * 32;
  T* sHYP = sHXP + RH * 32;

  const Layout L = a.L;
  const long long SZ = L.sz;
  const long long PX = L.px;
  const T* __restrict__ iex = a.in[kEX];
  const T* __restrict__ iey = a.in[kEY];
  const T* __restrict__ iez = a.in[kEZ];
  const T* __restrict__ ihx = a.in[kHX];
  const T* __restrict__ ihy = a.in[kHY];
  const T* __restrict__ ihz = a.in[kHZ];
  const uint8_t* __restrict__ msk = a.co.mask;
  T* __restrict__ oex = a.out[kEX];
  T* __restrict__ oey = a.out[kEY];
  T* __restrict__ oez = a.out[kEZ];
  T* __restrict__ ohx = a.out[kHX];
  T* __restrict__ ohy = a.out[kHY];
  T* __restrict__ ohz = a.out[kHZ];
  const T uEX = a.co.u[kEX], uEY = a.co.u[kEY], uEZ = a.co.u[kEZ];
  const T uHX = a.co.u[kHX], uHY = a.co.u[kHY], uHZ = a.co.u[kHZ];

  const int ntile = a.tiles_x * a.tiles_y;
  const int tile = item % ntile, chunk = item / ntile;
  const int gi = (tile % a.tiles_x) * kWarpTileX - 2 + lane;
  const int jbase = (tile / a.tiles_x) * TY - 2;
  const int ci = min(gi, L.nx + 1);
  const bool own_x = lane >= 2 && lane < kWarpTileX + 2 && gi < L.nx;
  const bool line_x = a.b.on && gi == a.b.i0;
  const int line_r = a.b.j0 - jbase;
  const int own_r_end = min(TY + 2, L.ny - jbase);
  const int k0 = chunk * a.chunk_z;
  const int k1 = min(k0 + a.chunk_z, L.nz);
  const int kstart = k0 - 1;

  auto index = [&](int k, int r) -> long long {
    const int j = min(jbase + r, L.ny + 1);
    return (long long)(k + 1) * SZ + (long long)(j + 2) * PX + (ci + L.ox);
  };
  // queue the loads of stream row g (plane kstart + g / RH, row g % RH) into
  // ring slot g % kDepth; returns its activity byte (a plain load)
  auto issue_row = [&](int g) -> uint8_t {
    const int k = kstart + g / RH, r = g % RH;
    const long long id = index(k, r);
    T* sl = ring + (g % kDepth) * kArrs * 32 + lane;
    if (sizeof(T) == 4) {
      cp_async4(sl + 0 * 32, iez + id);
      cp_async4(sl + 1 * 32, ihx + id);
      cp_async4(sl + 2 * 32, ihy + id);
      cp_async4(sl + 3 * 32, ihz + id);
      cp_async4(sl + 4 * 32, iex + id);
      cp_async4(sl + 5 * 32, iey + id);
      cp_async4(sl + 6 * 32, iex + id + SZ);
      cp_async4(sl + 7 * 32, iey + id + SZ);
    } else {
      cp_async8(sl + 0 * 32, iez + id);
      cp_async8(sl + 1 * 32, ihx + id);
      cp_async8(sl + 2 * 32, ihy + id);
      cp_async8(sl + 3 * 32, ihz + id);
      cp_async8(sl + 4 * 32, iex + id);
      cp_async8(sl + 5 * 32, iey + id);
      cp_async8(sl + 6 * 32, iex + id + SZ);
      cp_async8(sl + 7 * 32, iey + id + SZ);
    }
    cp_async_commit();
    return msk[id];
  };

  for (int r = 0; r < RH; ++r) {
    sHXP[r * 32 + lane] = T(0);
    sHYP[r * 32 + lane] = T(0);
  }
  uint8_t mring[kDepth];
#pragma unroll
  for (int q = 0; q < kDepth; ++q) mring[q] = issue_row(q);
  int g = 0;  // stream row being processed

  for (int k = kstart; k < k1; ++k) {
    const bool te = k >= k0;  // the first plane only feeds the TE stage of k0
    // pipeline registers (values of earlier rows of this plane)
    T hxa_p = T(0), dey_p = T(0), cHX_p = T(0), ezn_p = T(0);   // row r-1 (TM)
    T hyn_p = T(0), hyn_pp = T(0), hxn_pp = T(0);              // new hy rows r-1, r-2; new hx row r-2
    T hz_p = T(0), hz_pp = T(0);                               // old hz rows r-1, r-2
    uint8_t m_p = 0, m_pp = 0;
    unsigned mo_p = 0, mo_pp = 0;                              // the warp's OR of m, rows r-1, r-2
    T ex0_p = T(0), ey0_p = T(0);                              // old ex, ey row r-1
    T exa_pp = T(0), eya_pp = T(0), hzn_ppp = T(0);            // aux ex, ey row r-2; new hz row r-3
    T dhy_p = T(0), dhx_p = T(0);                              // z-differences of new hy, hx, row r-2
#pragma unroll 1
    for (int rg = 0; rg < RH; rg += kDepth) {
#pragma unroll
      for (int u = 0; u < kDepth; ++u) {
        const int r = rg + u;
        cp_async_wait<kDepth - 2>();  // rows g and g+1 have landed
        const T* sl = ring + u * kArrs * 32 + lane;
        const T ez = sl[0], hx = sl[32], hy = sl[64], hz = sl[96];
        const T ex0r = sl[128], ey0r = sl[160], ex1 = sl[192], ey1 = sl[224];
        const uint8_t m = mring[u];
        // which of this row's objects carry a field anywhere in the warp: an
        // update whose objects carry none in any lane leaves its zeros as
        // they are (coefficient zero), so the warp skips its arithmetic
        const unsigned mo = __reduce_or_sync(0xffffffffu, (unsigned)m);
        const T ez_next = ring[((u + 1) % kDepth) * kArrs * 32 + lane];  // row r+1
        mring[u] = issue_row(g + kDepth);  // refill this slot kDepth rows ahead
        ++g;

        const long long id = index(k, r);
        const bool own_r = r >= 2 && r < own_r_end;
        // ---------------- TM stage, row r ----------------
        const T cHX = (m & 8) ? uHX : T(0), cHY = (m & 16) ? uHY : T(0);
        const T cEZ = (m & 4) ? uEZ : T(0);
        const T dey = ey1 - ey0r, dex = ex1 - ex0r;
        const bool line = line_x && r == line_r;
        T hxa = hx, hya = hy, ezn = ez, hyn = hy;
        if (mo & (4 | 8 | 16)) {
          hxa = hx + cHX * (dey - (ez_next - ez));                                 // U1
          hya = hy + cHY * (-dex + (shfl_dn(ez) - ez));                            // U2
          T cur = (hxa_p - hxa) - (shfl_up1(hya) - hya);
          if (line) {
            const long long dd = (long long)k - (a.n + a.b.kshift) + a.b.c0;
            if (dd >= -a.b.c0 && dd < a.b.c0) cur -= a.b.J[dd + a.b.c0];
          }
          ezn = ez + cEZ * cur;                                                    // U3
          hyn = hya + cHY * (-dex + (shfl_dn(ezn) - ezn));                         // U5
        }
        T hxn_p = hxa_p;
        if (mo_p & 8) hxn_p = hxa_p + cHX_p * (dey_p - (ezn - ezn_p));             // U4, row r-1
        if (te && own_x) {
          if (own_r) {
            oez[id] = ezn;
            ohy[id] = hyn;
            if (line) {
              const long long mm = (a.n + a.b.kshift) - k - a.b.c0;
              if (mm >= a.b.m_min && mm <= a.b.m_max)
                a.b.W[mm - a.b.m_min] -= (double)ezn * a.b.inv_q;
            }
          }
          if (r - 1 >= 2 && r - 1 < own_r_end) ohx[id - PX] = hxn_p;
        }
        // ---------------- TE stage, rows q = r-1 and p = r-2 ----------------
        // (rows 0 and 1 are halo rows: their TE values are never used)
        const int q = r - 1, p = r - 2;
        T exa = ex0_p, eya = ey0_p, dhy = T(0), dhx = T(0);
        if (mo_p & 3) {
          const T hxq_old = q >= 0 ? sHXP[q * 32 + lane] : T(0);
          const T hyq_old = q >= 0 ? sHYP[q * 32 + lane] : T(0);
          const T cEX = (m_p & 1) ? uEX : T(0), cEY = (m_p & 2) ? uEY : T(0);
          dhy = hyq_old - hyn_p;  // U9 of this row (next row step) takes the same differences
          dhx = hxq_old - hxn_p;
          exa = ex0_p + cEX * (dhy - (hz_pp - hz_p));                              // U6, row q
          eya = ey0_p + cEY * (-dhx + (shfl_up1(hz_p) - hz_p));                    // U7, row q
        }
        T hzn = hz_pp;
        if (mo_pp & 32) {
          const T cHZ = (m_pp & 32) ? uHZ : T(0);
          hzn = hz_pp + cHZ * ((exa - exa_pp) - (shfl_dn(eya_pp) - eya_pp));       // U8, row p
        }
        T exn = exa_pp, eyn = eya_pp;
        if (mo_pp & 3) {
          const T cEXp = (m_pp & 1) ? uEX : T(0), cEYp = (m_pp & 2) ? uEY : T(0);
          exn = exa_pp + cEXp * (dhy_p - (hzn_ppp - hzn));                          // U9, row p
          eyn = eya_pp + cEYp * (-dhx_p + (shfl_up1(hzn) - hzn));                   // U10, row p
        }
        if (te && own_x && p >= 2 && p < own_r_end) {
          const long long idp = id - 2 * PX;
          oex[idp] = exn;
          oey[idp] = eyn;
          ohz[idp] = hzn;
        }
        if (p >= 0) {  // row p is done: keep its new hx, hy for the next plane
          sHXP[p * 32 + lane] = hxn_pp;
          sHYP[p * 32 + lane] = hyn_pp;
        }
        if (r == RH - 1) sHYP[q * 32 + lane] = hyn_p;  // last row whose new hy is read next plane
        // shift the pipeline
        hxn_pp = hxn_p;
        hyn_pp = hyn_p;
        hyn_p = hyn;
        hxa_p = hxa; dey_p = dey; cHX_p = cHX; ezn_p = ezn;
        hz_pp = hz_p; hz_p = hz;
        m_pp = m_p; m_p = m;
        mo_pp = mo_p; mo_p = mo;
        ex0_p = ex0r; ey0_p = ey0r;
        exa_pp = exa; eya_pp = eya; hzn_ppp = hzn;
        dhy_p = dhy; dhx_p = dhx;
      }
    }
  }
  cp_async_wait<0>();  // the ring is reused by the next work item
}

template <typename T, int TY>
__global__ void __launch_bounds__(64)
fused_step_warp(const StepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nitems = a.work ? a.n_work : a.tiles_x * a.tiles_y * a.n_chunks;
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int witem = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); witem < nitems;
       witem += nwarps)
    fused_step_warp_item<T, TY>(a, a.work ? a.work[witem] : witem, smem_raw);
}

// Batched form: one launch advances every active member of a batch by one
// step; the work list holds (member, item) pairs of all members.
template <typename T, int TY>
__global__ void __launch_bounds__(64)
fused_step_warp_batch(const BatchMember<T>* __restrict__ members,
                            const int2* __restrict__ work, const int* __restrict__ n_work_p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n_work = *n_work_p;
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int witem = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); witem < n_work;
       witem += nwarps) {
    const int2 e = work[witem];
    const BatchMember<T>& mb = members[e.x];
    if (!mb.active) continue;
    fused_step_warp_item<T, TY>(mb.a, e.y, smem_raw);
  }
}

template <typename T, int TY>
cudaError_t launch_warp_shape(const StepArgs<T>& a, cudaStream_t st) {
  const int items = a.work ? a.n_work : a.tiles_x * a.tiles_y * a.n_chunks;
  if (items <= 0) return cudaSuccess;
  const int warps_per_block = 2;
  const size_t smem = (size_t)warps_per_block * (kDepth * kArrs + 2 * (TY + 4)) * 32 * sizeof(T);
  // persistent grid: as many blocks as fit on the device at once (queried
  // once per instantiation), each warp striding over the work items
  static int resident = 0;
  if (!resident) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(fused_step_warp<T, TY>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_step_warp<T, TY>,
                                                        32 * warps_per_block, smem);
    if (e != cudaSuccess) return e;
    resident = std::max(1, sms * per_sm);
  }
  const int blocks = std::min(resident, (items + warps_per_block - 1) / warps_per_block);
  fused_step_warp<T, TY><<<blocks, 32 * warps_per_block, smem, st>>>(a);
  return cudaGetLastError();
}



// ---------------------------------------------------------------------------
// Register-ring variant (float32): the same sweep, with the loads of the next
// kRing rows held in registers (issued where they are written, so the
// scheduler cannot sink them) and the old ex, ey of the current plane kept
// as per-row state in shared memory. Fewer instructions per row than the
// asynchronous-copy ring; it wins where registers, not memory latency, set
// the pace (float32).
// ---------------------------------------------------------------------------
constexpr int kRing = 4;

__device__ __forceinline__ float ld_early(const float* p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ double ld_early(const double* p) {
  double v;
  asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint8_t ld_early(const uint8_t* p) {
  unsigned short v;
  asm volatile("ld.global.nc.u8 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
  return (uint8_t)v;
}

template <typename T>
struct RowIn {
  T ez, hx, hy, hz;  // plane k
  T ex1, ey1;        // plane k+1
  uint8_t m;         // activity bits, plane k
};

template <typename T, int TY>
__device__ __forceinline__ void fused_step_warp_reg_item(const StepArgs<T>& a, int item,
                                                unsigned char* smem_raw) {

  constexpr int RH = TY + 4;
  static_assert(RH % kRing == 0, "rows per tile must be a multiple of the ring depth");
  // per-row state carried from plane to plane, lane-private: old ex, ey of
  // the current plane and new hx, hy of the previous plane
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  T* st = reinterpret_cast<T*>(smem_raw) + (size_t)wib * 4 * RH * 32;
  T* sEX0 = st;
  T* sEY0 = st + RH * 32;
  T* sHXP = st + 2 * RH * 32;
  T* sHYP = st + 3 * RH * 32;

  const Layout L = a.L;
  const long long SZ = L.sz;
  const long long PX = L.px;
  const T* __restrict__ iex = a.in[kEX];
  const T* __restrict__ iey = a.in[kEY];
  const T* __restrict__ iez = a.in[kEZ];
  const T* __restrict__ ihx = a.in[kHX];
  const T* __restrict__ ihy = a.in[kHY];
  const T* __restrict__ ihz = a.in[kHZ];
  const uint8_t* __restrict__ msk = a.co.mask;
  T* __restrict__ oex = a.out[kEX];
  T* __restrict__ oey = a.out[kEY];
  T* __restrict__ oez = a.out[kEZ];
  T* __restrict__ ohx = a.out[kHX];
  T* __restrict__ ohy = a.out[kHY];
  T* __restrict__ ohz = a.out[kHZ];
  const T uEX = a.co.u[kEX], uEY = a.co.u[kEY], uEZ = a.co.u[kEZ];
  const T uHX = a.co.u[kHX], uHY = a.co.u[kHY], uHZ = a.co.u[kHZ];

  const int ntile = a.tiles_x * a.tiles_y;
  const int tile = item % ntile, chunk = item / ntile;
  const int gi = (tile % a.tiles_x) * kWarpTileX - 2 + lane;
  const int jbase = (tile / a.tiles_x) * TY - 2;
  const int ci = min(gi, L.nx + 1);
  const bool own_x = lane >= 2 && lane < kWarpTileX + 2 && gi < L.nx;
  const bool line_x = a.b.on && gi == a.b.i0;
  const int line_r = a.b.j0 - jbase;
  const int own_r_end = min(TY + 2, L.ny - jbase);
  const int k0 = chunk * a.chunk_z;
  const int k1 = min(k0 + a.chunk_z, L.nz);

  auto index = [&](int k, int r) -> long long {
    const int j = min(jbase + r, L.ny + 1);
    return (long long)(k + 1) * SZ + (long long)(j + 2) * PX + (ci + L.ox);
  };
  auto load_row = [&](int k, int r, RowIn<T>& d) {
    const long long id = index(k, r);
    d.ez = ld_early(iez + id); d.hx = ld_early(ihx + id); d.hy = ld_early(ihy + id);
    d.hz = ld_early(ihz + id); d.m = ld_early(msk + id);
    d.ex1 = ld_early(iex + id + SZ); d.ey1 = ld_early(iey + id + SZ);
  };

  const int kstart = k0 - 1;
  for (int r = 0; r < RH; ++r) {
    const long long id = index(kstart, r);
    sEX0[r * 32 + lane] = iex[id];
    sEY0[r * 32 + lane] = iey[id];
    sHXP[r * 32 + lane] = T(0);
    sHYP[r * 32 + lane] = T(0);
  }
  RowIn<T> ring[kRing];
#pragma unroll
  for (int r = 0; r < kRing; ++r) load_row(kstart, r, ring[r]);

  for (int k = kstart; k < k1; ++k) {
    const bool te = k >= k0;
    T hxa_p = T(0), dey_p = T(0), cHX_p = T(0), ezn_p = T(0);
    T hyn_p = T(0), hyn_pp = T(0), hxn_pp = T(0);
    T hz_p = T(0), hz_pp = T(0);
    uint8_t m_p = 0, m_pp = 0;
    T ex1_p = T(0), ey1_p = T(0);
    T exa_pp = T(0), eya_pp = T(0), hzn_ppp = T(0);
#pragma unroll 1
    for (int rg = 0; rg < RH; rg += kRing) {
#pragma unroll
      for (int u = 0; u < kRing; ++u) {
        const int r = rg + u;
        const RowIn<T> d = ring[u];
        const T ez_next = ring[(u + 1) % kRing].ez;  // row r+1 (garbage past the last row)
        if (r + kRing < RH) load_row(k, r + kRing, ring[u]);
        else load_row(k + 1, r + kRing - RH, ring[u]);

        const long long id = index(k, r);
        const bool own_r = r >= 2 && r < own_r_end;
        const T ex0r = sEX0[r * 32 + lane], ey0r = sEY0[r * 32 + lane];
        const T cHX = (d.m & 8) ? uHX : T(0), cHY = (d.m & 16) ? uHY : T(0);
        const T cEZ = (d.m & 4) ? uEZ : T(0);
        const T dey = d.ey1 - ey0r, dex = d.ex1 - ex0r;
        const T hxa = d.hx + cHX * (dey - (ez_next - d.ez));                    // U1
        const T hya = d.hy + cHY * (-dex + (shfl_dn(d.ez) - d.ez));              // U2
        T cur = (hxa_p - hxa) - (shfl_up1(hya) - hya);
        const bool line = line_x && r == line_r;
        if (line) {
          const long long dd = (long long)k - (a.n + a.b.kshift) + a.b.c0;
          if (dd >= -a.b.c0 && dd < a.b.c0) cur -= a.b.J[dd + a.b.c0];
        }
        const T ezn = d.ez + cEZ * cur;                                         // U3
        const T hyn = hya + cHY * (-dex + (shfl_dn(ezn) - ezn));                 // U5
        const T hxn_p = hxa_p + cHX_p * (dey_p - (ezn - ezn_p));                 // U4, row r-1
        if (te && own_x) {
          if (own_r) {
            oez[id] = ezn;
            ohy[id] = hyn;
            if (line) {
              const long long mm = (a.n + a.b.kshift) - k - a.b.c0;
              if (mm >= a.b.m_min && mm <= a.b.m_max)
                a.b.W[mm - a.b.m_min] -= (double)ezn * a.b.inv_q;
            }
          }
          if (r - 1 >= 2 && r - 1 < own_r_end) ohx[id - PX] = hxn_p;
        }
        const int q = r - 1, p = r - 2;
        const T hxq_old = q >= 0 ? sHXP[q * 32 + lane] : T(0);
        const T hyq_old = q >= 0 ? sHYP[q * 32 + lane] : T(0);
        const T exq0 = q >= 0 ? sEX0[q * 32 + lane] : T(0);
        const T eyq0 = q >= 0 ? sEY0[q * 32 + lane] : T(0);
        const T cEX = (m_p & 1) ? uEX : T(0), cEY = (m_p & 2) ? uEY : T(0);
        const T exa = exq0 + cEX * ((hyq_old - hyn_p) - (hz_pp - hz_p));            // U6, row q
        const T eya = eyq0 + cEY * (-(hxq_old - hxn_p) + (shfl_up1(hz_p) - hz_p));   // U7, row q
        const T cHZ = (m_pp & 32) ? uHZ : T(0);
        const T cEXp = (m_pp & 1) ? uEX : T(0), cEYp = (m_pp & 2) ? uEY : T(0);
        const T hzn = hz_pp + cHZ * ((exa - exa_pp) - (shfl_dn(eya_pp) - eya_pp));   // U8, row p
        const T hxp_old = p >= 0 ? sHXP[p * 32 + lane] : T(0);
        const T hyp_old = p >= 0 ? sHYP[p * 32 + lane] : T(0);
        const T exn = exa_pp + cEXp * ((hyp_old - hyn_pp) - (hzn_ppp - hzn));       // U9, row p
        const T eyn = eya_pp + cEYp * (-(hxp_old - hxn_pp) + (shfl_up1(hzn) - hzn));  // U10, row p
        if (te && own_x && p >= 2 && p < own_r_end) {
          const long long idp = id - 2 * PX;
          oex[idp] = exn;
          oey[idp] = eyn;
          ohz[idp] = hzn;
        }
        if (p >= 0) {
          sHXP[p * 32 + lane] = hxn_pp;
          sHYP[p * 32 + lane] = hyn_pp;
        }
        if (q >= 0) {
          sEX0[q * 32 + lane] = ex1_p;
          sEY0[q * 32 + lane] = ey1_p;
        }
        if (r == RH - 1) sHYP[q * 32 + lane] = hyn_p;
        hxn_pp = hxn_p;
        hyn_pp = hyn_p;
        hyn_p = hyn;
        hxa_p = hxa; dey_p = dey; cHX_p = cHX; ezn_p = ezn;
        hz_pp = hz_p; hz_p = d.hz;
        m_pp = m_p; m_p = d.m;
        ex1_p = d.ex1; ey1_p = d.ey1;
        exa_pp = exa; eya_pp = eya; hzn_ppp = hzn;
      }
    }
  }
}

template <typename T, int TY>
__global__ void __launch_bounds__(128)
fused_step_warp_reg(const StepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nitems = a.work ? a.n_work : a.tiles_x * a.tiles_y * a.n_chunks;
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int witem = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); witem < nitems;
       witem += nwarps)
    fused_step_warp_reg_item<T, TY>(a, a.work ? a.work[witem] : witem, smem_raw);
}

// Batched form: one launch advances every active member of a batch by one
// step; the work list holds (member, item) pairs of all members.
template <typename T, int TY>
__global__ void __launch_bounds__(128)
fused_step_warp_reg_batch(const BatchMember<T>* __restrict__ members,
                            const int2* __restrict__ work, const int* __restrict__ n_work_p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n_work = *n_work_p;
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int witem = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); witem < n_work;
       witem += nwarps) {
    const int2 e = work[witem];
    const BatchMember<T>& mb = members[e.x];
    if (!mb.active) continue;
    fused_step_warp_reg_item<T, TY>(mb.a, e.y, smem_raw);
  }
}

template <typename T, int TY>
cudaError_t launch_warp_reg_shape(const StepArgs<T>& a, cudaStream_t st) {
  const int items = a.work ? a.n_work : a.tiles_x * a.tiles_y * a.n_chunks;
  if (items <= 0) return cudaSuccess;
  const int warps_per_block = 4;
  const size_t smem = (size_t)warps_per_block * 4 * (TY + 4) * 32 * sizeof(T);
  static int resident = 0;
  if (!resident) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(fused_step_warp_reg<T, TY>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_step_warp_reg<T, TY>,
                                                        32 * warps_per_block, smem);
    if (e != cudaSuccess) return e;
    resident = std::max(1, sms * per_sm);
  }
  const int blocks = std::min(resident, (items + warps_per_block - 1) / warps_per_block);
  fused_step_warp_reg<T, TY><<<blocks, 32 * warps_per_block, smem, st>>>(a);
  return cudaGetLastError();
}


// After a batch step: every active member swaps its field sets, counts the
// step and retires when it reaches its limit.
template <typename T>
__global__ void batch_advance(BatchMember<T>* members, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !members[i].active) return;
  StepArgs<T>& a = members[i].a;
  for (int c = 0; c < 6; ++c) {
    T* t = a.out[c];
    a.out[c] = const_cast<T*>(a.in[c]);
    a.in[c] = t;
  }
  a.n += 1;
  members[i].cur ^= 1;
  if (a.n >= members[i].limit) members[i].active = 0;
}

template <typename T, int TY, bool ASYNC, typename K>
cudaError_t launch_batch_kernel(K kern, const BatchMember<T>* members, const int2* work, const int* n_work,
                                int n_bound, cudaStream_t st) {
  const int warps_per_block = ASYNC ? 2 : 4;
  const size_t smem = ASYNC ? (size_t)warps_per_block * (kDepth * kArrs + 2 * (TY + 4)) * 32 * sizeof(T)
                            : (size_t)warps_per_block * 4 * (TY + 4) * 32 * sizeof(T);
  static int resident = 0;
  if (!resident) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * warps_per_block, smem);
    if (e != cudaSuccess) return e;
    resident = std::max(1, sms * per_sm);
  }
  const int blocks = std::min(resident, (n_bound + warps_per_block - 1) / warps_per_block);
  if (blocks > 0) kern<<<blocks, 32 * warps_per_block, smem, st>>>(members, work, n_work);
  return cudaGetLastError();
}

template <typename T, int TY, bool ASYNC>
cudaError_t launch_batch_shape(const BatchMember<T>* members, const int2* work, const int* n_work,
                               int n_bound, cudaStream_t st) {
  if constexpr (ASYNC)
    return launch_batch_kernel<T, TY, true>(fused_step_warp_batch<T, TY>, members, work, n_work, n_bound, st);
  else
    return launch_batch_kernel<T, TY, false>(fused_step_warp_reg_batch<T, TY>, members, work, n_work, n_bound,
                                             st);
}


// ---------------------------------------------------------------------------
// General materials: the six update coefficients are per-entry arrays
// (alpha M^-1 and 2 alpha M^-1 of each edge and face, zero on PEC and outside
// the box) streamed through the asynchronous-copy ring with the fields, four
// rows ahead. Each row's TE coefficients are carried to the TE lags of the
// sweep. Same sweep and lags as fused_step_warp.
// ---------------------------------------------------------------------------
constexpr int kMatDepth = 4;
constexpr int kMatArrs = 14;  // 8 field entries as in kArrs, then u_ex u_ey u_ez u_hx u_hy u_hz

template <typename T, int TY>
__device__ __forceinline__ void fused_step_warp_mat_item(const StepArgs<T>& a, int item,
                                                         unsigned char* smem_raw) {
  constexpr int RH = TY + 4;
  static_assert(RH % kMatDepth == 0, "rows per tile must be a multiple of the ring depth");
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  T* wbase = reinterpret_cast<T*>(smem_raw) + (size_t)wib * (kMatDepth * kMatArrs + 2 * RH) * 32;
  T* ring = wbase;
  T* sHXP = wbase + kMatDepth * kMatArrs * 32;
  T* sHYP = sHXP + RH * 32;

  const Layout L = a.L;
  const long long SZ = L.sz;
  const long long PX = L.px;
  const T* __restrict__ iex = a.in[kEX];
  const T* __restrict__ iey = a.in[kEY];
  const T* __restrict__ iez = a.in[kEZ];
  const T* __restrict__ ihx = a.in[kHX];
  const T* __restrict__ ihy = a.in[kHY];
  const T* __restrict__ ihz = a.in[kHZ];
  T* __restrict__ oex = a.out[kEX];
  T* __restrict__ oey = a.out[kEY];
  T* __restrict__ oez = a.out[kEZ];
  T* __restrict__ ohx = a.out[kHX];
  T* __restrict__ ohy = a.out[kHY];
  T* __restrict__ ohz = a.out[kHZ];

  const int ntile = a.tiles_x * a.tiles_y;
  const int tile = item % ntile, chunk = item / ntile;
  const int gi = (tile % a.tiles_x) * kWarpTileX - 2 + lane;
  const int jbase = (tile / a.tiles_x) * TY - 2;
  const int ci = min(gi, L.nx + 1);
  const bool own_x = lane >= 2 && lane < kWarpTileX + 2 && gi < L.nx;
  const bool line_x = a.b.on && gi == a.b.i0;
  const int line_r = a.b.j0 - jbase;
  const int own_r_end = min(TY + 2, L.ny - jbase);
  const int k0 = chunk * a.chunk_z;
  const int k1 = min(k0 + a.chunk_z, L.nz);
  const int kstart = k0 - 1;

  auto index = [&](int k, int r) -> long long {
    const int j = min(jbase + r, L.ny + 1);
    return (long long)(k + 1) * SZ + (long long)(j + 2) * PX + (ci + L.ox);
  };
  auto issue_row = [&](int g) {
    const int k = kstart + g / RH, r = g % RH;
    const long long id = index(k, r);
    T* sl = ring + (g % kMatDepth) * kMatArrs * 32 + lane;
    const T* src[kMatArrs] = {iez + id, ihx + id, ihy + id, ihz + id, iex + id, iey + id,
                              iex + id + SZ, iey + id + SZ,
                              a.co.ua[kEX] + id, a.co.ua[kEY] + id, a.co.ua[kEZ] + id,
                              a.co.ua[kHX] + id, a.co.ua[kHY] + id, a.co.ua[kHZ] + id};
#pragma unroll
    for (int q = 0; q < kMatArrs; ++q) {
      if (sizeof(T) == 4) cp_async4(sl + q * 32, src[q]);
      else cp_async8(sl + q * 32, src[q]);
    }
    cp_async_commit();
  };

  for (int r = 0; r < RH; ++r) {
    sHXP[r * 32 + lane] = T(0);
    sHYP[r * 32 + lane] = T(0);
  }
#pragma unroll
  for (int q = 0; q < kMatDepth; ++q) issue_row(q);
  int g = 0;

  for (int k = kstart; k < k1; ++k) {
    const bool te = k >= k0;
    T hxa_p = T(0), dey_p = T(0), cHX_p = T(0), ezn_p = T(0);
    T hyn_p = T(0), hyn_pp = T(0), hxn_pp = T(0);
    T hz_p = T(0), hz_pp = T(0);
    T cEX_p = T(0), cEY_p = T(0), cHZ_p = T(0);     // TE coefficients of row r-1
    T cEX_pp = T(0), cEY_pp = T(0), cHZ_pp = T(0);  // ... and of row r-2
    T ex0_p = T(0), ey0_p = T(0);
    T exa_pp = T(0), eya_pp = T(0), hzn_ppp = T(0);
#pragma unroll 1
    for (int rg = 0; rg < RH; rg += kMatDepth) {
#pragma unroll
      for (int u = 0; u < kMatDepth; ++u) {
        const int r = rg + u;
        cp_async_wait<kMatDepth - 2>();  // rows g and g+1 have landed
        const T* sl = ring + u * kMatArrs * 32 + lane;
        const T ez = sl[0], hx = sl[32], hy = sl[64], hz = sl[96];
        const T ex0r = sl[128], ey0r = sl[160], ex1 = sl[192], ey1 = sl[224];
        const T cEX = sl[256], cEY = sl[288], cEZ = sl[320];
        const T cHX = sl[352], cHY = sl[384], cHZ = sl[416];
        const T ez_next = ring[((u + 1) % kMatDepth) * kMatArrs * 32 + lane];  // row r+1
        issue_row(g + kMatDepth);
        ++g;

        const long long id = index(k, r);
        const bool own_r = r >= 2 && r < own_r_end;
        // ---------------- TM stage, row r ----------------
        const T dey = ey1 - ey0r, dex = ex1 - ex0r;
        const T hxa = hx + cHX * (dey - (ez_next - ez));                         // U1
        const T hya = hy + cHY * (-dex + (shfl_dn(ez) - ez));                    // U2
        T cur = (hxa_p - hxa) - (shfl_up1(hya) - hya);
        const bool line = line_x && r == line_r;
        if (line) {
          const long long dd = (long long)k - (a.n + a.b.kshift) + a.b.c0;
          if (dd >= -a.b.c0 && dd < a.b.c0) cur -= a.b.J[dd + a.b.c0];
        }
        const T ezn = ez + cEZ * cur;                                            // U3
        const T hyn = hya + cHY * (-dex + (shfl_dn(ezn) - ezn));                 // U5
        const T hxn_p = hxa_p + cHX_p * (dey_p - (ezn - ezn_p));                 // U4, row r-1
        if (te && own_x) {
          if (own_r) {
            oez[id] = ezn;
            ohy[id] = hyn;
            if (line) {
              const long long mm = (a.n + a.b.kshift) - k - a.b.c0;
              if (mm >= a.b.m_min && mm <= a.b.m_max)
                a.b.W[mm - a.b.m_min] -= (double)ezn * a.b.inv_q;
            }
          }
          if (r - 1 >= 2 && r - 1 < own_r_end) ohx[id - PX] = hxn_p;
        }
        // ---------------- TE stage, rows q = r-1 and p = r-2 ----------------
        const int q = r - 1, p = r - 2;
        const T hxq_old = q >= 0 ? sHXP[q * 32 + lane] : T(0);
        const T hyq_old = q >= 0 ? sHYP[q * 32 + lane] : T(0);
        const T exa = ex0_p + cEX_p * ((hyq_old - hyn_p) - (hz_pp - hz_p));           // U6, row q
        const T eya = ey0_p + cEY_p * (-(hxq_old - hxn_p) + (shfl_up1(hz_p) - hz_p));  // U7, row q
        const T hzn = hz_pp + cHZ_pp * ((exa - exa_pp) - (shfl_dn(eya_pp) - eya_pp)); // U8, row p
        const T hxp_old = p >= 0 ? sHXP[p * 32 + lane] : T(0);
        const T hyp_old = p >= 0 ? sHYP[p * 32 + lane] : T(0);
        const T exn = exa_pp + cEX_pp * ((hyp_old - hyn_pp) - (hzn_ppp - hzn));     // U9, row p
        const T eyn = eya_pp + cEY_pp * (-(hxp_old - hxn_pp) + (shfl_up1(hzn) - hzn));  // U10, row p
        if (te && own_x && p >= 2 && p < own_r_end) {
          const long long idp = id - 2 * PX;
          oex[idp] = exn;
          oey[idp] = eyn;
          ohz[idp] = hzn;
        }
        if (p >= 0) {
          sHXP[p * 32 + lane] = hxn_pp;
          sHYP[p * 32 + lane] = hyn_pp;
        }
        if (r == RH - 1) sHYP[q * 32 + lane] = hyn_p;
        hxn_pp = hxn_p;
        hyn_pp = hyn_p;
        hyn_p = hyn;
        hxa_p = hxa; dey_p = dey; cHX_p = cHX; ezn_p = ezn;
        hz_pp = hz_p; hz_p = hz;
        cEX_pp = cEX_p; cEY_pp = cEY_p; cHZ_pp = cHZ_p;
        cEX_p = cEX; cEY_p = cEY; cHZ_p = cHZ;
        ex0_p = ex0r; ey0_p = ey0r;
        exa_pp = exa; eya_pp = eya; hzn_ppp = hzn;
      }
    }
  }
  cp_async_wait<0>();
}

template <typename T, int TY>
__global__ void __launch_bounds__(64)
fused_step_warp_mat(const StepArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nitems = a.work ? a.n_work : a.tiles_x * a.tiles_y * a.n_chunks;
  const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int witem = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); witem < nitems;
       witem += nwarps)
    fused_step_warp_mat_item<T, TY>(a, a.work ? a.work[witem] : witem, smem_raw);
}

template <typename T, int TY>
cudaError_t launch_warp_mat_shape(const StepArgs<T>& a, cudaStream_t st) {
  const int items = a.work ? a.n_work : a.tiles_x * a.tiles_y * a.n_chunks;
  if (items <= 0) return cudaSuccess;
  const int warps_per_block = 2;
  const size_t smem = (size_t)warps_per_block * (kMatDepth * kMatArrs + 2 * (TY + 4)) * 32 * sizeof(T);
  static int resident = 0;
  if (!resident) {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(fused_step_warp_mat<T, TY>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused_step_warp_mat<T, TY>,
                                                        32 * warps_per_block, smem);
    if (e != cudaSuccess) return e;
    resident = std::max(1, sms * per_sm);
  }
  const int blocks = std::min(resident, (items + warps_per_block - 1) / warps_per_block);
  fused_step_warp_mat<T, TY><<<blocks, 32 * warps_per_block, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool warp_shape_ok(int tx, int ty) {
  return tx == kWarpTileX && (ty == 4 || ty == 8 || ty == 12 || ty == 16 || ty == 20 || ty == 28);
}

// float32: register ring (any tile height above); float64: asynchronous-copy
// ring (tile heights 4, 12, 20, 28; 8 and 16 fall back to the register ring)
template <typename T>
cudaError_t launch_fused_warp_step(const StepArgs<T>& a, int tx, int ty, cudaStream_t st) {
  if (tx != kWarpTileX) return cudaErrorInvalidValue;
  if (a.co.ua[0]) {  // per-entry coefficient arrays (general materials)
    if (ty == 4) return launch_warp_mat_shape<T, 4>(a, st);
    if (ty == 8) return launch_warp_mat_shape<T, 8>(a, st);
    if (ty == 12) return launch_warp_mat_shape<T, 12>(a, st);
    if (ty == 16) return launch_warp_mat_shape<T, 16>(a, st);
    if (ty == 20) return launch_warp_mat_shape<T, 20>(a, st);
    if (ty == 28) return launch_warp_mat_shape<T, 28>(a, st);
    return cudaErrorInvalidValue;
  }
  if constexpr (sizeof(T) == 8) {
    if (ty == 4) return launch_warp_shape<T, 4>(a, st);
    if (ty == 12) return launch_warp_shape<T, 12>(a, st);
    if (ty == 20) return launch_warp_shape<T, 20>(a, st);
    if (ty == 28) return launch_warp_shape<T, 28>(a, st);
  }
  if (ty == 4) return launch_warp_reg_shape<T, 4>(a, st);
  if (ty == 8) return launch_warp_reg_shape<T, 8>(a, st);
  if (ty == 12) return launch_warp_reg_shape<T, 12>(a, st);
  if (ty == 16) return launch_warp_reg_shape<T, 16>(a, st);
  if (ty == 20) return launch_warp_reg_shape<T, 20>(a, st);
  if (ty == 28) return launch_warp_reg_shape<T, 28>(a, st);
  return cudaErrorInvalidValue;
}


template <typename T>
cudaError_t launch_fused_warp_batch(const BatchMember<T>* members, int n_members, const int2* work,
                                    const int* n_work, int n_bound, int ty, int nz_max, cudaStream_t st) {
  cudaError_t e = cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 8) {
    if (ty == 4) e = launch_batch_shape<T, 4, true>(members, work, n_work, n_bound, st);
    else if (ty == 12) e = launch_batch_shape<T, 12, true>(members, work, n_work, n_bound, st);
    else if (ty == 20) e = launch_batch_shape<T, 20, true>(members, work, n_work, n_bound, st);
    else if (ty == 28) e = launch_batch_shape<T, 28, true>(members, work, n_work, n_bound, st);
    else if (ty == 8) e = launch_batch_shape<T, 8, false>(members, work, n_work, n_bound, st);
    else if (ty == 16) e = launch_batch_shape<T, 16, false>(members, work, n_work, n_bound, st);
  } else {
    if (ty == 4) e = launch_batch_shape<T, 4, false>(members, work, n_work, n_bound, st);
    else if (ty == 8) e = launch_batch_shape<T, 8, false>(members, work, n_work, n_bound, st);
    else if (ty == 12) e = launch_batch_shape<T, 12, false>(members, work, n_work, n_bound, st);
    else if (ty == 16) e = launch_batch_shape<T, 16, false>(members, work, n_work, n_bound, st);
    else if (ty == 20) e = launch_batch_shape<T, 20, false>(members, work, n_work, n_bound, st);
    else if (ty == 28) e = launch_batch_shape<T, 28, false>(members, work, n_work, n_bound, st);
  }
  if (e != cudaSuccess) return e;
  e = launch_transverse_after_batch_step<T>(members, n_members, nz_max, st);
  if (e != cudaSuccess) return e;
  batch_advance<T><<<(n_members + 127) / 128, 128, 0, st>>>(const_cast<BatchMember<T>*>(members),
                                                            n_members);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_batch_advance(BatchMember<T>* members, int n_members, cudaStream_t st) {
  batch_advance<T><<<(n_members + 127) / 128, 128, 0, st>>>(members, n_members);
  return cudaGetLastError();
}
template cudaError_t launch_batch_advance<float>(BatchMember<float>*, int, cudaStream_t);
template cudaError_t launch_batch_advance<double>(BatchMember<double>*, int, cudaStream_t);

template cudaError_t launch_fused_warp_batch<float>(const BatchMember<float>*, int, const int2*, const int*,
                                                    int, int, int, cudaStream_t);
template cudaError_t launch_fused_warp_batch<double>(const BatchMember<double>*, int, const int2*, const int*,
                                                     int, int, int, cudaStream_t);

template cudaError_t launch_fused_warp_step<float>(const StepArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_fused_warp_step<double>(const StepArgs<double>&, int, int, cudaStream_t);

}  // namespace tetm
