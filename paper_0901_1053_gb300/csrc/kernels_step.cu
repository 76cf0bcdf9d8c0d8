// Update kernels of the explicit TE/TM scheme, Sec. 4.2, Eq. (23).
//
// Reference path: one launch per update equation (10 per step), each thread
// updating one entry in place, in the paper's order
//   TM: U1 hx, U2 hy, U3 ez (+ bunch current, + wake sample), U4 hx, U5 hy
//   TE: U6 ex, U7 ey, U8 hz, U9 ex, U10 ey.
// Every update writes one component from the others at the same time level,
// so each launch is race-free in place.
//
// Fused path: one launch per step. Each block owns a transverse tile of
// TX x TY nodes and a chunk of z-planes and marches through the planes in
// increasing k, doing the TM stage at plane k and then the TE stage at plane
// k (the TE stage at k needs the new hx, hy at planes k-1 and k; the TM stage
// at k needs the old ex, ey at k and k+1). The transverse chain
// hx,hy -> ez -> hx,hy -> ex,ey -> hz -> ex,ey reaches two nodes sideways,
// so each block also computes a 2-node halo ring (recomputed, not exchanged).
// The state is ping-ponged between two field sets (read y^n, write y^{n+1}),
// which makes blocks independent: no block reads what another writes in the
// same launch. A chunk starting at plane k0 recomputes the TM stage of plane
// k0-1 (without storing it) for its first TE plane.
#include <algorithm>

#include "tetm_internal.h"

namespace tetm {

namespace {

template <typename T>
__device__ __forceinline__ T coef_of(const Coefs<T>& co, int c, uint8_t m, long long id) {
  if (co.ua[c]) return co.ua[c][id];
  return ((m >> c) & 1) ? co.u[c] : T(0);
}

// ---------------------------------------------------------------------------
// Reference kernels
// ---------------------------------------------------------------------------

// Transverse wake of the reference path, between U5 and U6: e_x, e_y still
// of time n, h_x, h_y already of time n+1/2; one thread per plane.
template <typename T>
__global__ void ref_transverse_gather(StepArgs<T> a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (!a.b.obs_on || k >= a.L.nz) return;
  const long long id = a.L.idx(a.b.obs_i, a.b.obs_j, k);
  gather_wx(a.b, a.n, k, a.out[kEX][id], a.out[kHY][id]);
  gather_wy(a.b, a.n, k, a.out[kEY][id], a.out[kHX][id]);
}

}  // namespace

// Transverse wake of a ping-pong step: after the step the input set still
// holds e_x, e_y of time n and the output set h_x, h_y of time n+1/2, so one
// small launch gathers the observer column and the step kernels carry no
// extra registers for it. Threads stride over the planes.
template <typename T>
__device__ __forceinline__ void transverse_of_step(const StepArgs<T>& a, int k) {
  const long long id = a.L.idx(a.b.obs_i, a.b.obs_j, k);
  gather_wx(a.b, a.n, k, a.in[kEX][id], a.out[kHY][id]);
  gather_wy(a.b, a.n, k, a.in[kEY][id], a.out[kHX][id]);
}

template <typename T>
__global__ void transverse_after_step(StepArgs<T> a) {
  if (!a.b.obs_on) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < a.L.nz; k += gridDim.x * blockDim.x)
    transverse_of_step(a, k);
}

template <typename T>
__global__ void transverse_after_batch_step(const BatchMember<T>* members) {
  const BatchMember<T>& mb = members[blockIdx.y];
  if (!mb.active || !mb.a.b.obs_on) return;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < mb.a.L.nz; k += gridDim.x * blockDim.x)
    transverse_of_step(mb.a, k);
}

template <typename T>
cudaError_t launch_transverse_after_step(const StepArgs<T>& a, cudaStream_t st) {
  const int blocks = std::min(64, (a.L.nz + 127) / 128);
  transverse_after_step<T><<<blocks, 128, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_transverse_after_batch_step(const BatchMember<T>* members, int n_members, int nz_max,
                                               cudaStream_t st) {
  if (n_members <= 0 || nz_max <= 0) return cudaSuccess;  // no member gathers a transverse wake
  const dim3 grid(std::min(16, (nz_max + 127) / 128), n_members);
  transverse_after_batch_step<T><<<grid, 128, 0, st>>>(members);
  return cudaGetLastError();
}

template cudaError_t launch_transverse_after_step<float>(const StepArgs<float>&, cudaStream_t);
template cudaError_t launch_transverse_after_step<double>(const StepArgs<double>&, cudaStream_t);
template cudaError_t launch_transverse_after_batch_step<float>(const BatchMember<float>*, int, int,
                                                                cudaStream_t);
template cudaError_t launch_transverse_after_batch_step<double>(const BatchMember<double>*, int, int,
                                                                 cudaStream_t);

namespace {

template <typename T, int C>
__global__ void ref_update(StepArgs<T> a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= a.L.nx || j >= a.L.ny) return;  // entries with index nx, ny, nz never carry a field
  const long long id = a.L.idx(i, j, k);
  const long long sx = 1, sy = a.L.px, sz = a.L.sz;
  const uint8_t m = a.co.mask[id];
  const T c = coef_of(a.co, C, m, id);
  if (c == T(0)) return;
  T* const* F = a.out;
  const T* ex = F[kEX];
  const T* ey = F[kEY];
  const T* ez = F[kEZ];
  const T* hx = F[kHX];
  const T* hy = F[kHY];
  const T* hz = F[kHZ];
  if (C == kHX) {         // U1 / U4: hx += a M^-1 (P_z ey - P_y ez)
    F[kHX][id] = hx[id] + c * ((ey[id + sz] - ey[id]) - (ez[id + sy] - ez[id]));
  } else if (C == kHY) {  // U2 / U5: hy += a M^-1 (-P_z ex + P_x ez)
    F[kHY][id] = hy[id] + c * (-(ex[id + sz] - ex[id]) + (ez[id + sx] - ez[id]));
  } else if (C == kEZ) {  // U3: ez += 2a M^-1 (P_y^T hx - P_x^T hy - jj_z^n)
    T cur = (hx[id - sy] - hx[id]) - (hy[id - sx] - hy[id]);
    const bool line = a.b.on && i == a.b.i0 && j == a.b.j0;
    if (line) {
      const long long d = (long long)k - (a.n + a.b.kshift) + a.b.c0;
      if (d >= -a.b.c0 && d < a.b.c0) cur -= a.b.J[d + a.b.c0];
    }
    const T ezn = ez[id] + c * cur;
    F[kEZ][id] = ezn;
    if (line) {  // wake sample: W(s_m) -= ez^{n+1/2}(k) / Q with m = n - k - c0
      const long long mm = (a.n + a.b.kshift) - k - a.b.c0;
      if (mm >= a.b.m_min && mm <= a.b.m_max) a.b.W[mm - a.b.m_min] -= (double)ezn * a.b.inv_q;
    }
  } else if (C == kEX) {  // U6 / U9: ex += a M^-1 (P_z^T hy - P_y^T hz)
    F[kEX][id] = ex[id] + c * ((hy[id - sz] - hy[id]) - (hz[id - sy] - hz[id]));
  } else if (C == kEY) {  // U7 / U10: ey += a M^-1 (-P_z^T hx + P_x^T hz)
    F[kEY][id] = ey[id] + c * (-(hx[id - sz] - hx[id]) + (hz[id - sx] - hz[id]));
  } else {                // U8: hz += 2a M^-1 (P_y ex - P_x ey)
    F[kHZ][id] = hz[id] + c * ((ex[id + sy] - ex[id]) - (ey[id + sx] - ey[id]));
  }
}

// ---------------------------------------------------------------------------
// Fused z-marching kernel
// ---------------------------------------------------------------------------
template <typename T, int TX, int TY>
__global__ void __launch_bounds__((TX + 4) * (TY + 4))
fused_step(const StepArgs<T> a) {
  constexpr int WX = TX + 4, WY = TY + 4;  // thread columns: tile + halo of 2 per side
  constexpr int SX = WX + 2, SY = WY + 2;  // shared planes with a zero border of 1
  // Five exchange planes, reused through the step (hazards separated by barriers):
  //   A: old ez   B: old hz   C: hx aux / ex aux   D: hy aux / ey aux   E: new ez / new hz
  __shared__ T sA[SY][SX], sB[SY][SX], sC[SY][SX], sD[SY][SX], sE[SY][SX];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * WX + tx;
  for (int q = tid; q < SX * SY; q += WX * WY) {
    (&sA[0][0])[q] = T(0); (&sB[0][0])[q] = T(0); (&sC[0][0])[q] = T(0);
    (&sD[0][0])[q] = T(0); (&sE[0][0])[q] = T(0);
  }

  const int item = a.work ? a.work[blockIdx.x] : (int)blockIdx.x;
  const int ntile = a.tiles_x * a.tiles_y;
  const int tile = item % ntile, chunk = item / ntile;
  const int gi = (tile % a.tiles_x) * TX - 2 + tx;
  const int gj = (tile / a.tiles_x) * TY - 2 + ty;
  const Layout L = a.L;
  const int ci = min(max(gi, -2), L.nx + 1);
  const int cj = min(max(gj, -2), L.ny + 1);
  const bool own = tx >= 2 && tx < TX + 2 && ty >= 2 && ty < TY + 2 && gi < L.nx && gj < L.ny;
  const bool line = a.b.on && gi == a.b.i0 && gj == a.b.j0;
  const int k0 = chunk * a.chunk_z;
  const int k1 = min(k0 + a.chunk_z, L.nz);
  const long long SZ = L.sz;
  const int sx = tx + 1, sy = ty + 1;

  const T* __restrict__ iex = a.in[kEX];
  const T* __restrict__ iey = a.in[kEY];
  const T* __restrict__ iez = a.in[kEZ];
  const T* __restrict__ ihx = a.in[kHX];
  const T* __restrict__ ihy = a.in[kHY];
  const T* __restrict__ ihz = a.in[kHZ];
  const uint8_t* __restrict__ msk = a.co.mask;
  const T uEX = a.co.u[kEX], uEY = a.co.u[kEY], uEZ = a.co.u[kEZ];
  const T uHX = a.co.u[kHX], uHY = a.co.u[kHY], uHZ = a.co.u[kHZ];

  long long id = L.idx(ci, cj, k0 - 1);
  // plane k0-1 inputs of the TM stage, and ex, ey of plane k0
  T ex0 = iex[id], ey0 = iey[id];
  T ex1 = iex[id + SZ], ey1 = iey[id + SZ];
  T ez = iez[id], hx = ihx[id], hy = ihy[id], hz = T(0);
  uint8_t m = msk[id];
  T hxp = T(0), hyp = T(0);
  __syncthreads();

  for (int k = k0 - 1; k < k1; ++k, id += SZ) {
    // prefetch plane k+1 (and ex, ey of plane k+2) for the next iteration
    const T nez = iez[id + SZ], nhx = ihx[id + SZ], nhy = ihy[id + SZ], nhz = ihz[id + SZ];
    const uint8_t nm = msk[id + SZ];
    const T nex = iex[id + 2 * SZ], ney = iey[id + 2 * SZ];

    const T cHX = (m & 8) ? uHX : T(0), cHY = (m & 16) ? uHY : T(0), cEZ = (m & 4) ? uEZ : T(0);
    // ---- TM stage at plane k (time n-1/2 -> n+1/2) ----
    sA[sy][sx] = ez;
    sB[sy][sx] = hz;
    __syncthreads();
    const T dey = ey1 - ey0, dex = ex1 - ex0;
    const T hxa = hx + cHX * (dey - (sA[sy + 1][sx] - ez));   // U1
    const T hya = hy + cHY * (-dex + (sA[sy][sx + 1] - ez));  // U2
    sC[sy][sx] = hxa;
    sD[sy][sx] = hya;
    __syncthreads();
    T cur = (sC[sy - 1][sx] - hxa) - (sD[sy][sx - 1] - hya);
    if (line) {
      const long long d = (long long)k - (a.n + a.b.kshift) + a.b.c0;
      if (d >= -a.b.c0 && d < a.b.c0) cur -= a.b.J[d + a.b.c0];
    }
    const T ezn = ez + cEZ * cur;                               // U3
    sE[sy][sx] = ezn;
    __syncthreads();
    const T hxn = hxa + cHX * (dey - (sE[sy + 1][sx] - ezn));  // U4
    const T hyn = hya + cHY * (-dex + (sE[sy][sx + 1] - ezn)); // U5
    if (k >= k0) {
      if (own) {
        a.out[kHX][id] = hxn;
        a.out[kHY][id] = hyn;
        a.out[kEZ][id] = ezn;
        if (line) {
          const long long mm = (a.n + a.b.kshift) - k - a.b.c0;
          if (mm >= a.b.m_min && mm <= a.b.m_max) a.b.W[mm - a.b.m_min] -= (double)ezn * a.b.inv_q;
        }
      }
      // ---- TE stage at plane k (time n -> n+1) ----
      const T cEX = (m & 1) ? uEX : T(0), cEY = (m & 2) ? uEY : T(0), cHZ = (m & 32) ? uHZ : T(0);
      const T dhy = hyp - hyn, dhx = hxp - hxn;
      const T exa = ex0 + cEX * (dhy - (sB[sy - 1][sx] - hz));    // U6
      const T eya = ey0 + cEY * (-dhx + (sB[sy][sx - 1] - hz));   // U7
      sC[sy][sx] = exa;
      sD[sy][sx] = eya;
      __syncthreads();
      const T hzn = hz + cHZ * ((sC[sy + 1][sx] - exa) - (sD[sy][sx + 1] - eya));  // U8
      sE[sy][sx] = hzn;
      __syncthreads();
      const T exn = exa + cEX * (dhy - (sE[sy - 1][sx] - hzn));   // U9
      const T eyn = eya + cEY * (-dhx + (sE[sy][sx - 1] - hzn));  // U10
      if (own) {
        a.out[kEX][id] = exn;
        a.out[kEY][id] = eyn;
        a.out[kHZ][id] = hzn;
      }
    }
    hxp = hxn;
    hyp = hyn;
    ex0 = ex1; ey0 = ey1; ex1 = nex; ey1 = ney;
    ez = nez; hx = nhx; hy = nhy; hz = nhz; m = nm;
  }
}

// ---------------------------------------------------------------------------
// Two steps per pass (temporal blocking): y^n is read once and y^{n+2}
// written once per two steps. Same block-tiled sweep and arithmetic as
// fused_step, with a halo of four nodes per side: the first step is valid on
// the inner (TX+4) x (TY+4) nodes, the second, which rides one plane behind
// it and reads its results from registers and the exchange planes, on the
// owned TX x TY. A chunk [k0, k1) computes the first step's TM stage from
// plane k0-2 and its TE stage from k0-1 up to k1, the second step's TM stage
// from k0-1 and its TE stage on [k0, k1). Both steps deposit their bunch
// current in their halo computations too; each adds its wake samples for its
// owned nodes and planes with an atomic add (the second step of one chunk and
// the first step of the next may add to the same sample).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T ld_plane(const T* __restrict__ p, long long id, bool ok) {
  return ok ? p[id] : T(0);
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__((TX + 8) * (TY + 8))
fused_step2(const StepArgs<T> a) {
  constexpr int WX = TX + 8, WY = TY + 8;  // thread columns: tile + halo of 4 per side
  constexpr int SX = WX + 2, SY = WY + 2;  // shared planes with a zero border of 1
  __shared__ T sA[SY][SX], sB[SY][SX], sC[SY][SX], sD[SY][SX], sE[SY][SX];

  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * WX + tx;
  for (int q = tid; q < SX * SY; q += WX * WY) {
    (&sA[0][0])[q] = T(0); (&sB[0][0])[q] = T(0); (&sC[0][0])[q] = T(0);
    (&sD[0][0])[q] = T(0); (&sE[0][0])[q] = T(0);
  }

  const int item = a.work ? a.work[blockIdx.x] : (int)blockIdx.x;
  const int ntile = a.tiles_x * a.tiles_y;
  const int tile = item % ntile, chunk = item / ntile;
  const int gi = (tile % a.tiles_x) * TX - 4 + tx;
  const int gj = (tile / a.tiles_x) * TY - 4 + ty;
  const Layout L = a.L;
  const int ci = min(max(gi, -2), L.nx + 1);
  const int cj = min(max(gj, -2), L.ny + 1);
  const bool own = tx >= 4 && tx < TX + 4 && ty >= 4 && ty < TY + 4 && gi < L.nx && gj < L.ny;
  const bool line = a.b.on && gi == a.b.i0 && gj == a.b.j0;
  const int k0 = chunk * a.chunk_z;
  const int k1 = min(k0 + a.chunk_z, L.nz);
  const long long SZ = L.sz;
  const int sx = tx + 1, sy = ty + 1;

  const T* __restrict__ iex = a.in[kEX];
  const T* __restrict__ iey = a.in[kEY];
  const T* __restrict__ iez = a.in[kEZ];
  const T* __restrict__ ihx = a.in[kHX];
  const T* __restrict__ ihy = a.in[kHY];
  const T* __restrict__ ihz = a.in[kHZ];
  const uint8_t* __restrict__ msk = a.co.mask;
  const T uEX = a.co.u[kEX], uEY = a.co.u[kEY], uEZ = a.co.u[kEZ];
  const T uHX = a.co.u[kHX], uHY = a.co.u[kHY], uHZ = a.co.u[kHZ];

  // planes -1 .. nz+1 exist in the layout (the outer ones are zero guards);
  // the pass reaches from k0-2 to k1+2, so planes beyond read as zero
  auto plane_ok = [&](int k) { return k >= -1 && k <= L.nz + 1; };
  const int ks = k0 - 2;
  long long id = ((long long)(ks + 1) * (L.ny + 4) + (cj + 2)) * L.px + (ci + L.ox);
  // first-step inputs of plane ks (and e_x, e_y of plane ks+1)
  T ex0a = ld_plane(iex, id, plane_ok(ks)), ey0a = ld_plane(iey, id, plane_ok(ks));
  T ex0b = ld_plane(iex, id + SZ, plane_ok(ks + 1)), ey0b = ld_plane(iey, id + SZ, plane_ok(ks + 1));
  T ez0 = ld_plane(iez, id, plane_ok(ks)), hx0 = ld_plane(ihx, id, plane_ok(ks));
  T hy0 = ld_plane(ihy, id, plane_ok(ks)), hz0 = ld_plane(ihz, id, plane_ok(ks));
  uint8_t m0 = plane_ok(ks) ? msk[id] : (uint8_t)0;
  // carried: first-step results of the plane below (all six components and
  // its activity byte), second-step h_x, h_y of the plane below that
  T hx1p = T(0), hy1p = T(0), ez1p = T(0), ex1p = T(0), ey1p = T(0), hz1p = T(0);
  uint8_t mp = 0;
  T hx2p = T(0), hy2p = T(0);
  __syncthreads();

  for (int k = ks; k <= k1; ++k, id += SZ) {
    const bool okn = plane_ok(k + 1), okn2 = plane_ok(k + 2);
    const T nez = ld_plane(iez, id + SZ, okn), nhx = ld_plane(ihx, id + SZ, okn);
    const T nhy = ld_plane(ihy, id + SZ, okn), nhz = ld_plane(ihz, id + SZ, okn);
    const uint8_t nm = okn ? msk[id + SZ] : (uint8_t)0;
    const T nex = ld_plane(iex, id + 2 * SZ, okn2), ney = ld_plane(iey, id + 2 * SZ, okn2);

    // ======== first step (time n -> n+1) at plane k ========
    const T cHX = (m0 & 8) ? uHX : T(0), cHY = (m0 & 16) ? uHY : T(0), cEZ = (m0 & 4) ? uEZ : T(0);
    sA[sy][sx] = ez0;
    sB[sy][sx] = hz0;
    __syncthreads();
    const T dey = ey0b - ey0a, dex = ex0b - ex0a;
    const T hxa = hx0 + cHX * (dey - (sA[sy + 1][sx] - ez0));   // U1
    const T hya = hy0 + cHY * (-dex + (sA[sy][sx + 1] - ez0));  // U2
    sC[sy][sx] = hxa;
    sD[sy][sx] = hya;
    __syncthreads();
    T cur = (sC[sy - 1][sx] - hxa) - (sD[sy][sx - 1] - hya);
    if (line) {
      const long long d = (long long)k - (a.n + a.b.kshift) + a.b.c0;
      if (d >= -a.b.c0 && d < a.b.c0) cur -= a.b.J[d + a.b.c0];
    }
    const T ez1 = ez0 + cEZ * cur;                               // U3
    sE[sy][sx] = ez1;
    __syncthreads();
    const T hx1 = hxa + cHX * (dey - (sE[sy + 1][sx] - ez1));   // U4
    const T hy1 = hya + cHY * (-dex + (sE[sy][sx + 1] - ez1));  // U5
    if (own && line && k >= k0 && k < k1) {
      const long long mm = (a.n + a.b.kshift) - k - a.b.c0;
      if (mm >= a.b.m_min && mm <= a.b.m_max) atomicAdd(a.b.W + (mm - a.b.m_min), -(double)ez1 * a.b.inv_q);
    }
    T ex1 = T(0), ey1 = T(0), hz1 = T(0);
    if (k >= k0 - 1) {
      const T cEX = (m0 & 1) ? uEX : T(0), cEY = (m0 & 2) ? uEY : T(0), cHZ = (m0 & 32) ? uHZ : T(0);
      const T dhy = hy1p - hy1, dhx = hx1p - hx1;
      const T exa = ex0a + cEX * (dhy - (sB[sy - 1][sx] - hz0));    // U6
      const T eya = ey0a + cEY * (-dhx + (sB[sy][sx - 1] - hz0));   // U7
      __syncthreads();  // the TM stage's reads of sC, sD are done
      sC[sy][sx] = exa;
      sD[sy][sx] = eya;
      __syncthreads();
      hz1 = hz0 + cHZ * ((sC[sy + 1][sx] - exa) - (sD[sy][sx + 1] - eya));  // U8
      __syncthreads();  // the TM stage's reads of sE are done
      sE[sy][sx] = hz1;
      __syncthreads();
      ex1 = exa + cEX * (dhy - (sE[sy - 1][sx] - hz1));   // U9
      ey1 = eya + cEY * (-dhx + (sE[sy][sx - 1] - hz1));  // U10
    }

    // ======== second step (time n+1 -> n+2) at plane p = k-1 ========
    if (k >= k0) {
      const int p = k - 1;
      const T cHX2 = (mp & 8) ? uHX : T(0), cHY2 = (mp & 16) ? uHY : T(0), cEZ2 = (mp & 4) ? uEZ : T(0);
      __syncthreads();  // the first step's reads of every exchange plane are done
      sA[sy][sx] = ez1p;
      sB[sy][sx] = hz1p;
      __syncthreads();
      const T dey2 = ey1 - ey1p, dex2 = ex1 - ex1p;
      const T hxa2 = hx1p + cHX2 * (dey2 - (sA[sy + 1][sx] - ez1p));   // U1
      const T hya2 = hy1p + cHY2 * (-dex2 + (sA[sy][sx + 1] - ez1p));  // U2
      sC[sy][sx] = hxa2;
      sD[sy][sx] = hya2;
      __syncthreads();
      T cur2 = (sC[sy - 1][sx] - hxa2) - (sD[sy][sx - 1] - hya2);
      if (line) {
        const long long d = (long long)p - (a.n + 1 + a.b.kshift) + a.b.c0;
        if (d >= -a.b.c0 && d < a.b.c0) cur2 -= a.b.J[d + a.b.c0];
      }
      const T ez2 = ez1p + cEZ2 * cur2;                                 // U3
      sE[sy][sx] = ez2;
      __syncthreads();
      const T hx2 = hxa2 + cHX2 * (dey2 - (sE[sy + 1][sx] - ez2));     // U4
      const T hy2 = hya2 + cHY2 * (-dex2 + (sE[sy][sx + 1] - ez2));    // U5
      if (p >= k0) {
        const long long idp = id - SZ;
        if (own) {
          a.out[kHX][idp] = hx2;
          a.out[kHY][idp] = hy2;
          a.out[kEZ][idp] = ez2;
          if (line) {
            const long long mm = (a.n + 1 + a.b.kshift) - p - a.b.c0;
            if (mm >= a.b.m_min && mm <= a.b.m_max)
              atomicAdd(a.b.W + (mm - a.b.m_min), -(double)ez2 * a.b.inv_q);
          }
        }
        const T cEX2 = (mp & 1) ? uEX : T(0), cEY2 = (mp & 2) ? uEY : T(0), cHZ2 = (mp & 32) ? uHZ : T(0);
        const T dhy2 = hy2p - hy2, dhx2 = hx2p - hx2;
        const T exa2 = ex1p + cEX2 * (dhy2 - (sB[sy - 1][sx] - hz1p));    // U6
        const T eya2 = ey1p + cEY2 * (-dhx2 + (sB[sy][sx - 1] - hz1p));   // U7
        __syncthreads();
        sC[sy][sx] = exa2;
        sD[sy][sx] = eya2;
        __syncthreads();
        const T hz2 = hz1p + cHZ2 * ((sC[sy + 1][sx] - exa2) - (sD[sy][sx + 1] - eya2));  // U8
        __syncthreads();
        sE[sy][sx] = hz2;
        __syncthreads();
        const T ex2 = exa2 + cEX2 * (dhy2 - (sE[sy - 1][sx] - hz2));   // U9
        const T ey2 = eya2 + cEY2 * (-dhx2 + (sE[sy][sx - 1] - hz2));  // U10
        if (own) {
          a.out[kEX][idp] = ex2;
          a.out[kEY][idp] = ey2;
          a.out[kHZ][idp] = hz2;
        }
      }
      hx2p = hx2;
      hy2p = hy2;
    }
    __syncthreads();  // the next plane's first writes follow every read of this one
    // shift: first-step results of plane k become the second step's inputs
    hx1p = hx1; hy1p = hy1; ez1p = ez1; ex1p = ex1; ey1p = ey1; hz1p = hz1; mp = m0;
    ex0a = ex0b; ey0a = ey0b; ex0b = nex; ey0b = ney;
    ez0 = nez; hx0 = nhx; hy0 = nhy; hz0 = nhz; m0 = nm;
  }
}

template <typename T, int TX, int TY>
cudaError_t launch_fused2_shape(const StepArgs<T>& a, cudaStream_t st) {
  const int items = a.work ? a.n_work : a.tiles_x * a.tiles_y * a.n_chunks;
  if (items <= 0) return cudaSuccess;
  fused_step2<T, TX, TY><<<items, dim3(TX + 8, TY + 8), 0, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int TX, int TY>
cudaError_t launch_fused_shape(const StepArgs<T>& a, cudaStream_t st) {
  const int items = a.work ? a.n_work : a.tiles_x * a.tiles_y * a.n_chunks;
  if (items <= 0) return cudaSuccess;
  fused_step<T, TX, TY><<<items, dim3(TX + 4, TY + 4), 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool fused_shape_ok(int tx, int ty) {
  return (tx == 32 && (ty == 4 || ty == 8 || ty == 16)) || (tx == 64 && (ty == 4 || ty == 8));
}

template <typename T>
cudaError_t launch_fused_step(const StepArgs<T>& a, int tx, int ty, cudaStream_t st) {
  if (tx == 32 && ty == 4) return launch_fused_shape<T, 32, 4>(a, st);
  if (tx == 32 && ty == 8) return launch_fused_shape<T, 32, 8>(a, st);
  if (tx == 32 && ty == 16) return launch_fused_shape<T, 32, 16>(a, st);
  if (tx == 64 && ty == 4) return launch_fused_shape<T, 64, 4>(a, st);
  if (tx == 64 && ty == 8) return launch_fused_shape<T, 64, 8>(a, st);
  return cudaErrorInvalidValue;
}

bool fused2_shape_ok(int tx, int ty) { return (tx == 32 && (ty == 4 || ty == 8)) || (tx == 64 && ty == 4); }

template <typename T>
cudaError_t launch_fused_two_steps(const StepArgs<T>& a, int tx, int ty, cudaStream_t st) {
  if (tx == 32 && ty == 4) return launch_fused2_shape<T, 32, 4>(a, st);
  if (tx == 32 && ty == 8) return launch_fused2_shape<T, 32, 8>(a, st);
  if (tx == 64 && ty == 4) return launch_fused2_shape<T, 64, 4>(a, st);
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_reference_step(const StepArgs<T>& a, cudaStream_t st) {
  if (a.L.nz > 65535) return cudaErrorInvalidConfiguration;  // one grid z-slice per plane
  const dim3 blk(32, 8, 1);
  const dim3 grd((a.L.nx + 31) / 32, (a.L.ny + 7) / 8, a.L.nz);
  ref_update<T, kHX><<<grd, blk, 0, st>>>(a);  // U1
  ref_update<T, kHY><<<grd, blk, 0, st>>>(a);  // U2
  ref_update<T, kEZ><<<grd, blk, 0, st>>>(a);  // U3 (+ current, + wake)
  ref_update<T, kHX><<<grd, blk, 0, st>>>(a);  // U4
  ref_update<T, kHY><<<grd, blk, 0, st>>>(a);  // U5
  if (a.b.obs_on) ref_transverse_gather<T><<<(a.L.nz + 127) / 128, 128, 0, st>>>(a);
  ref_update<T, kEX><<<grd, blk, 0, st>>>(a);  // U6
  ref_update<T, kEY><<<grd, blk, 0, st>>>(a);  // U7
  ref_update<T, kHZ><<<grd, blk, 0, st>>>(a);  // U8
  ref_update<T, kEX><<<grd, blk, 0, st>>>(a);  // U9
  ref_update<T, kEY><<<grd, blk, 0, st>>>(a);  // U10
  return cudaGetLastError();
}

template cudaError_t launch_fused_two_steps<float>(const StepArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_fused_two_steps<double>(const StepArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_fused_step<float>(const StepArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_fused_step<double>(const StepArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_reference_step<float>(const StepArgs<float>&, cudaStream_t);
template cudaError_t launch_reference_step<double>(const StepArgs<double>&, cudaStream_t);

}  // namespace tetm
