// Yee's E/M leapfrog (Sec. 3, Eq. (7)) on the solver's device layout: the
// scheme the paper measures the TE/TM scheme against, field-only. The state is
// (e^{n-1/2}, h^n); one step is
//   e^{n+1/2} = e^{n-1/2} + dt M_eps^-1 C~ h^n,   h^{n+1} = h^n - dt M_mu^-1 C e^{n+1/2},
// in components the TE/TM updates U3, U6, U7 (electric) and U1, U2, U8
// (magnetic), each with the full step dt. Stable for
// c*dt <= (dx^-2 + dy^-2 + dz^-2)^-1/2, Eq. (8).
//
// Two implementations:
//  * reference: two in-place launches (electric, then magnetic) over every
//    node, per-entry or per-component coefficients;
//  * fused: one pass per step, ping-pong sets. A CTA of 512 threads takes
//    (tile, z chunk) items; a thread holds V = 16 / sizeof(T) x-consecutive
//    nodes of one row (16-byte loads and stores), 64 columns per row, so a CTA
//    loads 64 x 32 (float) or 64 x 16 (double) nodes and owns 56 x 30 or
//    60 x 14 of them. Marching up the chunk, plane k's pass computes e^{n+1/2}
//    of plane k+1 (it reads h^n one node down in x, y and one plane down in z)
//    and h^{n+1} of plane k (it reads e^{n+1/2} one node up in x, y and one
//    plane up in z). The rows a stage needs from other warps (h_x, h_z of
//    plane k+1; e_x, e_z of plane k) go through one of two shared-memory
//    buffers used by alternate planes, the columns by warp shuffles: one block
//    barrier per plane. Each chunk recomputes e^{n+1/2} of its first plane
//    from the plane below, so chunks never wait on each other.
#include <algorithm>

#include "tetm_internal.h"

namespace tetm {

namespace {

// Yee's coefficient dt M^-1 of component c at entry id: the per-component
// constants arrive as dt M^-1; the per-entry arrays hold the TE/TM scheme's
// alpha M^-1 (x, y components) or 2 alpha M^-1 (z components), alpha = dt/2.
template <typename T>
__device__ __forceinline__ T ycoef(const Coefs<T>& co, long long id, int c, unsigned m) {
  if (co.ua[c]) return (c == kEZ || c == kHZ) ? co.ua[c][id] : T(2) * co.ua[c][id];
  return ((m >> c) & 1u) ? co.u[c] : T(0);
}

// electric half, in place: reads h^n only
template <typename T>
__global__ void yee_electric_ref(const StepArgs<T> a) {
  const Layout L = a.L;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i > L.nx) return;
  const long long sy = L.px, sz = L.sz;
  T *ex = a.out[kEX], *ey = a.out[kEY], *ez = a.out[kEZ];
  const T *hx = a.in[kHX], *hy = a.in[kHY], *hz = a.in[kHZ];
  for (int k = blockIdx.z; k <= L.nz; k += gridDim.z) {
    const long long id = L.idx(i, j, k);
    const unsigned m = a.co.mask[id];
    ex[id] += ycoef(a.co, id, kEX, m) * ((hy[id - sz] - hy[id]) - (hz[id - sy] - hz[id]));
    ey[id] += ycoef(a.co, id, kEY, m) * (-(hx[id - sz] - hx[id]) + (hz[id - 1] - hz[id]));
    ez[id] += ycoef(a.co, id, kEZ, m) * ((hx[id - sy] - hx[id]) - (hy[id - 1] - hy[id]));
  }
}

// magnetic half, in place: reads e^{n+1/2} only
template <typename T>
__global__ void yee_magnetic_ref(const StepArgs<T> a) {
  const Layout L = a.L;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i > L.nx) return;
  const long long sy = L.px, sz = L.sz;
  const T *ex = a.in[kEX], *ey = a.in[kEY], *ez = a.in[kEZ];
  T *hx = a.out[kHX], *hy = a.out[kHY], *hz = a.out[kHZ];
  for (int k = blockIdx.z; k <= L.nz; k += gridDim.z) {
    const long long id = L.idx(i, j, k);
    const unsigned m = a.co.mask[id];
    hx[id] += ycoef(a.co, id, kHX, m) * ((ey[id + sz] - ey[id]) - (ez[id + sy] - ez[id]));
    hy[id] += ycoef(a.co, id, kHY, m) * (-(ex[id + sz] - ex[id]) + (ez[id + 1] - ez[id]));
    hz[id] += ycoef(a.co, id, kHZ, m) * ((ex[id + sy] - ex[id]) - (ey[id + 1] - ey[id]));
  }
}

// ---- fused ------------------------------------------------------------------
constexpr int kYThreads = 512;
constexpr int kYCols = 64;  // loaded columns per row

template <typename T>
struct YS {
  static constexpr int V = 16 / (int)sizeof(T);  // nodes per thread
  static constexpr int NQ = kYCols / V;          // threads per row
  static constexpr int R = kYThreads / NQ;       // loaded rows
  static constexpr int TX = kYCols - 2 * V;      // owned columns
  static constexpr int TY = R - 2;               // owned rows
  static constexpr size_t smem = 2u * 4u * R * kYCols * sizeof(T);
};

template <typename T>
struct Vv {
  T v[YS<T>::V];
};

template <typename T>
__device__ __forceinline__ Vv<T> vzero() {
  Vv<T> r;
#pragma unroll
  for (int e = 0; e < YS<T>::V; ++e) r.v[e] = T(0);
  return r;
}
__device__ __forceinline__ Vv<float> vld(const float* p) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(p));
  return Vv<float>{{t.x, t.y, t.z, t.w}};
}
__device__ __forceinline__ Vv<double> vld(const double* p) {
  const double2 t = __ldg(reinterpret_cast<const double2*>(p));
  return Vv<double>{{t.x, t.y}};
}
__device__ __forceinline__ void vst(float* p, const Vv<float>& a) {
  *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}
__device__ __forceinline__ void vst(double* p, const Vv<double>& a) {
  *reinterpret_cast<double2*>(p) = make_double2(a.v[0], a.v[1]);
}
template <typename T>
__device__ __forceinline__ Vv<T> vlds(const T* p) {
  if constexpr (sizeof(T) == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    return Vv<T>{{t.x, t.y, t.z, t.w}};
  } else {
    const double2 t = *reinterpret_cast<const double2*>(p);
    return Vv<T>{{t.x, t.y}};
  }
}
// activity bytes of the V nodes (byte e = node e)
__device__ __forceinline__ unsigned mld(const uint8_t* p, float*) { return *reinterpret_cast<const unsigned*>(p); }
__device__ __forceinline__ unsigned mld(const uint8_t* p, double*) {
  return *reinterpret_cast<const unsigned short*>(p);
}

// the neighbouring thread's value one column left (x-1) or right (x+1) of this
// thread's nodes, zero at the tile edge (a row is NQ consecutive lanes)
template <typename T>
__device__ __forceinline__ T yleft(T vlast, int q) {
  const T t = __shfl_up_sync(0xffffffffu, vlast, 1);
  return q >= 1 ? t : T(0);
}
template <typename T>
__device__ __forceinline__ T yright(T vfirst, int q) {
  const T t = __shfl_down_sync(0xffffffffu, vfirst, 1);
  return q + 1 < YS<T>::NQ ? t : T(0);
}

template <typename T>
__global__ void __launch_bounds__(kYThreads, 1) yee_fused(const StepArgs<T> a) {
  using S = YS<T>;
  constexpr int V = S::V, NQ = S::NQ, R = S::R;
  extern __shared__ __align__(16) unsigned char yee_raw[];
  // [buffer][h_x, h_z of plane k+1 | e_x, e_z of plane k][row][column]
  T(*sb)[4][R][kYCols] = reinterpret_cast<T(*)[4][R][kYCols]>(yee_raw);
  const int tid = threadIdx.x, q = tid % NQ, row = tid / NQ;
  const Layout L = a.L;
  const long long SZ = L.sz, PX = L.px;
  const int ntile = a.tiles_x * a.tiles_y;
  const int nitems = a.work ? a.n_work : ntile * a.n_chunks;

  for (int wi = blockIdx.x; wi < nitems; wi += gridDim.x) {
    const int item = a.work ? a.work[wi] : wi;
    const int tile = item % ntile, chunk = item / ntile;
    const int gx0 = (tile % a.tiles_x) * S::TX - V;  // global i of loaded column 0
    const int gy0 = (tile / a.tiles_x) * S::TY - 1;  // global j of loaded row 0
    const int k0 = chunk * a.chunk_z, k1 = min(k0 + a.chunk_z, L.nz);
    const int kstart = k0 - 1;
    const int gi = gx0 + V * q, gj = gy0 + row;
    const int jc = min(gj, L.ny + 1);
    // vectors start on multiples of V in a row whose pitch is a multiple of V:
    // a vector lies wholly inside the padded row or wholly past it
    const bool inrow = gi + L.ox + V <= L.px;
    const bool own = q >= 1 && q <= NQ - 2 && row >= 1 && row <= R - 2 && gj < L.ny;
    auto gid = [&](int k) { return (long long)(k + 1) * SZ + (long long)(jc + 2) * PX + (gi + L.ox); };
    auto ld = [&](const T* base, int k) -> Vv<T> { return inrow ? vld(base + gid(k)) : vzero<T>(); };
    auto ldm = [&](int k) -> unsigned { return inrow ? mld(a.co.mask + gid(k), (T*)nullptr) : 0u; };
    auto st = [&](T* base, int k, const Vv<T>& v) {
      const long long id = gid(k);
      if (gi + V - 1 < L.nx) {
        vst(base + id, v);
      } else {
#pragma unroll
        for (int e = 0; e < V; ++e)
          if (gi + e < L.nx) base[id + e] = v.v[e];
      }
    };
    // one coefficient per component, switched by the activity bytes (the
    // solver runs material arrays on the reference updates)
    auto cof = [&](int c, int e, unsigned mw) -> T { return ((mw >> (8 * e + c)) & 1u) ? a.co.u[c] : T(0); };

    // h^n of the plane below the chunk, h^n and e^{n-1/2} of its first plane
    Vv<T> hOx = ld(a.in[kHX], kstart), hOy = ld(a.in[kHY], kstart), hOz = ld(a.in[kHZ], kstart);
    Vv<T> h1x = ld(a.in[kHX], k0), h1y = ld(a.in[kHY], k0), h1z = ld(a.in[kHZ], k0);
    Vv<T> e1x = ld(a.in[kEX], k0), e1y = ld(a.in[kEY], k0), e1z = ld(a.in[kEZ], k0);
    unsigned m1 = ldm(k0), m0 = 0u;
    Vv<T> eNx = vzero<T>(), eNy = vzero<T>(), eNz = vzero<T>();  // e^{n+1/2} of plane k

    for (int k = kstart; k < k1; ++k) {
      const int b = (k - kstart) & 1;
      // the next plane's inputs, early
      const bool more = k + 1 < k1;
      Vv<T> h2x, h2y, h2z, e2x, e2y, e2z;
      unsigned m2 = 0u;
      if (more) {
        h2x = ld(a.in[kHX], k + 2);
        h2y = ld(a.in[kHY], k + 2);
        h2z = ld(a.in[kHZ], k + 2);
        e2x = ld(a.in[kEX], k + 2);
        e2y = ld(a.in[kEY], k + 2);
        e2z = ld(a.in[kEZ], k + 2);
        m2 = ldm(k + 2);
      }
      // rows for the neighbours: h_x, h_z of plane k+1 (read one row up),
      // e_x, e_z of plane k (read one row down)
      *reinterpret_cast<Vv<T>*>(&sb[b][0][row][V * q]) = h1x;
      *reinterpret_cast<Vv<T>*>(&sb[b][1][row][V * q]) = h1z;
      *reinterpret_cast<Vv<T>*>(&sb[b][2][row][V * q]) = eNx;
      *reinterpret_cast<Vv<T>*>(&sb[b][3][row][V * q]) = eNz;
      __syncthreads();

      // electric half of plane k+1 (h^n of planes k, k+1)
      const Vv<T> hxD = row >= 1 ? vlds(&sb[b][0][row - 1][V * q]) : vzero<T>();
      const Vv<T> hzD = row >= 1 ? vlds(&sb[b][1][row - 1][V * q]) : vzero<T>();
      const T hzL = yleft(h1z.v[V - 1], q), hyL = yleft(h1y.v[V - 1], q);
      Vv<T> enx, eny, enz;
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const T hzl = e > 0 ? h1z.v[e - 1] : hzL;
        const T hyl = e > 0 ? h1y.v[e - 1] : hyL;
        enx.v[e] = e1x.v[e] + cof(kEX, e, m1) * ((hOy.v[e] - h1y.v[e]) - (hzD.v[e] - h1z.v[e]));
        eny.v[e] = e1y.v[e] + cof(kEY, e, m1) * (-(hOx.v[e] - h1x.v[e]) + (hzl - h1z.v[e]));
        enz.v[e] = e1z.v[e] + cof(kEZ, e, m1) * ((hxD.v[e] - h1x.v[e]) - (hyl - h1y.v[e]));
      }
      // magnetic half of plane k (e^{n+1/2} of planes k, k+1)
      const Vv<T> ezU = row + 1 < R ? vlds(&sb[b][3][row + 1][V * q]) : vzero<T>();
      const Vv<T> exU = row + 1 < R ? vlds(&sb[b][2][row + 1][V * q]) : vzero<T>();
      const T ezR = yright(eNz.v[0], q), eyR = yright(eNy.v[0], q);
      Vv<T> hnx, hny, hnz;
#pragma unroll
      for (int e = 0; e < V; ++e) {
        const T ezr = e < V - 1 ? eNz.v[e + 1] : ezR;
        const T eyr = e < V - 1 ? eNy.v[e + 1] : eyR;
        hnx.v[e] = hOx.v[e] + cof(kHX, e, m0) * ((eny.v[e] - eNy.v[e]) - (ezU.v[e] - eNz.v[e]));
        hny.v[e] = hOy.v[e] + cof(kHY, e, m0) * (-(enx.v[e] - eNx.v[e]) + (ezr - eNz.v[e]));
        hnz.v[e] = hOz.v[e] + cof(kHZ, e, m0) * ((exU.v[e] - eNx.v[e]) - (eyr - eNy.v[e]));
      }
      if (own) {
        if (k >= k0) {
          st(a.out[kHX], k, hnx);
          st(a.out[kHY], k, hny);
          st(a.out[kHZ], k, hnz);
        }
        if (k + 1 < k1) {  // the next chunk computes (and stores) its own first plane
          st(a.out[kEX], k + 1, enx);
          st(a.out[kEY], k + 1, eny);
          st(a.out[kEZ], k + 1, enz);
        }
      }
      // carry up one plane
      eNx = enx;
      eNy = eny;
      eNz = enz;
      hOx = h1x;
      hOy = h1y;
      hOz = h1z;
      m0 = m1;
      if (more) {
        h1x = h2x;
        h1y = h2y;
        h1z = h2z;
        e1x = e2x;
        e1y = e2y;
        e1z = e2z;
        m1 = m2;
      }
    }
    __syncthreads();  // the buffers are free before the next item writes them
  }
}

}  // namespace

void yee_shape(int elem_bytes, int* tile_x, int* tile_y) {
  if (elem_bytes == 4) {
    *tile_x = YS<float>::TX;
    *tile_y = YS<float>::TY;
  } else {
    *tile_x = YS<double>::TX;
    *tile_y = YS<double>::TY;
  }
}

template <typename T>
cudaError_t launch_yee_reference_step(const StepArgs<T>& a, cudaStream_t st) {
  const dim3 grid((unsigned)((a.L.nx + 1 + 127) / 128), (unsigned)(a.L.ny + 1),
                  (unsigned)std::min(a.L.nz + 1, 65535));
  if (a.L.ny + 1 > 65535) return cudaErrorInvalidValue;
  yee_electric_ref<T><<<grid, 128, 0, st>>>(a);
  yee_magnetic_ref<T><<<grid, 128, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_yee_fused_step(const StepArgs<T>& a, cudaStream_t st) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(yee_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)YS<T>::smem);
    if (e != cudaSuccess) {
      sms = 0;
      return e;
    }
  }
  const int items = a.work ? a.n_work : a.tiles_x * a.tiles_y * a.n_chunks;
  if (items <= 0) return cudaSuccess;
  yee_fused<T><<<std::min(items, sms), kYThreads, YS<T>::smem, st>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_yee_reference_step<float>(const StepArgs<float>&, cudaStream_t);
template cudaError_t launch_yee_reference_step<double>(const StepArgs<double>&, cudaStream_t);
template cudaError_t launch_yee_fused_step<float>(const StepArgs<float>&, cudaStream_t);
template cudaError_t launch_yee_fused_step<double>(const StepArgs<double>&, cudaStream_t);

}  // namespace tetm
