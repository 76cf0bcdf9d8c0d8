// Block-tiled fused step with tensor staging, float32 (Sec. 4.2, Eq. (23)).
//
// One CTA of 512 threads per SM takes (tile, z chunk) work items in turn. A
// tile owns 56 x 28 nodes and loads 64 x 32 (4 halo columns and 2 halo rows on
// each side: the ten updates reach two nodes sideways). Thread t holds the
// four consecutive columns 4 (t mod 16) .. +3 of row t / 16 (a quad), so its
// loads and stores are 16-byte vectors, and marches through the chunk plane by
// plane with the z-state of its quad in registers (old e_x, e_y of the plane,
// new h_x, h_y of the plane below): no per-row state in shared memory.
//
// Only entries that carry a field move through the per-thread loads and
// stores. Each thread reads the activity bytes of its quad (one 32-bit word
// per plane, three planes ahead) and
//  * loads h_x, h_y, e_x, e_y of the quad (16-byte loads one plane ahead) only
//    when one of its four nodes carries that component, else takes zero (an
//    entry without a field holds zero for ever);
//  * stores each new component of the quad only when one of its nodes
//    carries it (the other field set's entry already holds that zero).
// e_z and h_z are the inputs a node reads at its neighbours; they (and with
// material arrays the six per-entry coefficient arrays, read at the node)
// arrive through a ring of two planes in shared memory, filled two planes
// ahead: each thread copies its own quad of every array into the slot with a
// 16-byte asynchronous copy, or writes zeros without a read where none of
// the quad's nodes carries that component (an entry without a field, and its
// coefficient, hold zero), so the ring reads no pipe wall. Completion by the
// thread's copy group, publication by the last block barrier of the plane
// before.
//
// The intermediates a stage reads one row up or down (hx~, ez', ex~, hz') go
// through two shared-memory buffers, those one column left or right through
// warp shuffles; four block barriers per plane, the first of which also
// settles the slot waits:
//   S1 hx~, hy~ (U1, U2)  | S2 ez' (U3, + current) | S3 hx', hy' (U4, U5)
//   S4 ex~, ey~ (U6, U7)  | S5 hz' (U8)            | S6 ex', ey' (U9, U10)
// The column of i = 0 sits at 8 in the float32 layout, so the 224-byte rows a
// tile writes start and end on 32-byte sectors and no two tiles write into
// the same sector.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "tetm_internal.h"

namespace tetm {

namespace {

constexpr int kSX = 64, kSY = 32;   // loaded columns, rows
constexpr int kOX = 56, kOY = 28;   // owned columns, rows
constexpr int kQ = kSX / 4;         // column quads per row
constexpr int kSThreads = kQ * kSY; // 512

// One material: a two-plane ring of e_z and h_z (one coefficient per
// component, switched by the activity bytes).
struct SlabSmemU {
  static constexpr int SD = 2;      // planes in the ring (the next plane lands while this one is worked on)
  float ez[SD][kSY * kSX];
  float hz[SD][kSY * kSX];
  float x1[kSY][kSX], x2[kSY][kSX];
  int next[2];                      // the CTA's next work item (dynamic schedule)
};
// Material arrays: a two-plane ring of e_z, h_z and the six per-entry
// coefficient arrays (alpha M^-1, 2 alpha M^-1 for e_z and h_z), 144 KB.
struct SlabSmemM {
  static constexpr int SD = 2;
  float ez[SD][kSY * kSX];
  float hz[SD][kSY * kSX];
  float co[SD][6][kSY][kSX];
  float x1[kSY][kSX], x2[kSY][kSX];
  int next[2];
};
template <bool MAT>
using SlabSmem = typename std::conditional<MAT, SlabSmemM, SlabSmemU>::type;


__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
// loads and stores under a predicate, without a branch (zero where not loaded)
__device__ __forceinline__ unsigned ld_word_if(const uint8_t* p, bool c) {
  unsigned v;
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n mov.u32 %0, 0;\n @q ld.global.nc.u32 %0, [%1];\n}"
      : "=r"(v)
      : "l"(p), "r"((unsigned)c));
  return v;
}
// 16 bytes into shared memory by an asynchronous copy, or (c false) 16 zero
// bytes without a global read
__device__ __forceinline__ void cp16_or_zero(void* sdst, const void* gsrc, bool c) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(sdst)), "l"(gsrc), "r"(c ? 16u : 0u)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
// the quad's word holds one activity byte per node: component c of any node
__device__ __forceinline__ bool has(unsigned m, int c) { return (m & (0x01010101u << c)) != 0u; }

struct Q4 {
  float v[4];
};
__device__ __forceinline__ Q4 q4(float4 a) { return Q4{{a.x, a.y, a.z, a.w}}; }
__device__ __forceinline__ Q4 ld4_if(const float* p, bool c) {
  Q4 r;
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.u32 q, %5, 0;\n mov.f32 %0, 0f00000000;\n mov.f32 %1, 0f00000000;\n"
      " mov.f32 %2, 0f00000000;\n mov.f32 %3, 0f00000000;\n"
      " @q ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];\n}"
      : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3])
      : "l"(p), "r"((unsigned)c));
  return r;
}
__device__ __forceinline__ void st4_if(float* p, const Q4& v, bool c) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %5, 0;\n @q st.global.v4.f32 [%0], {%1,%2,%3,%4};\n}" ::"l"(p),
               "f"(v.v[0]), "f"(v.v[1]), "f"(v.v[2]), "f"(v.v[3]), "r"((unsigned)c)
               : "memory");
}
__device__ __forceinline__ Q4 lds4(const float* p) { return q4(*reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void sts4(float* p, const Q4& a) {
  *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}

// the neighbouring quad's value one column left (x-1) or right (x+1) of this
// quad, zero at the tile edge (lanes: one row per half warp)
__device__ __forceinline__ float left_of(float v3, int q) {
  const float t = __shfl_up_sync(0xffffffffu, v3, 1);
  return q >= 1 ? t : 0.f;
}
__device__ __forceinline__ float right_of(float v0, int q) {
  const float t = __shfl_down_sync(0xffffffffu, v0, 1);
  return q + 1 < kQ ? t : 0.f;
}

// One (tile, z-chunk) work item of solve a (the ten updates of every plane
// of the chunk).
template <bool MAT>
__device__ __forceinline__ void slab_item(const StepArgs<float>& a, int item, SlabSmem<MAT>& S) {
  using Smem = SlabSmem<MAT>;
  constexpr int kSD = Smem::SD;
  const int tid = threadIdx.x, q = tid % kQ, row = tid / kQ;
  const Layout L = a.L;
  const long long SZ = L.sz, PX = L.px;
  const float uEX = a.co.u[kEX], uEY = a.co.u[kEY], uEZ = a.co.u[kEZ];
  const float uHX = a.co.u[kHX], uHY = a.co.u[kHY], uHZ = a.co.u[kHZ];
  const int ntile = a.tiles_x * a.tiles_y;
  const Q4 zero{{0.f, 0.f, 0.f, 0.f}};
  const int tile = item % ntile, chunk = item / ntile;
  const int gx0 = (tile % a.tiles_x) * kOX - 4;  // global i of loaded column 0
  const int gy0 = (tile / a.tiles_x) * kOY - 2;  // global j of loaded row 0
  const int k0 = chunk * a.chunk_z, k1 = min(k0 + a.chunk_z, L.nz);
  const int kstart = k0 - 1;
  const int nplanes = k1 - kstart;
  const int cx = gx0 + L.ox;                   // layout column of loaded column 0

  // this thread's quad; a quad with an active node lies inside its layout
  // row (columns i <= nx + 2 < px - ox), so every predicated access is a
  // whole 16-byte vector (a quad across i = nx stores the zeros its entries
  // past the cells compute: zero input, zero coefficient)
  const int gi = gx0 + 4 * q, gj = gy0 + row;
  const bool inq = gj + 2 < L.ny + 4 && cx + 4 * q + 4 <= PX;  // the quad lies inside the arrays
  const long long qoff = (long long)(gj + 2) * PX + cx + 4 * q;
  const bool own_q = q >= 1 && q <= kQ - 2 && row >= 2 && row < kSY - 2 && gj < L.ny;
  auto gidx = [&](int k) { return (long long)(k + 1) * SZ + qoff; };
  auto word = [&](int k) -> unsigned { return ld_word_if(a.co.mask + gidx(k), inq); };
  auto load_if = [&](const float* base, int k, bool p) -> Q4 { return ld4_if(base + gidx(k), p); };
  // plane k into its slot: each thread copies the quad of its own node row
  // and columns of e_z, h_z (and of the six coefficient arrays), only where
  // one of the quad's nodes carries that component (zeros otherwise: the
  // entry and its coefficient hold zero), so the ring reads no pipe wall;
  // completion by the thread's copy group and the block barrier after it
  auto issue_q = [&](int k, unsigned mw) {
    const int s = (k - kstart) % kSD;
    const long long g = inq ? gidx(k) : 0;
    cp16_or_zero(&S.ez[s][row * kSX + 4 * q], a.in[kEZ] + g, has(mw, kEZ));
    cp16_or_zero(&S.hz[s][row * kSX + 4 * q], a.in[kHZ] + g, has(mw, kHZ));
    if constexpr (MAT) {
#pragma unroll
      for (int c = 0; c < 6; ++c) cp16_or_zero(&S.co[s][c][row][4 * q], a.co.ua[c] + g, has(mw, c));
    }
  };
  // activity words of planes kstart .. kstart + 2 (m0 of the plane being
  // worked on, m1, m2 of the next two); z-state and the register prefetch
  // (plane k: hx, hy of k; ex, ey of k+1)
  unsigned m0 = word(kstart), m1 = word(kstart + 1), m2 = word(kstart + 2);
  issue_q(kstart, m0);
  cp_commit();
  if (nplanes > 1) issue_q(kstart + 1, m1);
  cp_commit();
  cp_wait<1>();
  __syncthreads();  // plane kstart's slot is in
  Q4 ex0 = load_if(a.in[kEX], kstart, has(m0, kEX)), ey0 = load_if(a.in[kEY], kstart, has(m0, kEY));
  Q4 hxc = load_if(a.in[kHX], kstart, has(m0, kHX)), hyc = load_if(a.in[kHY], kstart, has(m0, kHY));
  Q4 ex1 = load_if(a.in[kEX], kstart + 1, has(m1, kEX)), ey1 = load_if(a.in[kEY], kstart + 1, has(m1, kEY));
  Q4 hxp = zero, hyp = zero;
  const bool line_row = a.b.on && gj == a.b.j0;
  const bool line_q = line_row && a.b.i0 >= gi && a.b.i0 < gi + 4;  // the quad holds the bunch line node

  for (int k = kstart; k < k1; ++k) {
    const int s = (k - kstart) % kSD;
    // next plane's register inputs and the activity word three planes on, early
    Q4 hxn_in, hyn_in, exn_in, eyn_in;
    unsigned m3 = 0u;
    const bool more = k + 1 < k1;
    if (more) {
      hxn_in = load_if(a.in[kHX], k + 1, has(m1, kHX));
      hyn_in = load_if(a.in[kHY], k + 1, has(m1, kHY));
      exn_in = load_if(a.in[kEX], k + 2, has(m2, kEX));
      eyn_in = load_if(a.in[kEY], k + 2, has(m2, kEY));
      if (k + 3 <= k1) m3 = word(k + 3);
    }
    // slot inputs: e_z, h_z of this quad and its neighbours
    const float* sez = &S.ez[s][0];
    const float* shz = &S.hz[s][0];
    const Q4 ez = lds4(sez + row * kSX + 4 * q);
    const Q4 ezU = row + 1 < kSY ? lds4(sez + (row + 1) * kSX + 4 * q) : zero;
    const float ezR = q + 1 < kQ ? sez[row * kSX + 4 * q + 4] : 0.f;
    const Q4 hz = lds4(shz + row * kSX + 4 * q);
    const Q4 hzD = row >= 1 ? lds4(shz + (row - 1) * kSX + 4 * q) : zero;
    const float hzL = q >= 1 ? shz[row * kSX + 4 * q - 1] : 0.f;
    float cHX[4], cHY[4], cEZ[4], cEX[4], cEY[4], cHZ[4], dey[4], dex[4];
    if constexpr (MAT) {  // per-entry coefficients from the slot
      const Q4 c0 = lds4(&S.co[s][kEX][row][4 * q]), c1 = lds4(&S.co[s][kEY][row][4 * q]);
      const Q4 c2 = lds4(&S.co[s][kEZ][row][4 * q]), c3 = lds4(&S.co[s][kHX][row][4 * q]);
      const Q4 c4 = lds4(&S.co[s][kHY][row][4 * q]), c5 = lds4(&S.co[s][kHZ][row][4 * q]);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        cEX[e] = c0.v[e];
        cEY[e] = c1.v[e];
        cEZ[e] = c2.v[e];
        cHX[e] = c3.v[e];
        cHY[e] = c4.v[e];
        cHZ[e] = c5.v[e];
      }
    } else {  // one coefficient per component, switched by the activity bytes
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const unsigned m = (m0 >> (8 * e)) & 0xFFu;
        cEX[e] = (m & 1) ? uEX : 0.f;
        cEY[e] = (m & 2) ? uEY : 0.f;
        cEZ[e] = (m & 4) ? uEZ : 0.f;
        cHX[e] = (m & 8) ? uHX : 0.f;
        cHY[e] = (m & 16) ? uHY : 0.f;
        cHZ[e] = (m & 32) ? uHZ : 0.f;
      }
    }
    Q4 hxa, hya;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      dey[e] = ey1.v[e] - ey0.v[e];
      dex[e] = ex1.v[e] - ex0.v[e];
      const float ezx = e < 3 ? ez.v[e + 1] : ezR;
      hxa.v[e] = hxc.v[e] + cHX[e] * (dey[e] - (ezU.v[e] - ez.v[e]));   // U1
      hya.v[e] = hyc.v[e] + cHY[e] * (-dex[e] + (ezx - ez.v[e]));      // U2
    }
    sts4(&S.x1[row][4 * q], hxa);
    __syncthreads();  // (1) the slot is read and hx~ is out
    if (k + kSD < k1) issue_q(k + kSD, m2);  // into the freed slot
    cp_commit();
    // S2: ez' = ez + 2a M^-1 (P_y^T hx~ - P_x^T hy~ - jj_z)
    const Q4 hxaD = row >= 1 ? lds4(&S.x1[row - 1][4 * q]) : zero;
    const float hyaL = left_of(hya.v[3], q);
    float cur[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float hyl = e > 0 ? hya.v[e - 1] : hyaL;
      cur[e] = (hxaD.v[e] - hxa.v[e]) - (hyl - hya.v[e]);
    }
    if (line_q) {  // the bunch current on its line (one quad of a tile row)
      const long long dd = (long long)k - (a.n + a.b.kshift) + a.b.c0;
      if (dd >= -a.b.c0 && dd < a.b.c0) {
        const float jj = a.b.J[dd + a.b.c0];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (gi + e == a.b.i0) cur[e] -= jj;
      }
    }
    Q4 ezn;
#pragma unroll
    for (int e = 0; e < 4; ++e) ezn.v[e] = ez.v[e] + cEZ[e] * cur[e];   // U3
    sts4(&S.x2[row][4 * q], ezn);
    __syncthreads();  // (2)
    // S3: hx', hy'
    const Q4 eznU = row + 1 < kSY ? lds4(&S.x2[row + 1][4 * q]) : zero;
    const float eznR = right_of(ezn.v[0], q);
    Q4 hxn, hyn;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float ezx = e < 3 ? ezn.v[e + 1] : eznR;
      hxn.v[e] = hxa.v[e] + cHX[e] * (dey[e] - (eznU.v[e] - ezn.v[e]));  // U4
      hyn.v[e] = hya.v[e] + cHY[e] * (-dex[e] + (ezx - ezn.v[e]));     // U5
    }
    const bool st = k >= k0 && own_q;
    st4_if(a.out[kEZ] + gidx(k), ezn, st && has(m0, kEZ));
    st4_if(a.out[kHX] + gidx(k), hxn, st && has(m0, kHX));
    st4_if(a.out[kHY] + gidx(k), hyn, st && has(m0, kHY));
    if (st) {
      if (line_q && a.b.i0 < L.nx) {
        const long long mm = (a.n + a.b.kshift) - k - a.b.c0;
        if (mm >= a.b.m_min && mm <= a.b.m_max)
        {
          const int e = a.b.i0 - gi;  // the quad's entry on the bunch line (no indexed register array)
          const float v = e == 0 ? ezn.v[0] : e == 1 ? ezn.v[1] : e == 2 ? ezn.v[2] : ezn.v[3];
          a.b.W[mm - a.b.m_min] -= (double)v * a.b.inv_q;
        }
      }
    }
    // S4: ex~, ey~ with the new hx, hy of this plane and of the plane below
    Q4 exa, eya;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float hzl = e > 0 ? hz.v[e - 1] : hzL;
      exa.v[e] = ex0.v[e] + cEX[e] * ((hyp.v[e] - hyn.v[e]) - (hzD.v[e] - hz.v[e]));   // U6
      eya.v[e] = ey0.v[e] + cEY[e] * (-(hxp.v[e] - hxn.v[e]) + (hzl - hz.v[e]));       // U7
    }
    sts4(&S.x1[row][4 * q], exa);
    __syncthreads();  // (3)
    // S5: hz'
    const Q4 exaU = row + 1 < kSY ? lds4(&S.x1[row + 1][4 * q]) : zero;
    const float eyaR = right_of(eya.v[0], q);
    Q4 hzn;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float eyx = e < 3 ? eya.v[e + 1] : eyaR;
      hzn.v[e] = hz.v[e] + cHZ[e] * ((exaU.v[e] - exa.v[e]) - (eyx - eya.v[e]));      // U8
    }
    sts4(&S.x2[row][4 * q], hzn);
    cp_wait<1>();     // this thread's copies of the next plane are in
    __syncthreads();  // (4) (and the next plane's slot is in)
    // S6: ex', ey'
    const Q4 hznD = row >= 1 ? lds4(&S.x2[row - 1][4 * q]) : zero;
    const float hznL = left_of(hzn.v[3], q);
    Q4 exn, eyn;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float hzl = e > 0 ? hzn.v[e - 1] : hznL;
      exn.v[e] = exa.v[e] + cEX[e] * ((hyp.v[e] - hyn.v[e]) - (hznD.v[e] - hzn.v[e]));   // U9
      eyn.v[e] = eya.v[e] + cEY[e] * (-(hxp.v[e] - hxn.v[e]) + (hzl - hzn.v[e]));       // U10
    }
    st4_if(a.out[kEX] + gidx(k), exn, st && has(m0, kEX));
    st4_if(a.out[kEY] + gidx(k), eyn, st && has(m0, kEY));
    st4_if(a.out[kHZ] + gidx(k), hzn, st && has(m0, kHZ));
    // carry the z-state, take the prefetched inputs
    hxp = hxn;
    hyp = hyn;
    ex0 = ex1;
    ey0 = ey1;
    m0 = m1;
    m1 = m2;
    m2 = m3;
    if (more) {
      hxc = hxn_in;
      hyc = hyn_in;
      ex1 = exn_in;
      ey1 = eyn_in;
    }
  }
  cp_wait<0>();
  __syncthreads();  // every thread is done with the ring before the next item refills it
}

template <bool MAT>
__global__ void __launch_bounds__(kSThreads, 1) fused_step_slab(const StepArgs<float> a, int* sched) {
  using Smem = SlabSmem<MAT>;
  extern __shared__ __align__(128) unsigned char slab_raw[];
  Smem& S = *reinterpret_cast<Smem*>(slab_raw);
  const int tid = threadIdx.x;
  const int nitems = a.work ? a.n_work : a.tiles_x * a.tiles_y * a.n_chunks;

  // Items in list order: the first per CTA by its index, then (with a
  // schedule counter) whichever item is next when the CTA gets free, fetched
  // one item ahead. Items that run at the same time stay neighbours (shared
  // halo rows in L2) and CTAs that drew cheap items (much PEC) take more.
  const int G = gridDim.x;
  int wi = blockIdx.x, par = 0;
  while (wi < nitems) {
    if (tid == 0 && sched) S.next[par] = G + atomicAdd(sched, 1);
    const int item = a.work ? a.work[wi] : wi;
    slab_item<MAT>(a, item, S);
    wi = sched ? S.next[par] : wi + G;
    par ^= 1;
  }
  // the last CTA to finish resets the schedule counter for the next launch
  if (tid == 0 && sched) {
    __threadfence();
    if (atomicAdd(sched + 1, 1) == G - 1) {
      atomicExch(sched, 0);
      atomicExch(sched + 1, 0);
    }
  }
}

// Batches: one launch steps every active member (one material, float32);
// work = (member, item) pairs, the member's arguments from device memory (its
// e_z, h_z come through the per-thread copies of the one-material ring, so
// no tensor map is involved).
__global__ void __launch_bounds__(kSThreads, 1)
fused_step_slab_batch(const BatchMember<float>* __restrict__ members, const int2* __restrict__ work,
                      const int* __restrict__ n_work_p, int* sched) {
  using Smem = SlabSmem<false>;
  extern __shared__ __align__(128) unsigned char slab_raw[];
  Smem& S = *reinterpret_cast<Smem*>(slab_raw);
  const int tid = threadIdx.x;
  const int G = gridDim.x;
  const int n_work = *n_work_p;  // written before the launch (stream order)
  int wi = blockIdx.x, par = 0;
  while (wi < n_work) {
    if (tid == 0 && sched) S.next[par] = G + atomicAdd(sched, 1);
    const int2 w = work[wi];
    const BatchMember<float>& mb = members[w.x];
    if (mb.active) {
      slab_item<false>(mb.a, w.y, S);
    } else {
      // an item of a member past its limit: no work, but the ticket thread 0
      // wrote above must be visible before every thread reads it (slab_item
      // ends with a block barrier; this branch needs its own)
      __syncthreads();
    }
    wi = sched ? S.next[par] : wi + G;
    par ^= 1;
  }
  if (tid == 0 && sched) {
    __threadfence();
    if (atomicAdd(sched + 1, 1) == G - 1) {
      atomicExch(sched, 0);
      atomicExch(sched + 1, 0);
    }
  }
}

}  // namespace

bool slab_shape_ok(int tx, int ty) { return tx == kOX && ty == kOY; }

namespace {
template <bool MAT>
cudaError_t launch_slab(const StepArgs<float>& a, int* sched, cudaStream_t st) {
  static int sms = 0;
  const size_t smem = sizeof(SlabSmem<MAT>);
  if (!sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fused_step_slab<MAT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
      sms = 0;
      return e;
    }
  }
  const int items = a.work ? a.n_work : a.tiles_x * a.tiles_y * a.n_chunks;
  if (items <= 0) return cudaSuccess;
  fused_step_slab<MAT><<<std::min(items, sms), kSThreads, smem, st>>>(a, sched);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_fused_slab_batch(BatchMember<float>* members, int n_members, const int2* work,
                                    const int* n_work, int n_bound, int* sched, int nz_max, cudaStream_t st) {
  static int sms = 0;
  const size_t smem = sizeof(SlabSmem<false>);
  if (!sms) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fused_step_slab_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
      sms = 0;
      return e;
    }
  }
  if (n_bound > 0) {
    fused_step_slab_batch<<<std::min(n_bound, sms), kSThreads, smem, st>>>(members, work, n_work, sched);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = launch_transverse_after_batch_step<float>(members, n_members, nz_max, st);
  if (e != cudaSuccess) return e;
  return launch_batch_advance<float>(members, n_members, st);
}

cudaError_t launch_fused_slab_step(const StepArgs<float>& a, int* sched, cudaStream_t st) {
  // per-entry coefficient arrays (material runs) stream through the ring too
  if (a.co.ua[0]) return launch_slab<true>(a, sched, st);
  return launch_slab<false>(a, sched, st);
}

}  // namespace tetm
