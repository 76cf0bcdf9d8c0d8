// Block-tiled fused step, float32 (Sec. 4.2, Eq. (23)).
//
// One CTA of 512 threads per SM takes (tile, z chunk) work items in turn. A
// tile owns 56 x 28 nodes and loads 64 x 32 (4 halo columns and 2 halo rows on
// each side: the ten updates reach two nodes sideways); with coefficient
// arrays two CTAs of 256 threads per SM do the same on 56 x 12 tiles (64 x 16
// loaded), one CTA's barriers and copy waits overlapping the other's work.
// Thread t holds the four consecutive columns 4 (t mod 16) .. +3 of row
// t / 16 (a quad), so its loads and stores are 16-byte vectors, and marches
// through the chunk plane by plane with the z-state of its quad in registers
// (old e_x, e_y, new h_x, h_y of the planes below): no per-row state in
// shared memory.
//
// Only entries that carry a field move through the per-thread loads and
// stores. Each thread reads the activity bytes of its quad (one 32-bit word
// per plane, a few planes ahead) and
//  * loads h_x, h_y, e_x, e_y of the quad (16-byte loads one plane ahead) only
//    when one of its four nodes carries that component, else takes zero (an
//    entry without a field holds zero for ever);
//  * stores each new component of the quad only when one of its nodes
//    carries it (the other field set's entry already holds that zero).
// e_z and h_z are the inputs a node reads at its neighbours; they (and with
// material arrays the six per-entry coefficient arrays, read at the node)
// arrive through rings of two planes in shared memory: each thread copies its
// own quad of every array into the slot with a 16-byte asynchronous copy, or
// writes zeros without a read where none of the quad's nodes carries that
// component (an entry without a field, and its coefficient, hold zero), so the
// rings read no pipe wall. Completion by the thread's copy group, publication
// by a block barrier.
//
// The intermediates a stage reads one row up or down (hx~, ez', ex~, hz') go
// through shared-memory buffers, those one column left or right through warp
// shuffles. Six stages per plane:
//   S1 hx~, hy~ (U1, U2)  | S2 ez' (U3, + current) | S3 hx', hy' (U4, U5)
//   S4 ex~, ey~ (U6, U7)  | S5 hz' (U8)            | S6 ex', ey' (U9, U10)
// With one material they run plane by plane, a block barrier after S1, S2,
// S4 and S5 (two buffers). With coefficient arrays the sweep is skewed by half
// a step: iteration i runs S1..S3 of plane i+1 (the TM half reads only old
// fields) beside S4..S6 of plane i (the TE half reads the new h_x, h_y of
// planes i and i-1), as pairs A = S1|S4, B = S2|S5, C = S3|S6 with a barrier
// after A and after B (four buffers: C reads what B wrote, and the next A
// writes only buffers that other threads last read in B); the copies then
// have two planes of work to land. (The skew costs the one-material sweep more
// instructions than its barriers do: its coefficients come from the activity
// words, and a third plane of e_x, e_y rides in registers.) Per node the
// arithmetic and its order are the same in both, so the results are the same
// bits.
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
// with coefficient arrays: a 64 x 16 box (56 x 12 owned), two CTAs of 256
// threads per SM, whose barriers interleave
constexpr int kSYM = 16, kOYM = 12;
constexpr int kMThreads = kQ * kSYM; // 256

// One material: a two-plane ring of e_z and h_z (one coefficient per
// component, switched by the activity bytes) and two exchange buffers, laid
// out in one array with a spare row at the end, so that a read one row or
// one column past a buffer's edge stays inside it (see slab_item).
struct SlabSmemU {
  static constexpr int SD = 2;             // planes in the ring (the next plane lands while this one is worked on)
  static constexpr int kP = kSY * kSX;     // one box plane
  float f[(2 * SD + 2) * kP + kSX];        // e_z slots, h_z slots, x1, x2, spare row
  int next[2];                             // the CTA's next work item (dynamic schedule)
  __device__ __forceinline__ float* ez(int s) { return f + s * kP; }
  __device__ __forceinline__ float* hz(int s) { return f + (SD + s) * kP; }
  __device__ __forceinline__ float* x1() { return f + 2 * SD * kP; }
  __device__ __forceinline__ float* x2() { return f + (2 * SD + 1) * kP; }
};
// Material arrays: two-plane rings of e_z and h_z with the six per-entry
// coefficient arrays (alpha M^-1, 2 alpha M^-1 for e_z and h_z), and the four
// exchange buffers of the skewed sweep (hx~, ez', ex~, hz'), 160 KB, in one
// array with a spare row at the end (reads past a buffer's edge stay inside).
struct SlabSmemM {
  static constexpr int kP = kSYM * kSX;
  float f[20 * kP + kSX];  // e_z slots (2), h_z slots (2), 2 x 6 coefficient planes, x1..x4, spare row
  int next[2];
  __device__ __forceinline__ float* ez(int s) { return f + s * kP; }
  __device__ __forceinline__ float* hz(int s) { return f + (2 + s) * kP; }
  __device__ __forceinline__ float* co(int s, int c) { return f + (4 + 6 * s + c) * kP; }
  __device__ __forceinline__ float* x(int b) { return f + (15 + b) * kP; }  // b = 1..4: planes 16..19
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
// the same as a word, nonzero where true (a predicate operand for the
// accesses below, without a conversion from bool)
__device__ __forceinline__ unsigned hw(unsigned m, int c) { return m & (0x01010101u << c); }

struct Q4 {
  float v[4];
};
__device__ __forceinline__ Q4 q4(float4 a) { return Q4{{a.x, a.y, a.z, a.w}}; }
__device__ __forceinline__ Q4 ld4_if(const float* p, unsigned c) {
  Q4 r;
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.u32 q, %5, 0;\n mov.f32 %0, 0f00000000;\n mov.f32 %1, 0f00000000;\n"
      " mov.f32 %2, 0f00000000;\n mov.f32 %3, 0f00000000;\n"
      " @q ld.global.nc.v4.f32 {%0,%1,%2,%3}, [%4];\n}"
      : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3])
      : "l"(p), "r"(c));
  return r;
}
__device__ __forceinline__ void st4_if(float* p, const Q4& v, unsigned c) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %5, 0;\n @q st.global.v4.f32 [%0], {%1,%2,%3,%4};\n}" ::"l"(p),
               "f"(v.v[0]), "f"(v.v[1]), "f"(v.v[2]), "f"(v.v[3]), "r"(c)
               : "memory");
}
__device__ __forceinline__ Q4 lds4(const float* p) { return q4(*reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void sts4(float* p, const Q4& a) {
  *reinterpret_cast<float4*>(p) = make_float4(a.v[0], a.v[1], a.v[2], a.v[3]);
}

// the neighbouring quad's value one column left (x-1) or right (x+1) of this
// quad (lanes: one row per half warp); at the tile edge a lane takes a value
// of the other half warp's row, which only halo nodes read
__device__ __forceinline__ float left_any(float v3) { return __shfl_up_sync(0xffffffffu, v3, 1); }
__device__ __forceinline__ float right_any(float v0) { return __shfl_down_sync(0xffffffffu, v0, 1); }

// One (tile, z-chunk) work item of solve a with one material (the ten
// updates of every plane of the chunk, plane by plane: four block barriers
// per plane).
//
// The reads of a neighbour one row or column outside the 64 x 32 box take
// whatever the neighbouring shared-memory words or lanes hold, without an
// edge test. Each of the six stages reaches one node sideways, and a value
// computed from an outside neighbour is wrong only on the box's outermost
// row or column; through the stages that error reaches at most two rows and
// two columns in, all of them halo (the tile owns rows 2..29 and columns
// 4..59 of the box), and halo nodes are never stored.
__device__ __forceinline__ void slab_item(const StepArgs<float>& a, int item, SlabSmemU& S) {
  constexpr int kSD = SlabSmemU::SD;
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
  auto load_if = [&](const float* base, int k, unsigned p) -> Q4 { return ld4_if(base + gidx(k), p); };
  // plane k into its slot: each thread copies the quad of its own node row
  // and columns of e_z, h_z, only where one of the quad's nodes carries that
  // component (zeros otherwise: the entry holds zero), so the ring reads no
  // pipe wall; completion by the thread's copy group and the block barrier
  // after it
  auto issue_q = [&](int k, unsigned mw) {
    const int s = (k - kstart) % kSD;
    const long long g = inq ? gidx(k) : 0;
    cp16_or_zero(S.ez(s) + row * kSX + 4 * q, a.in[kEZ] + g, has(mw, kEZ));
    cp16_or_zero(S.hz(s) + row * kSX + 4 * q, a.in[kHZ] + g, has(mw, kHZ));
  };
  // activity words of planes k .. k + kSD (m[0] of the plane being worked
  // on; m[kSD] of the plane whose copy is issued next); z-state and the
  // register prefetch (plane k: hx, hy of k; ex, ey of k+1)
  unsigned m[kSD + 1];
#pragma unroll
  for (int i = 0; i <= kSD; ++i) m[i] = kstart + i <= k1 ? word(kstart + i) : 0u;
#pragma unroll
  for (int i = 0; i < kSD; ++i) {
    if (i < nplanes) issue_q(kstart + i, m[i]);
    cp_commit();
  }
  cp_wait<kSD - 1>();
  __syncthreads();  // plane kstart's slot is in
  Q4 ex0 = load_if(a.in[kEX], kstart, hw(m[0], kEX)), ey0 = load_if(a.in[kEY], kstart, hw(m[0], kEY));
  Q4 hxc = load_if(a.in[kHX], kstart, hw(m[0], kHX)), hyc = load_if(a.in[kHY], kstart, hw(m[0], kHY));
  Q4 ex1 = load_if(a.in[kEX], kstart + 1, hw(m[1], kEX)), ey1 = load_if(a.in[kEY], kstart + 1, hw(m[1], kEY));
  Q4 hxp = zero, hyp = zero;
  const bool line_row = a.b.on && gj == a.b.j0;
  const bool line_q = line_row && a.b.i0 >= gi && a.b.i0 < gi + 4;  // the quad holds the bunch line node

  for (int k = kstart; k < k1; ++k) {
    const int s = (k - kstart) % kSD;
    // next plane's register inputs and the activity word kSD + 1 planes on, early
    Q4 hxn_in, hyn_in, exn_in, eyn_in;
    unsigned mn = 0u;
    const bool more = k + 1 < k1;
    if (more) {
      hxn_in = load_if(a.in[kHX], k + 1, hw(m[1], kHX));
      hyn_in = load_if(a.in[kHY], k + 1, hw(m[1], kHY));
      exn_in = load_if(a.in[kEX], k + 2, hw(m[2], kEX));
      eyn_in = load_if(a.in[kEY], k + 2, hw(m[2], kEY));
      if (k + kSD + 1 <= k1) mn = word(k + kSD + 1);
    }
    // slot inputs: e_z, h_z of this quad and its neighbours
    const float* sez = S.ez(s) + row * kSX + 4 * q;
    const float* shz = S.hz(s) + row * kSX + 4 * q;
    const Q4 ez = lds4(sez);
    const Q4 ezU = lds4(sez + kSX);
    const float ezR = sez[4];
    const Q4 hz = lds4(shz);
    const Q4 hzD = lds4(shz - kSX);
    const float hzL = shz[-1];
    float* const x1 = S.x1() + row * kSX + 4 * q;  // this thread's quad in the exchange buffers
    float* const x2 = S.x2() + row * kSX + 4 * q;
    // one coefficient per component, switched by the activity bytes
    float cHX[4], cHY[4], cEZ[4], cEX[4], cEY[4], cHZ[4], dey[4], dex[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const unsigned b = (m[0] >> (8 * e)) & 0xFFu;
      cEX[e] = (b & 1) ? uEX : 0.f;
      cEY[e] = (b & 2) ? uEY : 0.f;
      cEZ[e] = (b & 4) ? uEZ : 0.f;
      cHX[e] = (b & 8) ? uHX : 0.f;
      cHY[e] = (b & 16) ? uHY : 0.f;
      cHZ[e] = (b & 32) ? uHZ : 0.f;
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
    sts4(x1, hxa);
    __syncthreads();  // (1) the slot is read and hx~ is out
    if (k + kSD < k1) issue_q(k + kSD, m[kSD]);  // into the freed slot
    cp_commit();
    // S2: ez' = ez + 2a M^-1 (P_y^T hx~ - P_x^T hy~ - jj_z)
    const Q4 hxaD = lds4(x1 - kSX);
    const float hyaL = left_any(hya.v[3]);
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
    sts4(x2, ezn);
    __syncthreads();  // (2)
    // S3: hx', hy'
    const Q4 eznU = lds4(x2 + kSX);
    const float eznR = right_any(ezn.v[0]);
    Q4 hxn, hyn;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float ezx = e < 3 ? ezn.v[e + 1] : eznR;
      hxn.v[e] = hxa.v[e] + cHX[e] * (dey[e] - (eznU.v[e] - ezn.v[e]));  // U4
      hyn.v[e] = hya.v[e] + cHY[e] * (-dex[e] + (ezx - ezn.v[e]));     // U5
    }
    const bool st = k >= k0 && own_q;
    const unsigned ms = st ? m[0] : 0u;  // the plane's word where this thread stores
    st4_if(a.out[kEZ] + gidx(k), ezn, hw(ms, kEZ));
    st4_if(a.out[kHX] + gidx(k), hxn, hw(ms, kHX));
    st4_if(a.out[kHY] + gidx(k), hyn, hw(ms, kHY));
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
    sts4(x1, exa);
    __syncthreads();  // (3)
    // S5: hz'
    const Q4 exaU = lds4(x1 + kSX);
    const float eyaR = right_any(eya.v[0]);
    Q4 hzn;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float eyx = e < 3 ? eya.v[e + 1] : eyaR;
      hzn.v[e] = hz.v[e] + cHZ[e] * ((exaU.v[e] - exa.v[e]) - (eyx - eya.v[e]));      // U8
    }
    sts4(x2, hzn);
    cp_wait<kSD - 1>();  // this thread's copies of the next plane are in
    __syncthreads();  // (4) (and the next plane's slot is in)
    // S6: ex', ey'
    const Q4 hznD = lds4(x2 - kSX);
    const float hznL = left_any(hzn.v[3]);
    Q4 exn, eyn;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float hzl = e > 0 ? hzn.v[e - 1] : hznL;
      exn.v[e] = exa.v[e] + cEX[e] * ((hyp.v[e] - hyn.v[e]) - (hznD.v[e] - hzn.v[e]));   // U9
      eyn.v[e] = eya.v[e] + cEY[e] * (-(hxp.v[e] - hxn.v[e]) + (hzl - hzn.v[e]));       // U10
    }
    st4_if(a.out[kEX] + gidx(k), exn, hw(ms, kEX));
    st4_if(a.out[kEY] + gidx(k), eyn, hw(ms, kEY));
    st4_if(a.out[kHZ] + gidx(k), hzn, hw(ms, kHZ));
    // carry the z-state, take the prefetched inputs
    hxp = hxn;
    hyp = hyn;
    ex0 = ex1;
    ey0 = ey1;
#pragma unroll
    for (int i = 0; i < kSD; ++i) m[i] = m[i + 1];
    m[kSD] = mn;
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

// One (tile, z-chunk) work item of solve a with per-entry coefficient
// arrays, skewed by half a step: iteration i runs the TM half of plane i+1
// (U1..U5, which reads only old fields) beside the TE half of plane i
// (U6..U10, which reads the new h_x, h_y of planes i and i-1), two block
// barriers per iteration. Neighbour reads past the box edge go without edge
// tests, as in slab_item (the two-node halo absorbs what they return).
__device__ __forceinline__ void slab_item_mat(const StepArgs<float>& a, int item, SlabSmemM& S) {
  const int tid = threadIdx.x, q = tid % kQ, row = tid / kQ;
  const Layout L = a.L;
  const long long SZ = L.sz, PX = L.px;
  const int ntile = a.tiles_x * a.tiles_y;
  const Q4 zero{{0.f, 0.f, 0.f, 0.f}};
  const int tile = item % ntile, chunk = item / ntile;
  const int gx0 = (tile % a.tiles_x) * kOX - 4;  // global i of loaded column 0
  const int gy0 = (tile / a.tiles_x) * kOYM - 2;  // global j of loaded row 0
  const int k0 = chunk * a.chunk_z, k1 = min(k0 + a.chunk_z, L.nz);
  const int kstart = k0 - 1;                   // the plane below the chunk: its new h_x, h_y feed U6, U7 of k0
  const int cx = gx0 + L.ox;                   // layout column of loaded column 0

  // this thread's quad; a quad with an active node lies inside its layout
  // row (columns i <= nx + 2 < px - ox), so every predicated access is a
  // whole 16-byte vector (a quad across i = nx stores the zeros its entries
  // past the cells compute: zero input, zero coefficient)
  const int gi = gx0 + 4 * q, gj = gy0 + row;
  const bool inq = gj + 2 < L.ny + 4 && cx + 4 * q + 4 <= PX;  // the quad lies inside the arrays
  const long long qoff = (long long)(gj + 2) * PX + cx + 4 * q;
  const bool own_q = q >= 1 && q <= kQ - 2 && row >= 2 && row < kSYM - 2 && gj < L.ny;
  const int qo = row * kSX + 4 * q;  // this thread's quad in a box plane
  float* const x1 = S.x(1) + qo;     // and in the exchange buffers
  float* const x2 = S.x(2) + qo;
  float* const x3 = S.x(3) + qo;
  float* const x4 = S.x(4) + qo;
  auto gidx = [&](int k) { return (long long)(k + 1) * SZ + qoff; };
  auto word = [&](int k) -> unsigned { return ld_word_if(a.co.mask + gidx(k), inq); };
  auto load_if = [&](const float* base, int k, unsigned p) -> Q4 { return ld4_if(base + gidx(k), p); };
  // e_z of plane k with the coefficient arrays of h_x, h_y, e_z (the TM
  // half), h_z of plane k with those of e_x, e_y, h_z (the TE half), into
  // their slots: each thread copies the quads of its own
  // node row and columns, only where one of the quad's nodes carries that
  // component (zeros otherwise: the entry and its coefficient hold zero), so
  // the ring reads no pipe wall; completion by the thread's copy group and
  // the block barrier after it
  auto issue_ez = [&](int k, unsigned mw) {
    const int s = (k - kstart) & 1;
    const long long g = inq ? gidx(k) : 0;
    const int o = row * kSX + 4 * q;
    cp16_or_zero(S.ez(s) + o, a.in[kEZ] + g, has(mw, kEZ));
    cp16_or_zero(S.co(s, kHX) + o, a.co.ua[kHX] + g, has(mw, kHX));
    cp16_or_zero(S.co(s, kHY) + o, a.co.ua[kHY] + g, has(mw, kHY));
    cp16_or_zero(S.co(s, kEZ) + o, a.co.ua[kEZ] + g, has(mw, kEZ));
  };
  auto issue_hz = [&](int k, unsigned mw) {
    const int s = (k - kstart) & 1;
    const long long g = inq ? gidx(k) : 0;
    const int o = row * kSX + 4 * q;
    cp16_or_zero(S.hz(s) + o, a.in[kHZ] + g, has(mw, kHZ));
    cp16_or_zero(S.co(s, kEX) + o, a.co.ua[kEX] + g, has(mw, kEX));
    cp16_or_zero(S.co(s, kEY) + o, a.co.ua[kEY] + g, has(mw, kEY));
    cp16_or_zero(S.co(s, kHZ) + o, a.co.ua[kHZ] + g, has(mw, kHZ));
  };
  // Iteration i works on the TM half of plane i+1 and the TE half of plane
  // i; m[j] is the activity word of plane i + j. The ring holds e_z of
  // planes i+1, i+2 and h_z of planes i, i+1; after the first barrier the
  // slots read in A take e_z of i+3 and h_z of i+2 (two planes of work to
  // land). Registers: old e_x, e_y of planes i, i+1, i+2 (exA, exB, exC),
  // old h_x, h_y of plane i+1, new h_x, h_y of planes i (hxn) and i-1 (hxp),
  // and the loads of the next iteration, one iteration ahead.
  unsigned m[4];
  m[0] = 0u;  // plane kstart - 1: no TE half there
#pragma unroll
  for (int j = 1; j < 4; ++j) m[j] = kstart + j - 1 <= k1 ? word(kstart + j - 1) : 0u;
  issue_ez(kstart, m[1]);
  if (kstart + 1 < k1) issue_ez(kstart + 1, m[2]);
  cp_commit();
  Q4 exA = zero, eyA = zero;
  Q4 exB = load_if(a.in[kEX], kstart, hw(m[1], kEX)), eyB = load_if(a.in[kEY], kstart, hw(m[1], kEY));
  Q4 exC = load_if(a.in[kEX], kstart + 1, hw(m[2], kEX)), eyC = load_if(a.in[kEY], kstart + 1, hw(m[2], kEY));
  Q4 hxc = load_if(a.in[kHX], kstart, hw(m[1], kHX)), hyc = load_if(a.in[kHY], kstart, hw(m[1], kHY));
  Q4 hxp = zero, hyp = zero, hxn = zero, hyn = zero;
  const bool line_row = a.b.on && gj == a.b.j0;
  const bool line_q = line_row && a.b.i0 >= gi && a.b.i0 < gi + 4;  // the quad holds the bunch line node
  cp_wait<0>();
  __syncthreads();  // e_z of planes kstart, kstart + 1 is in

  for (int i = kstart - 1; i < k1; ++i) {
    const bool tm = i + 1 < k1;  // the TM half of plane p = i + 1 (block-uniform)
    const bool te = i >= k0;     // the TE half of plane i (block-uniform)
    const int p = i + 1;
    const int se = (p - kstart) & 1, sh = (i - kstart) & 1;
    // the next iteration's register inputs and the activity word four planes on, early
    Q4 hxn_in = zero, hyn_in = zero, exn_in = zero, eyn_in = zero;
    unsigned mn = 0u;
    if (i + 3 <= k1) {
      hxn_in = load_if(a.in[kHX], i + 2, hw(m[2], kHX));
      hyn_in = load_if(a.in[kHY], i + 2, hw(m[2], kHY));
      exn_in = load_if(a.in[kEX], i + 3, hw(m[3], kEX));
      eyn_in = load_if(a.in[kEY], i + 3, hw(m[3], kEY));
      if (i + 4 <= k1) mn = word(i + 4);
    }
    // A warp none of whose quads carries a component in a plane (PEC rows of
    // a tile at the pipe wall) computes nothing there: every value it would
    // compute is zero (an entry without a field and its coefficients hold
    // zero), so it writes zeros where its neighbours read them and keeps to
    // the barriers and the ring.
    const bool wtm = __any_sync(0xffffffffu, m[1] != 0u || line_q);
    const bool wte = __any_sync(0xffffffffu, m[0] != 0u);
    float cHX[4], cHY[4], cEZ[4], cEX[4], cEY[4], cHZ[4];
    // ---- A: S1 of plane p (hx~, hy~: U1, U2) | S4 of plane i (ex~, ey~: U6, U7)
    Q4 ez = zero, hxa = zero, hya = zero;
    if (tm) {
      if (wtm) {
        const float* sez = S.ez(se) + qo;
        ez = lds4(sez);
        const Q4 ezU = lds4(sez + kSX);
        const float ezR = sez[4];
        const Q4 c0 = lds4(S.co(se, kHX) + qo), c1 = lds4(S.co(se, kHY) + qo);
        const Q4 c2 = lds4(S.co(se, kEZ) + qo);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          cHX[e] = c0.v[e];
          cHY[e] = c1.v[e];
          cEZ[e] = c2.v[e];
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float dey = eyC.v[e] - eyB.v[e], dex = exC.v[e] - exB.v[e];
          const float ezx = e < 3 ? ez.v[e + 1] : ezR;
          hxa.v[e] = hxc.v[e] + cHX[e] * (dey - (ezU.v[e] - ez.v[e]));   // U1
          hya.v[e] = hyc.v[e] + cHY[e] * (-dex + (ezx - ez.v[e]));      // U2
        }
      }
      sts4(x1, hxa);
    }
    Q4 hz = zero, exa = zero, eya = zero;
    if (te) {
      if (wte) {
        const float* shz = S.hz(sh) + qo;
        hz = lds4(shz);
        const Q4 hzD = lds4(shz - kSX);
        const float hzL = shz[-1];
        const Q4 c0 = lds4(S.co(sh, kEX) + qo), c1 = lds4(S.co(sh, kEY) + qo);
        const Q4 c2 = lds4(S.co(sh, kHZ) + qo);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          cEX[e] = c0.v[e];
          cEY[e] = c1.v[e];
          cHZ[e] = c2.v[e];
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float hzl = e > 0 ? hz.v[e - 1] : hzL;
          exa.v[e] = exA.v[e] + cEX[e] * ((hyp.v[e] - hyn.v[e]) - (hzD.v[e] - hz.v[e]));   // U6
          eya.v[e] = eyA.v[e] + cEY[e] * (-(hxp.v[e] - hxn.v[e]) + (hzl - hz.v[e]));       // U7
        }
      }
      sts4(x3, exa);
    }
    __syncthreads();  // (1) the slots are read; hx~ and ex~ are out
    if (i + 3 < k1) issue_ez(i + 3, m[3]);  // into the freed slots
    if (i + 2 < k1) issue_hz(i + 2, m[2]);
    cp_commit();
    // ---- B: S2 of plane p (ez': U3 with the bunch current) | S5 of plane i (hz': U8)
    Q4 ezn = zero;
    if (tm) {
      if (wtm) {
        const Q4 hxaD = lds4(x1 - kSX);
        const float hyaL = left_any(hya.v[3]);
        float cur[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float hyl = e > 0 ? hya.v[e - 1] : hyaL;
          cur[e] = (hxaD.v[e] - hxa.v[e]) - (hyl - hya.v[e]);
        }
        if (line_q) {  // the bunch current on its line (one quad of a tile row)
          const long long dd = (long long)p - (a.n + a.b.kshift) + a.b.c0;
          if (dd >= -a.b.c0 && dd < a.b.c0) {
            const float jj = a.b.J[dd + a.b.c0];
#pragma unroll
            for (int e = 0; e < 4; ++e)
              if (gi + e == a.b.i0) cur[e] -= jj;
          }
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) ezn.v[e] = ez.v[e] + cEZ[e] * cur[e];   // U3
      }
      sts4(x2, ezn);
    }
    Q4 hzn = zero;
    if (te) {
      if (wte) {
        const Q4 exaU = lds4(x3 + kSX);
        const float eyaR = right_any(eya.v[0]);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float eyx = e < 3 ? eya.v[e + 1] : eyaR;
          hzn.v[e] = hz.v[e] + cHZ[e] * ((exaU.v[e] - exa.v[e]) - (eyx - eya.v[e]));      // U8
        }
      }
      sts4(x4, hzn);
    }
    cp_wait<1>();     // this thread's copies issued one iteration ago are in
    __syncthreads();  // (2) ez' and hz' are out (and the slots the next A reads are in)
    // ---- C: S3 of plane p (hx', hy': U4, U5) | S6 of plane i (ex', ey': U9, U10)
    // (hx~, ez', ex~, hz' of the thread's own quad come back from the
    // exchange buffers rather than stay in registers across the barrier)
    Q4 hxN = zero, hyN = zero;
    if (tm && wtm) {
      const Q4 hxa2 = lds4(x1);
      const Q4 ezn2 = lds4(x2);
      const Q4 eznU = lds4(x2 + kSX);
      const float eznR = right_any(ezn2.v[0]);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float dey = eyC.v[e] - eyB.v[e], dex = exC.v[e] - exB.v[e];
        const float ezx = e < 3 ? ezn2.v[e + 1] : eznR;
        hxN.v[e] = hxa2.v[e] + cHX[e] * (dey - (eznU.v[e] - ezn2.v[e]));  // U4
        hyN.v[e] = hya.v[e] + cHY[e] * (-dex + (ezx - ezn2.v[e]));      // U5
      }
      const bool st = p >= k0 && own_q;
      const unsigned ms = st ? m[1] : 0u;
      st4_if(a.out[kEZ] + gidx(p), ezn2, hw(ms, kEZ));
      st4_if(a.out[kHX] + gidx(p), hxN, hw(ms, kHX));
      st4_if(a.out[kHY] + gidx(p), hyN, hw(ms, kHY));
      if (st && line_q && a.b.i0 < L.nx) {
        const long long mm = (a.n + a.b.kshift) - p - a.b.c0;
        if (mm >= a.b.m_min && mm <= a.b.m_max) {
          const int e = a.b.i0 - gi;  // the quad's entry on the bunch line (no indexed register array)
          const float v = e == 0 ? ezn2.v[0] : e == 1 ? ezn2.v[1] : e == 2 ? ezn2.v[2] : ezn2.v[3];
          a.b.W[mm - a.b.m_min] -= (double)v * a.b.inv_q;
        }
      }
    }
    if (te && wte) {
      const Q4 exa2 = lds4(x3);
      const Q4 hzn2 = lds4(x4);
      const Q4 hznD = lds4(x4 - kSX);
      const float hznL = left_any(hzn2.v[3]);
      Q4 exn, eyn;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float hzl = e > 0 ? hzn2.v[e - 1] : hznL;
        exn.v[e] = exa2.v[e] + cEX[e] * ((hyp.v[e] - hyn.v[e]) - (hznD.v[e] - hzn2.v[e]));   // U9
        eyn.v[e] = eya.v[e] + cEY[e] * (-(hxp.v[e] - hxn.v[e]) + (hzl - hzn2.v[e]));       // U10
      }
      const unsigned ms = own_q ? m[0] : 0u;
      st4_if(a.out[kEX] + gidx(i), exn, hw(ms, kEX));
      st4_if(a.out[kEY] + gidx(i), eyn, hw(ms, kEY));
      st4_if(a.out[kHZ] + gidx(i), hzn2, hw(ms, kHZ));
    }
    // carry the z-state, take the loads made for the next iteration
    hxp = hxn;
    hyp = hyn;
    hxn = hxN;
    hyn = hyN;
    exA = exB;
    eyA = eyB;
    exB = exC;
    eyB = eyC;
    exC = exn_in;
    eyC = eyn_in;
    hxc = hxn_in;
    hyc = hyn_in;
    m[0] = m[1];
    m[1] = m[2];
    m[2] = m[3];
    m[3] = mn;
  }
  cp_wait<0>();
  __syncthreads();  // every thread is done with the ring before the next item refills it
}

template <bool MAT>
__global__ void __launch_bounds__(MAT ? kMThreads : kSThreads, MAT ? 2 : 1)
    fused_step_slab(const StepArgs<float> a, int* sched) {
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
    if constexpr (MAT)
      slab_item_mat(a, item, S);
    else
      slab_item(a, item, S);
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
// work = (member, item) pairs, the member's arguments from device memory,
// copied into shared memory for each item.
__global__ void __launch_bounds__(kSThreads, 1)
fused_step_slab_batch(const BatchMember<float>* __restrict__ members, const int2* __restrict__ work,
                      const int* __restrict__ n_work_p, int* sched) {
  using Smem = SlabSmem<false>;
  extern __shared__ __align__(128) unsigned char slab_raw[];
  Smem& S = *reinterpret_cast<Smem*>(slab_raw);
  __shared__ StepArgs<float> sargs;
  static_assert(sizeof(StepArgs<float>) % 4 == 0, "StepArgs copied as 32-bit words");
  const int tid = threadIdx.x;
  const int G = gridDim.x;
  const int n_work = *n_work_p;  // written before the launch (stream order)
  int wi = blockIdx.x, par = 0;
  while (wi < n_work) {
    if (tid == 0 && sched) S.next[par] = G + atomicAdd(sched, 1);
    const int2 w = work[wi];
    const BatchMember<float>& mb = members[w.x];
    if (mb.active) {
      // the member's arguments into shared memory once per item: the sweep
      // reads them at every plane, and from global memory (where the
      // single-solve kernel has them in its parameter space) each of those
      // reads was a load on the critical path (the batch ran 28% slower)
      {
        const unsigned* s4 = reinterpret_cast<const unsigned*>(&mb.a);
        unsigned* d4 = reinterpret_cast<unsigned*>(&sargs);
        for (int i = tid; i < (int)(sizeof(StepArgs<float>) / 4); i += kSThreads) d4[i] = s4[i];
      }
      __syncthreads();
      slab_item(sargs, w.y, S);
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

bool slab_shape_ok(int tx, int ty, bool mat) { return tx == kOX && ty == (mat ? kOYM : kOY); }

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
  constexpr int threads = MAT ? kMThreads : kSThreads, per_sm = MAT ? 2 : 1;
  fused_step_slab<MAT><<<std::min(items, per_sm * sms), threads, smem, st>>>(a, sched);
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
