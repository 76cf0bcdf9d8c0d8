// Static start of the bunch (tetm_set_bunch_static): the bunch begins inside a
// uniform vacuum entry section with its head at plane K, carrying its own
// discrete TEM field, as if it had come from an infinite ingoing pipe (the
// paper's examples, Sec. 5). At c*dt = dz that field moves exactly one cell
// per step with the bunch (zero z-dispersion, Sec. 4.5), so nothing is
// radiated before the first change of cross-section.
//
// Transverse part: the potential phi on the nodes of the entry cross-section
// solves (dy/dx P_x^T P_x + dx/dy P_y^T P_y) phi = delta(i0, j0) over the
// non-PEC transverse edges, with phi = 0 on every node whose ez edge is PEC
// (a node touching a PEC cell or the wall). It is set up once per solve on the
// host (conjugate gradients in float64 on the section's few thousand to few
// hundred thousand nodes). Longitudinal part: with the line current jj(u) =
// c Q_cell(u - K + c0)/dz of edge k at step n (u = k - n), the profile G with
// G(u) + G(u+1) = 2 eta0 jj(u) and G = 0 ahead of the head gives the field
//   ex = -P_x phi G(u), ey = -P_y phi G(u)                       (time n)
//   hx = (dx/dy) P_y phi G(u+1)/eta0, hy = -(dy/dx) P_x phi G(u+1)/eta0  (n - 1/2)
// which a device kernel writes into the current field set.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "tetm_internal.h"

using namespace tetm;

namespace {

// number of activity bytes of planes 2..K that differ from plane 1 (the
// entry section must carry the same objects on every plane the initial field
// or the first steps of the bunch touch)
__global__ void count_plane_mismatch(const uint8_t* mask, Layout L, int K, unsigned long long* out) {
  const long long plane = L.sz;
  const long long total = (long long)(K - 1) * plane;
  unsigned long long c = 0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const long long k = 2 + q / plane, r = q % plane;
    c += mask[(k + 1) * plane + r] != mask[2 * plane + r];
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// Writes the TEM field of planes k = 0..K+1 (zero where G vanishes or the
// object is PEC); pxp, pyp: P_x phi, P_y phi on the (nx+1)(ny+1) nodes; G[u+1],
// u = -1..K+2.
template <typename T>
__global__ void write_tem(T* ex, T* ey, T* ez, T* hx, T* hy, T* hz, const uint8_t* mask, Layout L,
                          const double* pxp, const double* pyp, const double* G, int K, double rx,
                          double ry, double eta0) {
  const long long nxy = (long long)(L.nx + 1) * (L.ny + 1);
  const long long total = nxy * (K + 2);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(q / nxy);
    const long long t = q % nxy;
    const int i = (int)(t % (L.nx + 1)), j = (int)(t / (L.nx + 1));
    const long long id = L.idx(i, j, k);
    const uint8_t m = mask[id];
    const double g0 = G[k + 1], g1 = G[k + 2];
    ex[id] = (m & (1 << kEX)) ? (T)(-pxp[t] * g0) : T(0);
    ey[id] = (m & (1 << kEY)) ? (T)(-pyp[t] * g0) : T(0);
    ez[id] = T(0);
    hx[id] = (m & (1 << kHX)) ? (T)(rx * pyp[t] * g1 / eta0) : T(0);
    hy[id] = (m & (1 << kHY)) ? (T)(-ry * pxp[t] * g1 / eta0) : T(0);
    hz[id] = T(0);
  }
}

// Conjugate gradients for the section's potential: unknown nodes u, edges
// (a, b, w) with a or b = -1 on the wall.
void solve_potential(int n, const std::vector<int>& ea, const std::vector<int>& eb,
                     const std::vector<double>& ew, int src, std::vector<double>& x) {
  std::vector<double> r((size_t)n, 0.0), p((size_t)n, 0.0), ap((size_t)n, 0.0);
  x.assign((size_t)n, 0.0);
  r[(size_t)src] = 1.0;
  p[(size_t)src] = 1.0;
  double rr = 1.0;
  const long long iters = 20LL * n + 100;
  for (long long it = 0; it < iters && rr > 1e-30; ++it) {
    std::fill(ap.begin(), ap.end(), 0.0);
    for (size_t e = 0; e < ew.size(); ++e) {
      const int a = ea[e], b = eb[e];
      const double pa = a >= 0 ? p[(size_t)a] : 0.0, pb = b >= 0 ? p[(size_t)b] : 0.0;
      if (a >= 0) ap[(size_t)a] += ew[e] * (pa - pb);
      if (b >= 0) ap[(size_t)b] += ew[e] * (pb - pa);
    }
    double pap = 0.0;
    for (int q = 0; q < n; ++q) pap += p[(size_t)q] * ap[(size_t)q];
    const double al = rr / pap;
    double rr2 = 0.0;
    for (int q = 0; q < n; ++q) {
      x[(size_t)q] += al * p[(size_t)q];
      r[(size_t)q] -= al * ap[(size_t)q];
      rr2 += r[(size_t)q] * r[(size_t)q];
    }
    const double be = rr2 / rr;
    for (int q = 0; q < n; ++q) p[(size_t)q] = r[(size_t)q] + be * p[(size_t)q];
    rr = rr2;
  }
}

}  // namespace

extern "C" int tetm_set_bunch_static(tetm_solver* s, double sigma_z, double charge, int32_t i0,
                                     int32_t j0, int32_t k_head) {
  if (!s) return TETM_E_ARG;
  if (!s->vacuum || s->is_slab()) return TETM_E_UNSUPPORTED;
  if (s->in_batch || s->step != 0 || s->bunch) return TETM_E_STATE;
  if (!(sigma_z > 0) || !isfinite(sigma_z)) return TETM_E_ARG;
  const double dz = s->g.dz;
  const int c0 = (int)ceil(5.0 * sigma_z / dz - 1e-12);
  const int K = k_head;
  if (K < 2 * c0 + 2 || K > s->g.nz) return TETM_E_ARG;
  const Layout& L = s->L;
  cudaStream_t st = s->stream;
  // the entry section: planes 2..K carry the objects of plane 1
  unsigned long long* dcount = nullptr;
  if (dev_alloc((void**)&dcount, sizeof(unsigned long long), st) != cudaSuccess) {
    cudaGetLastError();
    return TETM_E_NOMEM;
  }
  unsigned long long mism = 0;
  cudaError_t e = cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess && K >= 2) {
    count_plane_mismatch<<<512, 256, 0, st>>>(s->mask, L, K, dcount);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&mism, dcount, sizeof(mism), cudaMemcpyDeviceToHost, st);
  // the activity bytes of plane 1 define the section
  std::vector<uint8_t> plane((size_t)L.sz);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(plane.data(), s->mask + 2 * L.sz, (size_t)L.sz, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dev_free(dcount, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TETM_E_CUDA;
  }
  if (mism) return TETM_E_ARG;
  auto bits = [&](int i, int j) -> uint8_t {
    return plane[(size_t)((j + 2) * L.px + i + L.ox)];
  };
  const int nx = s->g.nx, ny = s->g.ny;
  const long long nxy = (long long)(nx + 1) * (ny + 1);
  std::vector<int> node((size_t)nxy, -1);
  int n_unk = 0;
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i <= nx; ++i)
      if (bits(i, j) & (1 << kEZ)) node[(size_t)(i + (nx + 1) * j)] = n_unk++;
  if (i0 < 0 || i0 > nx || j0 < 0 || j0 > ny || node[(size_t)(i0 + (nx + 1) * j0)] < 0) return TETM_E_ARG;
  std::vector<int> ea, eb;
  std::vector<double> ew;
  const double wx = s->g.dy / s->g.dx, wy = s->g.dx / s->g.dy;
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      if (i < nx && (bits(i, j) & (1 << kEX))) {
        ea.push_back(node[(size_t)(i + (nx + 1) * j)]);
        eb.push_back(node[(size_t)(i + 1 + (nx + 1) * j)]);
        ew.push_back(wx);
      }
      if (j < ny && (bits(i, j) & (1 << kEY))) {
        ea.push_back(node[(size_t)(i + (nx + 1) * j)]);
        eb.push_back(node[(size_t)(i + (nx + 1) * (j + 1))]);
        ew.push_back(wy);
      }
    }
  std::vector<double> x;
  solve_potential(n_unk, ea, eb, ew, node[(size_t)(i0 + (nx + 1) * j0)], x);
  std::vector<double> pxp((size_t)nxy, 0.0), pyp((size_t)nxy, 0.0);
  auto phi = [&](int i, int j) -> double {
    const int u = node[(size_t)(i + (nx + 1) * j)];
    return u >= 0 ? x[(size_t)u] : 0.0;
  };
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      const size_t t = (size_t)(i + (nx + 1) * j);
      if (i < nx) pxp[t] = phi(i + 1, j) - phi(i, j);
      if (j < ny) pyp[t] = phi(i, j + 1) - phi(i, j);
    }
  // the bunch itself (current profile, wake window) as for a cold start
  int rc = tetm_set_bunch(s, sigma_z, charge, i0, j0);
  if (rc != TETM_OK) return rc;
  // longitudinal profile G[u + 1], u = -1 .. K + 2 (zero from u = K on)
  const double eta0 = kMu0 * kC;
  std::vector<double> G((size_t)K + 4, 0.0);
  for (int u = K - 1; u >= K - 2 * c0; --u)
    G[(size_t)u + 1] = 2.0 * eta0 * (kC * s->qcell[(size_t)(u - K + 2 * c0)] / dz) - G[(size_t)u + 2];
  double *dp = nullptr, *dq = nullptr, *dg = nullptr;
  e = dev_alloc((void**)&dp, sizeof(double) * (size_t)nxy, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&dq, sizeof(double) * (size_t)nxy, st);
  if (e == cudaSuccess) e = dev_alloc((void**)&dg, sizeof(double) * G.size(), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dp, pxp.data(), sizeof(double) * (size_t)nxy, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dq, pyp.data(), sizeof(double) * (size_t)nxy, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dg, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    void* const* f = s->set[s->cur];
    if (s->esz == 8)
      write_tem<double><<<1024, 256, 0, st>>>((double*)f[kEX], (double*)f[kEY], (double*)f[kEZ],
                                              (double*)f[kHX], (double*)f[kHY], (double*)f[kHZ], s->mask, L,
                                              dp, dq, dg, K, s->g.dx / s->g.dy, s->g.dy / s->g.dx, eta0);
    else
      write_tem<float><<<1024, 256, 0, st>>>((float*)f[kEX], (float*)f[kEY], (float*)f[kEZ],
                                             (float*)f[kHX], (float*)f[kHY], (float*)f[kHZ], s->mask, L,
                                             dp, dq, dg, K, s->g.dx / s->g.dy, s->g.dy / s->g.dx, eta0);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  dev_free(dp, st);
  dev_free(dq, st);
  dev_free(dg, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TETM_E_CUDA;
  }
  s->kshift = K;
  s->prev_valid = false;
  return TETM_OK;
}
