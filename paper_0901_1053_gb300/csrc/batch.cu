// Batches of solves that advance together (tetm_batch_*): one launch per step
// covers the work items of every member, so many small solves of different
// sizes fill the GPU; the member descriptors live on the device and are
// advanced there (ping-pong swap, step count, retirement at the member's step
// limit), which lets a run of steps be captured once as a CUDA graph and
// replayed. Float32 batches whose members use the slab kernel's tile (56 x 28)
// run the batched slab kernel (each member's tensor maps in device memory),
// the others the batched warp-tiled kernel.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "tetm_internal.h"
#include <nvtx3/nvToolsExt.h>

using namespace tetm;

struct tetm_batch {
  std::vector<tetm_solver*> members;
  std::vector<long long> limit;   // per member: step index it stops at
  size_t esz;
  int tile_y;
  void* d_members;                // BatchMember<T>[n]
  int2* d_work;
  int n_work;
  cudaStream_t stream;
  bool own_stream;
  int graph_steps;                // steps per captured graph (0 = no graph)
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  bool warmed;                    // one uncaptured launch done (launch set-up outside capture)
  bool failed;                    // a launch failed: no further steps (members resynchronised)
  bool slab;                      // the batched slab kernel (float32, 56 x 28 tiles)
  SlabBatchMaps* d_maps;          // per member (slab batches)
  int* sched;                     // the slab kernel's schedule counters
  int* err;                       // the slab kernel's bounded-wait error word
};

namespace {

template <typename T>
int build_members(tetm_batch* b) {
  const int n = (int)b->members.size();
  std::vector<BatchMember<T>> h((size_t)n);
  std::vector<int2> work;
  for (int i = 0; i < n; ++i) {
    tetm_solver* s = b->members[(size_t)i];
    memset(&h[(size_t)i], 0, sizeof(BatchMember<T>));
    h[(size_t)i].a = step_args<T>(s, true);
    h[(size_t)i].a.work = nullptr;  // the batch's combined list is used instead
    h[(size_t)i].limit = b->limit[(size_t)i];
    h[(size_t)i].active = s->step < b->limit[(size_t)i] ? 1 : 0;
    h[(size_t)i].cur = s->cur;
    for (int item : s->work_host) work.push_back(make_int2(i, item));
  }
  b->n_work = (int)work.size();
  if (cudaMalloc(&b->d_members, sizeof(BatchMember<T>) * (size_t)n) != cudaSuccess) return TETM_E_NOMEM;
  if (!work.empty() && cudaMalloc(&b->d_work, sizeof(int2) * work.size()) != cudaSuccess)
    return TETM_E_NOMEM;
  if (cudaMemcpyAsync(b->d_members, h.data(), sizeof(BatchMember<T>) * (size_t)n,
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return TETM_E_CUDA;
  if (!work.empty() && cudaMemcpyAsync(b->d_work, work.data(), sizeof(int2) * work.size(),
                                       cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return TETM_E_CUDA;
  if (b->slab) {  // each member's tensor maps of e_z, h_z of both sets
    std::vector<SlabBatchMaps> hm((size_t)n);
    for (int i = 0; i < n; ++i) {
      tetm_solver* s = b->members[(size_t)i];
      SlabMaps m;
      void* ez[2] = {s->set[0][kEZ], s->set[1][kEZ]};
      void* hz[2] = {s->set[0][kHZ], s->set[1][kHZ]};
      if (build_slab_maps(&m, ez, hz, nullptr, s->L) != 0) return TETM_E_UNSUPPORTED;
      memcpy(hm[(size_t)i].ez, m.ez, sizeof(m.ez));
      memcpy(hm[(size_t)i].hz, m.hz, sizeof(m.hz));
    }
    if (cudaMalloc(&b->d_maps, sizeof(SlabBatchMaps) * (size_t)n) != cudaSuccess ||
        cudaMalloc(&b->sched, 2 * sizeof(int)) != cudaSuccess || cudaMalloc(&b->err, sizeof(int)) != cudaSuccess)
      return TETM_E_NOMEM;
    if (cudaMemcpy(b->d_maps, hm.data(), sizeof(SlabBatchMaps) * (size_t)n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->sched, 0, 2 * sizeof(int)) != cudaSuccess || cudaMemset(b->err, 0, sizeof(int)) != cudaSuccess)
      return TETM_E_CUDA;
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TETM_E_CUDA;
  return TETM_OK;
}

template <typename T>
cudaError_t launch_one(tetm_batch* b) {
  int nz_max = 0;  // over the members that gather a transverse wake
  for (tetm_solver* s : b->members)
    if (s->bunch && s->obs_on) nz_max = std::max(nz_max, s->g.nz);
  if constexpr (sizeof(T) == 4) {
    if (b->slab)
      return launch_fused_slab_batch((BatchMember<float>*)b->d_members, b->d_maps, (int)b->members.size(),
                                     b->d_work, b->n_work, b->err, b->sched, nz_max, b->stream);
  }
  return launch_fused_warp_batch<T>((const BatchMember<T>*)b->d_members, (int)b->members.size(),
                                    b->d_work, b->n_work, b->tile_y, nz_max, b->stream);
}

cudaError_t launch_one_any(tetm_batch* b) {
  return b->esz == 8 ? launch_one<double>(b) : launch_one<float>(b);
}

// After a failed launch the members' host bookkeeping (step, current field
// set) may lag the device, where some launches did advance them: read each
// member's descriptor back and take its step and current set from there.
template <typename T>
void resync_members(tetm_batch* b) {
  cudaGetLastError();
  const size_t n = b->members.size();
  std::vector<BatchMember<T>> h(n);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess ||
      cudaMemcpy(h.data(), b->d_members, sizeof(BatchMember<T>) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return;  // the context is lost: nothing on the device can be read
  }
  for (size_t i = 0; i < n; ++i) {
    tetm_solver* s = b->members[i];
    if (h[i].a.n != s->step) s->prev_valid = true;
    s->step = h[i].a.n;
    s->cur = (const void*)h[i].a.in[0] == s->set[1][0] ? 1 : 0;
  }
}
int batch_fail(tetm_batch* b) {
  b->failed = true;
  if (b->esz == 8)
    resync_members<double>(b);
  else
    resync_members<float>(b);
  return TETM_E_CUDA;
}

void release(tetm_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->d_members);
  cudaFree(b->d_work);
  cudaFree(b->d_maps);
  cudaFree(b->sched);
  cudaFree(b->err);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  for (tetm_solver* s : b->members) s->in_batch = false;
}

}  // namespace

extern "C" {

int tetm_batch_create(tetm_solver* const* solvers, const int64_t* step_limits, int32_t n,
                      int32_t graph_steps, tetm_batch** out) {
  if (!out) return TETM_E_ARG;
  *out = nullptr;
  if (!solvers || n < 1 || graph_steps < 0) return TETM_E_ARG;
  const size_t esz = solvers[0] ? solvers[0]->esz : 0;
  for (int i = 0; i < n; ++i) {
    tetm_solver* s = solvers[i];
    if (!s || s->esz != esz || s->in_batch) return TETM_E_ARG;
    if (!s->uniform) return TETM_E_UNSUPPORTED;  // the fused kernels need one material
    if (s->is_slab()) return TETM_E_UNSUPPORTED;     // a z-slab steps between plane exchanges
    if (s->scheme != TETM_SCHEME_TETM) return TETM_E_UNSUPPORTED;  // batches run the TE/TM scheme
    for (int j = 0; j < i; ++j)
      if (solvers[j] == s) return TETM_E_ARG;
  }
  tetm_batch* b = new (std::nothrow) tetm_batch();
  if (!b) return TETM_E_NOMEM;
  b->esz = esz;
  b->graph_steps = graph_steps;
  // float32 members of the slab kernel's tile (the float32 default) run the
  // batched slab kernel; otherwise every member runs the warp-tiled kernel
  // with the first member's tile height
  b->slab = esz == 4 && slab_shape_ok(solvers[0]->tile_x, solvers[0]->tile_y);
  b->tile_y = b->slab ? solvers[0]->tile_y : ((solvers[0]->tile_x == 28) ? solvers[0]->tile_y : 20);
  const int tx = b->slab ? solvers[0]->tile_x : 28;
  int rc = TETM_OK;
  for (int i = 0; i < n && rc == TETM_OK; ++i) {
    tetm_solver* s = solvers[i];
    b->members.push_back(s);
    b->limit.push_back(step_limits && step_limits[i] >= 0 ? (long long)step_limits[i] : (1LL << 62));
    if (s->tile_x != tx || s->tile_y != b->tile_y || s->work_dirty) {
      s->tile_x = tx;
      s->tile_y = b->tile_y;
      rc = rebuild_work(s);
    }
  }
  if (rc == TETM_OK) {
    // a blocking stream: work the caller queues on the legacy default stream
    // (member reads such as tetm_wake) is ordered after the batch's launches
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamDefault) != cudaSuccess) rc = TETM_E_CUDA;
    b->own_stream = true;
  }
  // the members' queued work must be done before the batch reads their state
  for (int i = 0; i < n && rc == TETM_OK; ++i)
    if (cudaStreamSynchronize(solvers[i]->stream) != cudaSuccess) rc = TETM_E_CUDA;
  if (rc == TETM_OK) rc = esz == 8 ? build_members<double>(b) : build_members<float>(b);
  if (rc != TETM_OK) {
    release(b);
    delete b;
    cudaGetLastError();
    return rc;
  }
  for (tetm_solver* s : b->members) s->in_batch = true;
  *out = b;
  return TETM_OK;
}

static int batch_step_impl(tetm_batch* b, int32_t nsteps) {
  if (!b || nsteps < 0) return TETM_E_ARG;
  if (b->failed) return TETM_E_STATE;
  int left = nsteps;
  if (left > 0 && !b->warmed) {  // first launch outside any capture (one-time launch set-up)
    if (launch_one_any(b) != cudaSuccess) return batch_fail(b);
    b->warmed = true;
    --left;
  }
  if (b->graph_steps > 0 && left >= b->graph_steps) {
    if (!b->exec) {
      if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return batch_fail(b);
      cudaError_t e = cudaSuccess;
      for (int q = 0; q < b->graph_steps && e == cudaSuccess; ++q) e = launch_one_any(b);
      cudaError_t e2 = cudaStreamEndCapture(b->stream, &b->graph);
      if (e != cudaSuccess || e2 != cudaSuccess) return batch_fail(b);
      if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) return batch_fail(b);
    }
    while (left >= b->graph_steps) {
      if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return batch_fail(b);
      left -= b->graph_steps;
    }
  }
  for (; left > 0; --left)
    if (launch_one_any(b) != cudaSuccess) return batch_fail(b);
  // mirror the device-side advance in the members' host bookkeeping
  for (size_t i = 0; i < b->members.size(); ++i) {
    tetm_solver* s = b->members[i];
    const long long taken = std::max(0LL, std::min((long long)nsteps, b->limit[i] - s->step));
    s->step += taken;
    if (taken & 1) s->cur = 1 - s->cur;
    if (taken > 0) s->prev_valid = true;
  }
  return TETM_OK;
}

int tetm_batch_step(tetm_batch* b, int32_t nsteps) {
  nvtxRangePushA("tetm_batch_step");
  const int rc = batch_step_impl(b, nsteps);
  nvtxRangePop();
  return rc;
}

int tetm_batch_sync(tetm_batch* b) {
  if (!b) return TETM_E_ARG;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TETM_E_CUDA;
  if (b->err) {  // a bounded wait of the slab kernel gave up
    int flag = 0;
    if (cudaMemcpy(&flag, b->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return TETM_E_CUDA;
    if (flag) return TETM_E_TIMEOUT;
  }
  return TETM_OK;
}

int tetm_batch_info(tetm_batch* b, int32_t* n_members, int32_t* n_active, int32_t* work_items) {
  if (!b) return TETM_E_ARG;
  int act = 0;
  for (size_t i = 0; i < b->members.size(); ++i)
    if (b->members[i]->step < b->limit[i]) ++act;
  if (n_members) *n_members = (int32_t)b->members.size();
  if (n_active) *n_active = act;
  if (work_items) *work_items = b->n_work;
  return TETM_OK;
}

void tetm_batch_destroy(tetm_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  release(b);
  delete b;
}

}  // extern "C"
