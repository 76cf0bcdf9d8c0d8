// Batches of solves that advance together (tetm_batch_*): one launch per step
// covers the work items of every member, so many small solves of different
// sizes fill the GPU; the member descriptors live on the device and are
// advanced there (ping-pong swap, step count, retirement at the member's step
// limit), which lets a run of steps be captured once as a CUDA graph and
// replayed. Float32 batches on the slab kernel's tile (56 x 28) run the
// batched slab kernel, the others the batched warp-tiled kernel.
//
// A batch is a table of slots. Members join and leave between step calls:
// a join writes the member's descriptor into a free slot, a
// leave clears the slot, and the combined (slot, item) work list is uploaded
// before the next step; all three are copies queued on the batch's stream
// from pinned host memory, so the host never waits for the GPU and the
// captured graph, whose launches read the descriptors, the list and its
// length from device memory, stays valid.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "tetm_internal.h"
#include <nvtx3/nvToolsExt.h>

using namespace tetm;

namespace {
constexpr int kRing = 64;    // step calls tracked by events
constexpr int kStages = 3;   // pinned staging buffers, reused round robin
constexpr int kHead = 4;     // ints ahead of the entries in the device work buffer (the count first)
constexpr size_t kStageBytes = 1u << 18;

struct Stage {
  unsigned char* host;
  size_t cap, used;
  cudaEvent_t ev;    // recorded after the latest copy out of this buffer
  bool pending;      // copies out of it may still be queued
};
}  // namespace

struct tetm_batch {
  int capacity;
  std::vector<tetm_solver*> slot;  // per slot: the member, or nullptr
  std::vector<long long> limit;    // per slot: the step index its member stops at
  size_t esz;
  int tile_x, tile_y;
  bool slab;                       // the batched slab kernel (float32, 56 x 28 tiles)
  void* d_members;                 // BatchMember<T>[capacity]
  int* d_wbuf;                     // kHead ints (entry count first), then int2 entries
  int wcap;                        // entries d_wbuf holds
  int n_work;                      // entries of the list last uploaded
  bool work_dirty;                 // membership changed since
  int nz_max;                      // transverse-wake grid bound of the launches (0: no member gathers)
  cudaStream_t stream;
  int graph_steps;                 // steps per captured graph (0 = no graph)
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  bool warmed;                     // one uncaptured launch done (launch set-up outside capture)
  bool failed;                     // a launch failed: no further steps (members resynchronised)
  int* sched;                      // the slab kernel's schedule counters
  Stage stage[kStages];
  int cur_stage;
  cudaEvent_t order_ev;            // orders the batch's stream against a member's
  cudaEvent_t ev_start[kRing], ev_end[kRing];
  long long calls, harvested;      // step calls queued / whose device time was added
  double busy_ms;
};

namespace {

size_t member_bytes(const tetm_batch* b) {
  return b->esz == 8 ? sizeof(BatchMember<double>) : sizeof(BatchMember<float>);
}

// Pinned host bytes for a copy queued on the batch's stream; a buffer is
// reused only after the copies out of it have run.
int stage_take(tetm_batch* b, size_t bytes, unsigned char** p) {
  bytes = (bytes + 15) & ~(size_t)15;
  Stage* s = &b->stage[b->cur_stage];
  if (s->used + bytes > s->cap) {
    b->cur_stage = (b->cur_stage + 1) % kStages;
    s = &b->stage[b->cur_stage];
    if (s->pending) {
      if (cudaEventSynchronize(s->ev) != cudaSuccess) return TETM_E_CUDA;
      s->pending = false;
    }
    s->used = 0;
    if (bytes > s->cap) {
      cudaFreeHost(s->host);
      s->host = nullptr;
      s->cap = 0;
      const size_t cap = std::max(bytes, 2 * kStageBytes);
      if (cudaHostAlloc((void**)&s->host, cap, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return TETM_E_NOMEM;
      }
      s->cap = cap;
    }
  }
  *p = s->host + s->used;
  s->used += bytes;
  return TETM_OK;
}

int stage_copy(tetm_batch* b, void* dst, const void* src, size_t bytes) {
  unsigned char* p = nullptr;
  const int rc = stage_take(b, bytes, &p);
  if (rc != TETM_OK) return rc;
  memcpy(p, src, bytes);
  Stage& s = b->stage[b->cur_stage];
  if (cudaMemcpyAsync(dst, p, bytes, cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
      cudaEventRecord(s.ev, b->stream) != cudaSuccess)
    return TETM_E_CUDA;
  s.pending = true;
  return TETM_OK;
}

void drop_graph(tetm_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// The combined list: (slot, item) for every item of every member below its
// limit, in slot order. Grows the device buffer when needed (the captured
// launches read it, so a new buffer means a new capture).
int upload_work(tetm_batch* b) {
  std::vector<int> h((size_t)kHead, 0);
  for (int i = 0; i < b->capacity; ++i) {
    tetm_solver* s = b->slot[(size_t)i];
    if (!s || s->step >= b->limit[(size_t)i]) continue;
    for (int item : s->work_host) {
      h.push_back(i);
      h.push_back(item);
    }
  }
  const int n = (int)((h.size() - kHead) / 2);
  if (n > b->wcap) {
    const int cap = std::max(n, 2 * b->wcap);
    int* nb = nullptr;
    if (dev_alloc((void**)&nb, sizeof(int) * ((size_t)kHead + 2 * (size_t)cap), b->stream) != cudaSuccess) {
      cudaGetLastError();
      return TETM_E_NOMEM;
    }
    dev_free(b->d_wbuf, b->stream);  // after the launches queued so far
    b->d_wbuf = nb;
    b->wcap = cap;
    drop_graph(b);
  }
  h[0] = n;
  const int rc = stage_copy(b, b->d_wbuf, h.data(), sizeof(int) * h.size());
  if (rc != TETM_OK) return rc;
  b->n_work = n;
  b->work_dirty = false;
  return TETM_OK;
}

template <typename T>
cudaError_t launch_one(tetm_batch* b) {
  const int2* work = reinterpret_cast<const int2*>(b->d_wbuf + kHead);
  if constexpr (sizeof(T) == 4) {
    if (b->slab)
      return launch_fused_slab_batch((BatchMember<float>*)b->d_members, b->capacity, work, b->d_wbuf,
                                     b->wcap, b->sched, b->nz_max, b->stream);
  }
  return launch_fused_warp_batch<T>((const BatchMember<T>*)b->d_members, b->capacity, work, b->d_wbuf, b->wcap,
                                    b->tile_y, b->nz_max, b->stream);
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
  const size_t n = (size_t)b->capacity;
  std::vector<BatchMember<T>> h(n);
  if (cudaStreamSynchronize(b->stream) != cudaSuccess ||
      cudaMemcpy(h.data(), b->d_members, sizeof(BatchMember<T>) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return;  // the context is lost: nothing on the device can be read
  }
  for (size_t i = 0; i < n; ++i) {
    tetm_solver* s = b->slot[i];
    if (!s) continue;
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

// adds the device time of tracked step calls up to index `upto` (waiting for
// them), then of any later ones already finished
int harvest(tetm_batch* b, long long upto) {
  for (; b->harvested < b->calls; ++b->harvested) {
    const int r = (int)(b->harvested % kRing);
    if (b->harvested < upto) {
      if (cudaEventSynchronize(b->ev_end[r]) != cudaSuccess) return TETM_E_CUDA;
    } else {
      const cudaError_t q = cudaEventQuery(b->ev_end[r]);
      if (q == cudaErrorNotReady) {
        cudaGetLastError();
        break;
      }
      if (q != cudaSuccess) return TETM_E_CUDA;
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->ev_start[r], b->ev_end[r]) == cudaSuccess) b->busy_ms += ms;
    cudaGetLastError();
  }
  return TETM_OK;
}

void release(tetm_batch* b) {
  drop_graph(b);
  if (b->stream) {
    dev_free(b->d_members, b->stream);
    dev_free(b->d_wbuf, b->stream);
    dev_free(b->sched, b->stream);
    cudaStreamSynchronize(b->stream);
  }
  for (Stage& s : b->stage) {
    if (s.host) cudaFreeHost(s.host);
    if (s.ev) cudaEventDestroy(s.ev);
  }
  for (int r = 0; r < kRing; ++r) {
    if (b->ev_start[r]) cudaEventDestroy(b->ev_start[r]);
    if (b->ev_end[r]) cudaEventDestroy(b->ev_end[r]);
  }
  if (b->order_ev) cudaEventDestroy(b->order_ev);
  if (b->stream) cudaStreamDestroy(b->stream);
  for (tetm_solver* s : b->slot)
    if (s) s->in_batch = false;
}

int create_slots(int capacity, size_t esz, int tile_x, int tile_y, int graph_steps, tetm_batch** out) {
  tetm_batch* b = new (std::nothrow) tetm_batch();
  if (!b) return TETM_E_NOMEM;
  b->capacity = capacity;
  b->slot.assign((size_t)capacity, nullptr);
  b->limit.assign((size_t)capacity, 0);
  b->esz = esz;
  b->tile_x = tile_x;
  b->tile_y = tile_y;
  b->slab = esz == 4 && slab_shape_ok(tile_x, tile_y, false);
  b->graph_steps = graph_steps;
  int rc = TETM_OK;
  // a blocking stream: work the caller queues on the legacy default stream
  // (member reads such as tetm_wake) is ordered after the batch's launches
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamDefault) != cudaSuccess) rc = TETM_E_CUDA;
  if (rc == TETM_OK && cudaEventCreateWithFlags(&b->order_ev, cudaEventDisableTiming) != cudaSuccess)
    rc = TETM_E_CUDA;
  for (int r = 0; r < kRing && rc == TETM_OK; ++r)
    if (cudaEventCreate(&b->ev_start[r]) != cudaSuccess || cudaEventCreate(&b->ev_end[r]) != cudaSuccess)
      rc = TETM_E_CUDA;
  for (int k = 0; k < kStages && rc == TETM_OK; ++k) {
    Stage& s = b->stage[k];
    if (cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaHostAlloc((void**)&s.host, kStageBytes, cudaHostAllocDefault) != cudaSuccess)
      rc = TETM_E_NOMEM;
    else
      s.cap = kStageBytes;
  }
  const size_t mbytes = member_bytes(b) * (size_t)capacity;
  b->wcap = 1024;
  const size_t wbytes = sizeof(int) * ((size_t)kHead + 2 * (size_t)b->wcap);
  if (rc == TETM_OK &&
      (dev_alloc(&b->d_members, mbytes, b->stream) != cudaSuccess ||
       dev_alloc((void**)&b->d_wbuf, wbytes, b->stream) != cudaSuccess ||
       dev_alloc((void**)&b->sched, 2 * sizeof(int), b->stream) != cudaSuccess))
    rc = TETM_E_NOMEM;
  // every slot starts empty (inactive), the list empty, the counters zero
  if (rc == TETM_OK &&
      (cudaMemsetAsync(b->d_members, 0, mbytes, b->stream) != cudaSuccess ||
       cudaMemsetAsync(b->d_wbuf, 0, wbytes, b->stream) != cudaSuccess ||
       cudaMemsetAsync(b->sched, 0, 2 * sizeof(int), b->stream) != cudaSuccess))
    rc = TETM_E_CUDA;
  if (rc != TETM_OK) {
    cudaGetLastError();
    release(b);
    delete b;
    return rc;
  }
  *out = b;
  return TETM_OK;
}

int check_member(const tetm_batch* b, const tetm_solver* s) {
  if (!s || s->esz != b->esz || s->in_batch) return TETM_E_ARG;
  if (!s->uniform) return TETM_E_UNSUPPORTED;                      // the fused kernels need one material
  if (s->is_slab()) return TETM_E_UNSUPPORTED;                     // a z-slab steps between plane exchanges
  if (s->scheme != TETM_SCHEME_TETM) return TETM_E_UNSUPPORTED;    // batches run the TE/TM scheme
  return TETM_OK;
}

template <typename T>
int write_member(tetm_batch* b, int i, tetm_solver* s) {
  BatchMember<T> m;
  memset(&m, 0, sizeof(m));
  m.a = step_args<T>(s, true);
  m.a.work = nullptr;  // the batch's combined list is used instead
  m.limit = b->limit[(size_t)i];
  m.active = s->step < b->limit[(size_t)i] ? 1 : 0;
  m.cur = s->cur;
  return stage_copy(b, (char*)b->d_members + sizeof(BatchMember<T>) * (size_t)i, &m, sizeof(m));
}

int add_member(tetm_batch* b, tetm_solver* s, long long limit, int* slot_out) {
  int rc = check_member(b, s);
  if (rc != TETM_OK) return rc;
  int i = 0;
  while (i < b->capacity && b->slot[(size_t)i]) ++i;
  if (i == b->capacity) return TETM_E_STATE;
  if (s->tile_x != b->tile_x || s->tile_y != b->tile_y || s->work_dirty) {
    s->tile_x = b->tile_x;
    s->tile_y = b->tile_y;
    rc = rebuild_work(s);
    if (rc != TETM_OK) return rc;
  }
  // the batch's stream first waits for the work queued on the member's own
  // stream (its creation and set-up)
  if (cudaEventRecord(b->order_ev, s->stream) != cudaSuccess ||
      cudaStreamWaitEvent(b->stream, b->order_ev, 0) != cudaSuccess)
    return TETM_E_CUDA;
  b->limit[(size_t)i] = limit;
  rc = b->esz == 8 ? write_member<double>(b, i, s) : write_member<float>(b, i, s);
  if (rc != TETM_OK) return rc;
  b->slot[(size_t)i] = s;
  s->in_batch = true;
  b->work_dirty = true;
  if (s->bunch && s->obs_on && s->g.nz > b->nz_max) {  // a larger transverse-wake grid
    b->nz_max = s->g.nz;
    drop_graph(b);
  }
  if (slot_out) *slot_out = i;
  return TETM_OK;
}

}  // namespace

extern "C" {

int tetm_batch_create_slots(int32_t capacity, int32_t precision, int32_t tile_x, int32_t tile_y,
                            int32_t graph_steps, tetm_batch** out) {
  if (!out) return TETM_E_ARG;
  *out = nullptr;
  if (capacity < 1 || capacity > (1 << 20) || graph_steps < 0) return TETM_E_ARG;
  if (precision != TETM_FP32 && precision != TETM_FP64) return TETM_E_ARG;
  const size_t esz = precision == TETM_FP64 ? 8 : 4;
  if (!(esz == 4 && slab_shape_ok(tile_x, tile_y, false)) && !warp_shape_ok(tile_x, tile_y)) return TETM_E_ARG;
  return create_slots(capacity, esz, tile_x, tile_y, graph_steps, out);
}

int tetm_batch_create(tetm_solver* const* solvers, const int64_t* step_limits, int32_t n,
                      int32_t graph_steps, tetm_batch** out) {
  if (!out) return TETM_E_ARG;
  *out = nullptr;
  if (!solvers || n < 1 || graph_steps < 0) return TETM_E_ARG;
  const size_t esz = solvers[0] ? solvers[0]->esz : 0;
  for (int i = 0; i < n; ++i) {
    tetm_solver* s = solvers[i];
    if (!s || s->esz != esz || s->in_batch) return TETM_E_ARG;
    if (!s->uniform || s->is_slab() || s->scheme != TETM_SCHEME_TETM) return TETM_E_UNSUPPORTED;
    for (int j = 0; j < i; ++j)
      if (solvers[j] == s) return TETM_E_ARG;
  }
  // float32 members of the slab kernel's tile (the float32 default) run the
  // batched slab kernel; otherwise every member runs the warp-tiled kernel
  // with the first member's tile height
  const bool slab = esz == 4 && slab_shape_ok(solvers[0]->tile_x, solvers[0]->tile_y, false);
  const int ty = slab ? solvers[0]->tile_y : ((solvers[0]->tile_x == 28) ? solvers[0]->tile_y : 20);
  const int tx = slab ? solvers[0]->tile_x : 28;
  tetm_batch* b = nullptr;
  int rc = create_slots(n, esz, tx, ty, graph_steps, &b);
  if (rc != TETM_OK) return rc;
  for (int i = 0; i < n && rc == TETM_OK; ++i)
    rc = add_member(b, solvers[i], step_limits && step_limits[i] >= 0 ? (long long)step_limits[i] : (1LL << 62),
                    nullptr);
  if (rc == TETM_OK) rc = upload_work(b);
  if (rc == TETM_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) rc = TETM_E_CUDA;
  if (rc != TETM_OK) {
    cudaGetLastError();
    release(b);
    delete b;
    return rc;
  }
  *out = b;
  return TETM_OK;
}

int tetm_batch_add(tetm_batch* b, tetm_solver* s, int64_t step_limit, int32_t* slot) {
  if (!b) return TETM_E_ARG;
  if (b->failed) return TETM_E_STATE;
  int i = -1;
  const int rc = add_member(b, s, step_limit >= 0 ? (long long)step_limit : (1LL << 62), &i);
  if (rc == TETM_OK && slot) *slot = i;
  return rc;
}

int tetm_batch_remove(tetm_batch* b, tetm_solver* s) {
  if (!b || !s) return TETM_E_ARG;
  int i = 0;
  while (i < b->capacity && b->slot[(size_t)i] != s) ++i;
  if (i == b->capacity) return TETM_E_ARG;
  // an all-zero descriptor is an inactive slot: no launch reads past its flag
  std::vector<unsigned char> zero(member_bytes(b), 0);
  int rc = stage_copy(b, (char*)b->d_members + zero.size() * (size_t)i, zero.data(), zero.size());
  // the member's own stream waits for the batch's launches queued so far
  if (rc == TETM_OK && (cudaEventRecord(b->order_ev, b->stream) != cudaSuccess ||
                        cudaStreamWaitEvent(s->stream, b->order_ev, 0) != cudaSuccess))
    rc = TETM_E_CUDA;
  b->slot[(size_t)i] = nullptr;
  s->in_batch = false;
  b->work_dirty = true;
  return rc;
}

static int batch_step_impl(tetm_batch* b, int32_t nsteps) {
  if (!b || nsteps < 0) return TETM_E_ARG;
  if (b->failed) return TETM_E_STATE;
  if (nsteps == 0) return TETM_OK;
  if (b->calls - b->harvested >= kRing && harvest(b, b->calls - kRing + 1) != TETM_OK) return batch_fail(b);
  const int r = (int)(b->calls % kRing);
  if (cudaEventRecord(b->ev_start[r], b->stream) != cudaSuccess) return batch_fail(b);
  if (b->work_dirty) {
    const int rc = upload_work(b);
    if (rc != TETM_OK) return rc == TETM_E_NOMEM ? rc : batch_fail(b);
  }
  int left = nsteps;
  if (!b->warmed) {  // first launch outside any capture (one-time launch set-up)
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
  if (cudaEventRecord(b->ev_end[r], b->stream) != cudaSuccess) return batch_fail(b);
  ++b->calls;
  // mirror the device-side advance in the members' host bookkeeping
  for (int i = 0; i < b->capacity; ++i) {
    tetm_solver* s = b->slot[(size_t)i];
    if (!s) continue;
    const long long taken = std::max(0LL, std::min((long long)nsteps, b->limit[(size_t)i] - s->step));
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

int tetm_batch_wait(tetm_batch* b, int32_t max_pending, double* busy_s) {
  if (!b || max_pending < 0) return TETM_E_ARG;
  const int rc = harvest(b, b->calls - max_pending);
  if (busy_s) *busy_s = 1e-3 * b->busy_ms;
  return rc;
}

int tetm_batch_sync(tetm_batch* b) {
  if (!b) return TETM_E_ARG;
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TETM_E_CUDA;
  if (harvest(b, b->calls) != TETM_OK) return TETM_E_CUDA;
  return TETM_OK;
}

int tetm_batch_info(tetm_batch* b, int32_t* n_members, int32_t* n_active, int32_t* work_items) {
  if (!b) return TETM_E_ARG;
  int mem = 0, act = 0;
  for (int i = 0; i < b->capacity; ++i) {
    tetm_solver* s = b->slot[(size_t)i];
    if (!s) continue;
    ++mem;
    if (s->step < b->limit[(size_t)i]) ++act;
  }
  if (n_members) *n_members = mem;
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
