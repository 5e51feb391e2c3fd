// Served mode (include/vlb.h, vlb_serve_*): cases arrive over time, wait in a
// first-come queue until their device bytes fit in the HBM budget, stay
// resident while they run, and advance together with one batched step
// (vlb_step_batch) per round; a case that has done its steps is read back
// (fields and particle state to host memory), freed, and its time to result
// recorded.  Host code only; every resident case runs on the server's one
// CUDA stream.
//
// Nothing in the round loop synchronises the device: a case's buffers come
// from the server's stream-ordered memory pool (cudaFree would synchronise),
// the host copy of its error word from a pinned arena made once (page-locked
// allocations synchronise too), the batch descriptors from one pinned
// staging block; a finished case's read-back is queued behind its last round
// into recycled pinned buffers and completed at a later poll, once its event
// has fired, so the next rounds are already on the GPU meanwhile.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <memory>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/vlb.h"
#include "vlb_internal.h"

namespace {

struct ServeCase {
  int64_t id = 0;
  vlb_params p{};
  int32_t n = 0;
  std::vector<double> xy, radius, T0, k_ratio;  // host copies until admission
  bool has_k = false;
  int64_t nsteps = 0, done_steps = 0;
  uint64_t bytes = 0;
  vlb_handle* h = nullptr;
  int32_t state = VLB_CASE_QUEUED;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  vlb_status status = VLB_OK;  // failure of a VLB_CASE_FAILED case
  std::string error;
  std::vector<double> fields;  // rho, ux, uy, T, fs planes of the last level
  std::vector<double> pstate;  // [n][9]
  // queued read-back (draining): pinned buffers, event, error-word slot
  int fbuf = -1, pbuf = -1;
  cudaEvent_t ev = nullptr;
  int err_slot = -1;
};

// A page-locked host buffer of the server's recycled set.
struct PinnedBuf {
  void* p = nullptr;
  size_t cap = 0;
  bool used = false;
};
constexpr int kErrSlots = 4096;

}  // namespace

struct vlb_server {
  vlb_serve_params sp{};
  std::string err;
  cudaStream_t stream = nullptr;
  uint64_t budget = 0, used = 0;
  int64_t next_id = 1;
  std::deque<ServeCase*> queue;
  std::vector<ServeCase*> active;
  std::vector<ServeCase*> draining;  // read-back queued, not yet complete
  cudaMemPool_t pool = nullptr;
  unsigned* err_arena = nullptr;     // kErrSlots pinned error words
  std::vector<int> free_slots;
  unsigned char* stage = nullptr;    // batch descriptor staging
  size_t stage_cap = 0;
  cudaEvent_t stage_copied = nullptr;
  std::vector<PinnedBuf> bufs;
  std::vector<cudaEvent_t> events;   // free events
  std::unordered_map<int64_t, std::unique_ptr<ServeCase>> cases;
  std::chrono::steady_clock::time_point t0;

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

static thread_local std::string g_serve_error;

static vlb_status serve_fail(vlb_server* s, vlb_status st, const std::string& m) {
  if (s) s->err = m;
  else g_serve_error = m;
  return st;
}

// A pinned buffer of at least `bytes` from the recycled set (index), or -1.
static int take_buf(vlb_server* s, size_t bytes) {
  int best = -1;
  for (int i = 0; i < (int)s->bufs.size(); ++i)
    if (!s->bufs[i].used && s->bufs[i].cap >= bytes && (best < 0 || s->bufs[i].cap < s->bufs[best].cap)) best = i;
  if (best < 0) {
    PinnedBuf b;
    b.cap = bytes < 4096 ? 4096 : bytes;
    if (cudaHostAlloc(&b.p, b.cap, cudaHostAllocDefault) != cudaSuccess) return -1;
    s->bufs.push_back(b);
    best = (int)s->bufs.size() - 1;
  }
  s->bufs[best].used = true;
  return best;
}

static void release_case_resources(vlb_server* s, ServeCase* c) {
  if (c->fbuf >= 0) s->bufs[c->fbuf].used = false;
  if (c->pbuf >= 0) s->bufs[c->pbuf].used = false;
  c->fbuf = c->pbuf = -1;
  if (c->ev) s->events.push_back(c->ev);
  c->ev = nullptr;
}

// A case that fails (its device flags stopped it, or it could not be
// placed): handle freed, budget released (finish_done below).
static void finish_done(vlb_server* s, ServeCase* c, vlb_status st, const char* msg);
static void finish(vlb_server* s, ServeCase* c, vlb_status st, const char* msg) { finish_done(s, c, st, msg); }

// Create, fill and initialise the handle of a queued case.  The initial
// state is built on the handle's own stream, so that admission does not wait
// for the round running on the server's stream; the handle then moves to it.
static vlb_status admit(vlb_server* s, ServeCase* c) {
  vlb_handle_alloc a{s->pool, nullptr};
  if (!s->free_slots.empty()) {
    c->err_slot = s->free_slots.back();
    s->free_slots.pop_back();
    a.err_host = s->err_arena + c->err_slot;
  }
  vlb_status st = vlb_create_in(&c->p, &a, &c->h);
  if (st != VLB_OK) return st;
  if (c->n > 0)
    st = vlb_add_particles(c->h, c->n, c->xy.data(), c->radius.data(), c->T0.data(),
                           c->has_k ? c->k_ratio.data() : nullptr, nullptr, nullptr);
  if (st == VLB_OK) st = vlb_step(c->h, 0);  // initial state
  if (st == VLB_OK) st = vlb_set_stream(c->h, s->stream);
  return st;
}

// A case that has done its steps: its read-back queued into pinned buffers
// behind its last round (completed by complete_draining).
static void queue_readback(vlb_server* s, ServeCase* c) {
  const size_t fbytes = 5 * (size_t)c->p.nx * c->p.ny * vlb_value_bytes(c->h);
  const size_t pbytes = 12 * (size_t)std::max(c->n, 1) * sizeof(double);
  c->fbuf = take_buf(s, fbytes);
  c->pbuf = take_buf(s, pbytes);
  if (!c->ev) {
    if (!s->events.empty()) {
      c->ev = s->events.back();
      s->events.pop_back();
    } else if (cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming) != cudaSuccess) {
      c->ev = nullptr;
    }
  }
  vlb_status st = (c->fbuf < 0 || c->pbuf < 0 || !c->ev) ? VLB_ENOMEM : VLB_OK;
  if (st == VLB_OK)
    st = vlb_readback_async(c->h, s->bufs[c->fbuf].p, static_cast<double*>(s->bufs[c->pbuf].p), c->ev);
  if (st != VLB_OK) {
    finish(s, c, st, vlb_last_error(c->h));
    return;
  }
  s->draining.push_back(c);
}

// The end of a case whose read-back has completed (or failed): handle freed
// (its buffers go back to the pool in stream order), budget released.
static void finish_done(vlb_server* s, ServeCase* c, vlb_status st, const char* msg) {
  if (st != VLB_OK) {
    c->status = st;
    c->error = msg ? msg : "";
    c->fields.clear();
    c->pstate.clear();
  }
  if (c->h) vlb_destroy(c->h);
  c->h = nullptr;
  release_case_resources(s, c);
  if (c->err_slot >= 0) s->free_slots.push_back(c->err_slot);
  c->err_slot = -1;
  s->used -= c->bytes;
  c->state = st == VLB_OK ? VLB_CASE_DONE : VLB_CASE_FAILED;
  c->t_done = s->now();
  std::vector<double>().swap(c->xy);
  std::vector<double>().swap(c->radius);
  std::vector<double>().swap(c->T0);
  std::vector<double>().swap(c->k_ratio);
}

extern "C" {

vlb_status vlb_serve_params_default(vlb_serve_params* sp) {
  if (!sp) return VLB_EINVAL;
  std::memset(sp, 0, sizeof(*sp));
  sp->steps_per_round = 100;
  return VLB_OK;
}

vlb_status vlb_serve_create(const vlb_serve_params* sp, vlb_server** out) {
  if (!out) return serve_fail(nullptr, VLB_EINVAL, "out is NULL");
  *out = nullptr;
  if (!sp) return serve_fail(nullptr, VLB_EINVAL, "params is NULL");
  if (sp->steps_per_round < 0 || sp->max_active < 0)
    return serve_fail(nullptr, VLB_EINVAL, "steps_per_round and max_active must be >= 0");
  auto* s = new (std::nothrow) vlb_server();
  if (!s) return serve_fail(nullptr, VLB_ENOMEM, "host allocation");
  s->sp = *sp;
  if (s->sp.steps_per_round == 0) s->sp.steps_per_round = 100;
  s->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  size_t free_b = 0, total_b = 0;
  if (e == cudaSuccess && sp->hbm_budget == 0) e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) {
    g_serve_error = std::string("server stream or memory query: ") + cudaGetErrorString(e);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return VLB_ECUDA;
  }
  s->budget = sp->hbm_budget ? sp->hbm_budget : free_b / 2;
  // the cases' device memory: a stream-ordered pool of this device that keeps
  // up to the budget reserved between cases
  int dev = 0;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  e = cudaGetDevice(&dev);
  props.location.id = dev;
  if (e == cudaSuccess) e = cudaMemPoolCreate(&s->pool, &props);
  if (e == cudaSuccess) {
    uint64_t keep = s->budget;
    e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&s->err_arena), kErrSlots * sizeof(unsigned),
                                          cudaHostAllocDefault);
  if (e != cudaSuccess) {
    g_serve_error = std::string("server memory pool or pinned arena: ") + cudaGetErrorString(e);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    cudaStreamDestroy(s->stream);
    delete s;
    return VLB_ECUDA;
  }
  for (int k = kErrSlots - 1; k >= 0; --k) s->free_slots.push_back(k);
  *out = s;
  return VLB_OK;
}

vlb_status vlb_serve_submit(vlb_server* s, const vlb_params* p, int32_t n, const double* xy, const double* radius,
                            const double* T0, const double* k_ratio, int64_t nsteps, int64_t* id) {
  if (!s) return VLB_EINVAL;
  if (!p || !id || n < 0 || nsteps < 0 || (n > 0 && (!xy || !radius || !T0)))
    return serve_fail(s, VLB_EINVAL, "vlb_serve_submit: arguments");
  if (n > p->max_particles) return serve_fail(s, VLB_EINVAL, "vlb_serve_submit: n > max_particles");
  auto c = std::make_unique<ServeCase>();
  vlb_status st = vlb_device_bytes(p, n, radius, &c->bytes);
  if (st != VLB_OK) return serve_fail(s, st, vlb_last_error(nullptr));
  if (c->bytes > s->budget) return serve_fail(s, VLB_ENOMEM, "vlb_serve_submit: the case alone exceeds the HBM budget");
  c->id = s->next_id++;
  c->p = *p;
  c->n = n;
  c->xy.assign(xy, xy + 2 * (size_t)n);
  c->radius.assign(radius, radius + n);
  c->T0.assign(T0, T0 + n);
  c->has_k = k_ratio != nullptr;
  if (c->has_k) c->k_ratio.assign(k_ratio, k_ratio + n);
  c->nsteps = nsteps;
  c->t_submit = s->now();
  *id = c->id;
  s->queue.push_back(c.get());
  s->cases.emplace(c->id, std::move(c));
  return VLB_OK;
}

// Complete the queued read-backs whose events have fired (all of them, in
// order, when `wait`): results to the case's host vectors, handle freed.
static void complete_draining(vlb_server* s, bool wait) {
  std::vector<ServeCase*> keep;
  for (ServeCase* c : s->draining) {
    const cudaError_t q = wait ? cudaEventSynchronize(c->ev) : cudaEventQuery(c->ev);
    if (q == cudaErrorNotReady) {
      keep.push_back(c);
      continue;
    }
    vlb_status st = q == cudaSuccess ? vlb_check_flags(c->h) : VLB_ECUDA;  // the device flags of the last steps
    const char* msg = st == VLB_OK ? nullptr : (q == cudaSuccess ? vlb_last_error(c->h) : cudaGetErrorString(q));
    if (st == VLB_OK) {
      const size_t cells = (size_t)c->p.nx * c->p.ny;
      c->fields.resize(5 * cells);
      const void* f = s->bufs[c->fbuf].p;
      if (vlb_value_bytes(c->h) == 8) std::memcpy(c->fields.data(), f, 5 * cells * sizeof(double));
      else {
        const float* ff = static_cast<const float*>(f);
        for (size_t k = 0; k < 5 * cells; ++k) c->fields[k] = ff[k];
      }
      if (c->n > 0) {
        const double* ps = static_cast<const double*>(s->bufs[c->pbuf].p);
        const size_t n = (size_t)c->n;
        c->pstate.resize(9 * n);
        const int cols[9] = {0, 1, 2, 3, 4, 5, 9, 10, 11};  // x y theta ux uy omega F_c,x F_c,y T_c
        for (size_t k = 0; k < n; ++k)
          for (int q9 = 0; q9 < 9; ++q9) c->pstate[9 * k + q9] = ps[cols[q9] * n + k];
      }
    }
    finish_done(s, c, st, msg);
  }
  s->draining.swap(keep);
}

vlb_status vlb_serve_poll(vlb_server* s, int32_t* nqueued, int32_t* nactive, int32_t* ndone) {
  if (!s) return VLB_EINVAL;
  // 0. results of earlier rounds whose read-back has arrived
  complete_draining(s, false);
  // 1. one round, queued on the server's stream: every resident case advances
  //    by the same number of steps, at most steps_per_round and at most what
  //    the nearest case still needs
  int64_t chunk = 0;
  if (!s->active.empty()) {
    chunk = s->sp.steps_per_round;
    for (ServeCase* c : s->active) chunk = std::min(chunk, c->nsteps - c->done_steps);
    std::vector<vlb_handle*> hs;
    for (;;) {
      hs.clear();
      for (ServeCase* c : s->active) hs.push_back(c->h);
      int32_t failed = -1;
      const vlb_status st = vlb_step_batch_staged(hs.data(), (int32_t)hs.size(), (int32_t)chunk, &failed, &s->stage,
                                                  &s->stage_cap, &s->stage_copied);
      if (st == VLB_OK) break;
      if (failed < 0 || st == VLB_ECUDA) return serve_fail(s, st, vlb_last_error(failed >= 0 ? hs[failed] : nullptr));
      // a case whose device flags stopped it leaves; the others have not moved
      ServeCase* c = s->active[failed];
      s->active.erase(s->active.begin() + failed);
      finish(s, c, st, vlb_last_error(c->h));
      if (s->active.empty()) break;
    }
    for (ServeCase* c : s->active) c->done_steps += chunk;
  }
  // 2. admission while the round runs, first come first served, while the
  //    bytes fit; the new cases join the next round
  std::vector<ServeCase*> admitted;
  while (!s->queue.empty()) {
    ServeCase* c = s->queue.front();
    // (cases whose read-back is still in flight are resident too)
    if (s->sp.max_active > 0 &&
        (int)(s->active.size() + s->draining.size() + admitted.size()) >= s->sp.max_active)
      break;
    if (s->used + c->bytes > s->budget) break;
    s->queue.pop_front();
    s->used += c->bytes;
    c->t_admit = s->now();
    c->state = VLB_CASE_ACTIVE;
    const vlb_status st = admit(s, c);
    if (st != VLB_OK) finish(s, c, st, c->h ? vlb_last_error(c->h) : vlb_last_error(nullptr));
    else if (c->nsteps == 0) queue_readback(s, c);
    else admitted.push_back(c);
  }
  // 3. the cases that have done their steps: read-back queued behind the round
  std::vector<ServeCase*> keep;
  for (ServeCase* c : s->active) {
    if (c->done_steps == c->nsteps) queue_readback(s, c);
    else keep.push_back(c);
  }
  for (ServeCase* c : admitted) keep.push_back(c);
  s->active.swap(keep);
  // 4. no round to run: wait for the read-backs instead of spinning
  if (s->active.empty() && !s->draining.empty()) complete_draining(s, true);
  int32_t done = 0;
  for (auto& kv : s->cases)
    if (kv.second->state == VLB_CASE_DONE || kv.second->state == VLB_CASE_FAILED) ++done;
  if (nqueued) *nqueued = (int32_t)s->queue.size();
  if (nactive) *nactive = (int32_t)(s->active.size() + s->draining.size());
  if (ndone) *ndone = done;
  return VLB_OK;
}

vlb_status vlb_serve_case_info(vlb_server* s, int64_t id, int32_t* state, int32_t* nx, int32_t* ny, int32_t* n,
                               double* times) {
  if (!s) return VLB_EINVAL;
  auto it = s->cases.find(id);
  if (it == s->cases.end()) return serve_fail(s, VLB_EINVAL, "vlb_serve_case_info: unknown case id");
  const ServeCase& c = *it->second;
  if (state) *state = c.state;
  if (nx) *nx = c.p.nx;
  if (ny) *ny = c.p.ny;
  if (n) *n = c.n;
  if (times) {
    times[0] = c.t_submit;
    times[1] = c.t_admit;
    times[2] = c.t_done;
  }
  return VLB_OK;
}

vlb_status vlb_serve_take(vlb_server* s, int64_t id, double* rho, double* ux, double* uy, double* T, double* fs,
                          double* pstate) {
  if (!s) return VLB_EINVAL;
  auto it = s->cases.find(id);
  if (it == s->cases.end()) return serve_fail(s, VLB_EINVAL, "vlb_serve_take: unknown case id");
  ServeCase& c = *it->second;
  if (c.state == VLB_CASE_FAILED) {
    const vlb_status st = c.status;
    serve_fail(s, st, c.error);
    s->cases.erase(it);
    return st;
  }
  if (c.state != VLB_CASE_DONE) return serve_fail(s, VLB_ESTATE, "vlb_serve_take: the case has not finished");
  const size_t cells = (size_t)c.p.nx * c.p.ny;
  double* out[5] = {rho, ux, uy, T, fs};
  for (int k = 0; k < 5; ++k)
    if (out[k]) std::memcpy(out[k], c.fields.data() + k * cells, cells * sizeof(double));
  if (pstate && c.n > 0) std::memcpy(pstate, c.pstate.data(), c.pstate.size() * sizeof(double));
  s->cases.erase(it);
  return VLB_OK;
}

const char* vlb_serve_last_error(const vlb_server* s) { return s ? s->err.c_str() : g_serve_error.c_str(); }

void vlb_serve_destroy(vlb_server* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (ServeCase* c : s->active)
    if (c->h) vlb_destroy(c->h);
  for (ServeCase* c : s->draining)
    if (c->h) vlb_destroy(c->h);
  if (s->stream) {
    cudaStreamSynchronize(s->stream);  // the handles' stream-ordered frees
    cudaStreamDestroy(s->stream);
  }
  for (auto& kv : s->cases)
    if (kv.second->ev) cudaEventDestroy(kv.second->ev);
  for (cudaEvent_t e : s->events) cudaEventDestroy(e);
  if (s->stage_copied) cudaEventDestroy(s->stage_copied);
  if (s->stage) cudaFreeHost(s->stage);
  for (PinnedBuf& b : s->bufs) cudaFreeHost(b.p);
  if (s->err_arena) cudaFreeHost(s->err_arena);
  if (s->pool) {
    cudaDeviceSynchronize();  // frees queued on the cases' own streams
    cudaMemPoolDestroy(s->pool);
  }
  delete s;
}

}  // extern "C"
