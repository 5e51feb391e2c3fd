// Served mode (include/vlb.h, vlb_serve_*): cases arrive over time, wait in a
// first-come queue until their device bytes fit in the HBM budget, stay
// resident while they run, and advance together with one batched step
// (vlb_step_batch) per round; a case that has done its steps is read back
// (fields and particle state to host memory), freed, and its time to result
// recorded.  Host code only, on top of the library's public calls; every
// resident case runs on the server's one CUDA stream.
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
};

}  // namespace

struct vlb_server {
  vlb_serve_params sp{};
  std::string err;
  cudaStream_t stream = nullptr;
  uint64_t budget = 0, used = 0;
  int64_t next_id = 1;
  std::deque<ServeCase*> queue;
  std::vector<ServeCase*> active;
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

// A case stops: read back its result (on success), free its handle and budget.
static void finish(vlb_server* s, ServeCase* c, vlb_status st, const char* msg) {
  if (st == VLB_OK) {
    const size_t cells = (size_t)c->p.nx * c->p.ny;
    c->fields.assign(5 * cells, 0.0);
    double* f = c->fields.data();
    const uint32_t all = VLB_FIELD_RHO | VLB_FIELD_UX | VLB_FIELD_UY | VLB_FIELD_T | VLB_FIELD_FS;
    st = vlb_get_fields(c->h, all, f, f + cells, f + 2 * cells, f + 3 * cells, f + 4 * cells);
    if (st == VLB_OK && c->n > 0) {
      std::vector<double> xy(2 * c->n), th(c->n), uv(2 * c->n), om(c->n), fo(2 * c->n), to(c->n);
      st = vlb_get_particle_state(c->h, c->n, xy.data(), th.data(), uv.data(), om.data(), fo.data(), to.data());
      c->pstate.resize((size_t)9 * c->n);
      for (int k = 0; k < c->n; ++k) {
        double* r = c->pstate.data() + 9 * (size_t)k;
        r[0] = xy[2 * k]; r[1] = xy[2 * k + 1]; r[2] = th[k]; r[3] = uv[2 * k]; r[4] = uv[2 * k + 1];
        r[5] = om[k]; r[6] = fo[2 * k]; r[7] = fo[2 * k + 1]; r[8] = to[k];
      }
    }
    if (st != VLB_OK) msg = vlb_last_error(c->h);
  }
  if (st != VLB_OK) {
    c->status = st;
    c->error = msg ? msg : "";
    c->fields.clear();
    c->pstate.clear();
  }
  if (c->h) vlb_destroy(c->h);
  c->h = nullptr;
  s->used -= c->bytes;
  c->state = st == VLB_OK ? VLB_CASE_DONE : VLB_CASE_FAILED;
  c->t_done = s->now();
  // host copies of the inputs are no longer needed
  std::vector<double>().swap(c->xy);
  std::vector<double>().swap(c->radius);
  std::vector<double>().swap(c->T0);
  std::vector<double>().swap(c->k_ratio);
}

// Create, fill and initialise the handle of a queued case.  The initial
// state is built on the handle's own stream, so that admission does not wait
// for the round running on the server's stream; the handle then moves to it.
static vlb_status admit(vlb_server* s, ServeCase* c) {
  vlb_status st = vlb_create(&c->p, &c->h);
  if (st != VLB_OK) return st;
  if (c->n > 0)
    st = vlb_add_particles(c->h, c->n, c->xy.data(), c->radius.data(), c->T0.data(),
                           c->has_k ? c->k_ratio.data() : nullptr, nullptr, nullptr);
  if (st == VLB_OK) st = vlb_step(c->h, 0);  // initial state
  if (st == VLB_OK) st = vlb_set_stream(c->h, s->stream);
  return st;
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

vlb_status vlb_serve_poll(vlb_server* s, int32_t* nqueued, int32_t* nactive, int32_t* ndone) {
  if (!s) return VLB_EINVAL;
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
      const vlb_status st = vlb_step_batch(hs.data(), (int32_t)hs.size(), (int32_t)chunk, &failed);
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
    if (s->sp.max_active > 0 && (int)(s->active.size() + admitted.size()) >= s->sp.max_active) break;
    if (s->used + c->bytes > s->budget) break;
    s->queue.pop_front();
    s->used += c->bytes;
    c->t_admit = s->now();
    c->state = VLB_CASE_ACTIVE;
    const vlb_status st = admit(s, c);
    if (st != VLB_OK) finish(s, c, st, c->h ? vlb_last_error(c->h) : vlb_last_error(nullptr));
    else if (c->nsteps == 0) finish(s, c, VLB_OK, nullptr);
    else admitted.push_back(c);
  }
  // 3. the cases that have done their steps: results to host, then freed
  std::vector<ServeCase*> keep;
  for (ServeCase* c : s->active) {
    if (c->done_steps == c->nsteps) finish(s, c, VLB_OK, nullptr);
    else keep.push_back(c);
  }
  for (ServeCase* c : admitted) keep.push_back(c);
  s->active.swap(keep);
  int32_t done = 0;
  for (auto& kv : s->cases)
    if (kv.second->state == VLB_CASE_DONE || kv.second->state == VLB_CASE_FAILED) ++done;
  if (nqueued) *nqueued = (int32_t)s->queue.size();
  if (nactive) *nactive = (int32_t)s->active.size();
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
  for (ServeCase* c : s->active)
    if (c->h) vlb_destroy(c->h);
  if (s->stream) {
    cudaStreamSynchronize(s->stream);
    cudaStreamDestroy(s->stream);
  }
  delete s;
}

}  // extern "C"
