// memd_server.cu -- a request server over batched MEMD systems.
//
// Requests (a system and a number of steps) queue in arrival order.  Each
// call to memd_server_pump is one scheduling round: finished requests are
// retired (their results copied to host memory, their device memory
// released), queued requests are admitted while the device-memory budget and
// the slot count allow (FIFO, so a large request is not overtaken), the
// batch of live systems is rebuilt when membership changed, and the batch
// advances by one quantum of steps (or less, so that no request overshoots
// its step count).  Requests that arrive while others run join at the next
// round: their work shares every kernel launch with the systems already
// resident, which is continuous batching.  Each request's result is the
// same as when it runs alone (the batched kernels are the single-system
// kernels over a descriptor table).
//
// Admission (create: permittivity, Green's table, effective permittivity;
// init: Gauss scan and initial solve) runs on a few worker threads, each with
// its own CUDA stream, beside the batch stepping on the server's stream; a
// set-up system moves to the server's stream and joins the batch at the
// next round after its setup has finished.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "memd.h"
#include "memd_ctx.cuh"
#include "memd_internal.cuh"

struct memd_server {
  memd_server_options opt{};
  struct Req {
    int64_t id = 0;
    int32_t mesh[3] = {0, 0, 0};
    double box[3] = {0, 0, 0};
    int32_t eps_kind = 0, eps_axis = 0;
    std::vector<double> eps_values;
    double eps_params[8] = {0};
    double c_light = 1, dt = 0.01;
    std::vector<double> pos, mass, vel;
    std::vector<int32_t> q;
    uint64_t seed = 0;
    int64_t nsteps = 0, remaining = 0;
    int64_t footprint = 0;
    int32_t state = MEMD_REQ_QUEUED;
    memd_ctx* ctx = nullptr;
    // results
    std::vector<double> r_pos, r_vel, r_f;
    std::vector<int32_t> r_img;
    memd_energy_terms r_e{};
    std::string error;
  };
  std::map<int64_t, Req> reqs;
  std::deque<int64_t> queue;
  std::vector<int64_t> active;
  int64_t next_id = 1;
  int64_t used = 0;
  memd_batch* batch = nullptr;
  bool dirty = false;
  std::string last_error;
  memd_server_stats stats{};
  // admission workers: requests handed over (todo), set up (ready)
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> wstreams;
  std::mutex mu;
  std::condition_variable cv_todo, cv_ready;
  std::deque<Req*> todo;
  std::vector<std::pair<Req*, memd_status>> ready;
  int in_flight = 0;
  bool stop = false;
  bool own_stream = false;  // the server created opt.cuda_stream
  // an event pair around every quantum (added to step_gpu_s once both have
  // completed), the end of the latest quantum (ev_done), the event pairs free
  // for reuse; results of leaving requests are copied on rstream
  std::deque<std::pair<cudaEvent_t, cudaEvent_t>> timed, spare;
  cudaEvent_t ev_done = nullptr;
  cudaStream_t rstream = nullptr;
  bool any_launched = false;
};

constexpr int kAdmitWorkers = 3;  // concurrent setups unless the options say otherwise

namespace {

// device bytes a request holds while resident: double-buffered D and B,
// 1/eps in the field precision and in FP64, the int64 ledger and transfer
// buffer, particle arrays, plus the setup's multigrid scratch (released
// after init but needed at admission; the workers solve the cell problems
// in turn, one solver)
int64_t footprint(const memd_server_options& o, const memd_server::Req& r) {
  const int64_t V = (int64_t)r.mesh[0] * r.mesh[1] * r.mesh[2];
  const int64_t es = o.precision == MEMD_FP32 ? 4 : 8;
  // D, B (two parities each) and 1/eps in field precision; 1/eps FP64, the
  // ledger, the transfer buffer and the cell-problem potentials (8 B each)
  const int64_t fields = 3 * V * (5 * es + 8 + 16 + 8);
  const int64_t init = 3 * V * 8 * 7 + V * 16;
  const int64_t parts = (r.q.size() + 1) * (8 * 3 * 5 + 8 * 4 + 4 * 4 + 36);
  return fields + init + parts + (1 << 20);
}

memd_status sfail(memd_server* s, memd_status st, const std::string& why) {
  if (s) s->last_error = why;
  return st;
}

void retire(memd_server* s, memd_server::Req& r) {
  memd_ctx* c = r.ctx;
  const size_t n = r.q.size();
  r.r_pos.resize(3 * n);
  r.r_vel.resize(3 * n);
  r.r_f.resize(3 * n);
  r.r_img.resize(3 * n);
  memd_status st = memd_get_particles(c, n ? r.r_pos.data() : nullptr, n ? r.r_vel.data() : nullptr,
                                      n ? r.r_img.data() : nullptr);
  if (st == MEMD_OK && n) st = memd_forces(c, r.r_f.data());
  if (st == MEMD_OK) st = memd_energy(c, &r.r_e);
  if (st != MEMD_OK) {
    r.state = MEMD_REQ_FAILED;
    r.error = memd_last_error(c);
  } else {
    r.state = MEMD_REQ_DONE;
  }
  memd_destroy(c);
  r.ctx = nullptr;
  s->used -= r.footprint;
  r.pos.clear();
  r.vel.clear();
  r.mass.clear();
  r.eps_values.clear();
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// One request's setup on a worker's stream; the finished context is then
// moved to the server's stream (its setup work has completed).
memd_status admit(memd_server* s, memd_server::Req& r, cudaStream_t wst) {
  const double t0 = now_s();
  struct Timer {
    memd_server* s;
    double t0;
    ~Timer() {
      std::lock_guard<std::mutex> g(s->mu);
      s->stats.setup_s += now_s() - t0;
      s->stats.admitted += 1;
    }
  } timer{s, t0};
  memd_options o;
  memd_default_options(&o);
  o.precision = s->opt.precision;
  o.cuda_stream = wst;
  o.device = s->opt.device;
  o.alloc = s->opt.alloc;
  o.free = s->opt.free;
  o.alloc_user = s->opt.alloc_user;
  o.seed = r.seed;
  o.field_kernel = MEMD_FIELD_LDG;  // the batched kernels' arithmetic
  memd_eps_profile e{};
  e.kind = r.eps_kind;
  e.axis = r.eps_axis;
  e.values = r.eps_values.empty() ? nullptr : r.eps_values.data();
  std::memcpy(e.params, r.eps_params, sizeof(e.params));
  memd_status st = memd_create(r.mesh, r.box, &e, r.c_light, r.dt, &o, &r.ctx);
  if (st == MEMD_OK) {
    const int64_t n = (int64_t)r.q.size();
    st = memd_init_field(r.ctx, n, n ? r.pos.data() : nullptr, n ? r.q.data() : nullptr,
                         r.mass.empty() ? nullptr : r.mass.data(),
                         r.vel.empty() ? nullptr : r.vel.data());
    if (st == MEMD_OK && cudaStreamSynchronize(wst) != cudaSuccess) st = MEMD_ERR_CUDA;
    if (st != MEMD_OK) {
      r.error = memd_last_error(r.ctx);
      memd_destroy(r.ctx);
      r.ctx = nullptr;
    } else {
      r.ctx->stream = (cudaStream_t)s->opt.cuda_stream;
    }
  } else {
    r.error = std::string("memd_create: ") + memd_status_string(st);
  }
  return st;
}

void worker(memd_server* s, int w) {
  cudaSetDevice(s->opt.device);  // resolved at create
  // several workers already set systems up at once: each solves a system's
  // cell problems in turn (three at once per worker slowed the served
  // stream: p50 1.2-1.35 s -> 1.8-2.05 s)
  memd::memd_mg_cells_in_turn(true);
  for (;;) {
    memd_server::Req* r = nullptr;
    {
      std::unique_lock<std::mutex> g(s->mu);
      s->cv_todo.wait(g, [&] { return s->stop || !s->todo.empty(); });
      if (s->stop && s->todo.empty()) return;
      r = s->todo.front();
      s->todo.pop_front();
    }
    memd_status st;
    {
      memd::NvtxRange nvtx_("request setup");
      st = admit(s, *r, s->wstreams[w]);
    }
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->ready.emplace_back(r, st);
      s->in_flight -= 1;
    }
    s->cv_ready.notify_all();
  }
}

memd_status start_workers(memd_server* s) {
  if (!s->workers.empty()) return MEMD_OK;
  int dev = s->opt.device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return MEMD_ERR_CUDA;
  s->opt.device = dev;
  const int nw = s->opt.admission_workers > 0 ? s->opt.admission_workers : kAdmitWorkers;
  // setup runs many small, latency-bound kernels (multigrid levels, scans);
  // on streams of the highest priority their blocks are scheduled ahead of
  // the batch's waiting tiles instead of queueing behind a whole step
  int lo = 0, hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) {
    cudaGetLastError();
    lo = hi = 0;
  }
  for (int w = 0; w < nw; ++w) {
    cudaStream_t st;
    if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, hi) != cudaSuccess)
      return MEMD_ERR_CUDA;
    s->wstreams.push_back(st);
  }
  // as many workers as threads can be started (no exception leaves the C ABI)
  for (int w = 0; w < nw; ++w) {
    try {
      s->workers.emplace_back(worker, s, w);
    } catch (...) {
      break;
    }
  }
  return s->workers.empty() ? MEMD_ERR_OOM : MEMD_OK;
}

void stop_workers(memd_server* s) {
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    s->todo.clear();  // requests not yet started stay queued
  }
  s->cv_todo.notify_all();
  for (auto& t : s->workers) t.join();
  s->workers.clear();
  for (cudaStream_t st : s->wstreams) cudaStreamDestroy(st);
  s->wstreams.clear();
}

}  // namespace

extern "C" {

void memd_server_default_options(memd_server_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->precision = MEMD_FP32;
  o->budget_bytes = (int64_t)8 << 30;
  o->max_slots = 64;
  o->quantum = 50;
  o->device = -1;
}

memd_status memd_server_create(const memd_server_options* opt, memd_server** out) {
  if (!out) return MEMD_ERR_INVALID;
  *out = nullptr;
  memd_server* s = new memd_server();
  if (opt)
    s->opt = *opt;
  else
    memd_server_default_options(&s->opt);
  if (s->opt.max_slots < 1 || s->opt.quantum < 1 || s->opt.budget_bytes <= 0 ||
      (s->opt.precision != MEMD_FP32 && s->opt.precision != MEMD_FP64)) {
    delete s;
    return MEMD_ERR_INVALID;
  }
  // -1 means the device current at create: resolved here once, so the
  // admission threads (whose current device starts at 0) and the stream
  // below all use the same device
  if (s->opt.device < 0 && cudaGetDevice(&s->opt.device) != cudaSuccess) {
    delete s;
    return MEMD_ERR_CUDA;
  }
  if (cudaSetDevice(s->opt.device) != cudaSuccess) {
    delete s;
    return MEMD_ERR_CUDA;
  }
  if (!s->opt.cuda_stream) {
    // one stream shared by every resident system (a batch requirement)
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return MEMD_ERR_CUDA;
    }
    s->opt.cuda_stream = st;
    s->own_stream = true;
  }
  *out = s;
  return MEMD_OK;
}

void memd_server_destroy(memd_server* s) {
  if (!s) return;
  stop_workers(s);
  if (s->batch) memd_batch_destroy(s->batch);
  s->batch = nullptr;
  for (auto& kv : s->reqs)
    if (kv.second.ctx) memd_destroy(kv.second.ctx);
  for (auto* q : {&s->timed, &s->spare})
    for (auto& pr : *q) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  if (s->ev_done) cudaEventDestroy(s->ev_done);
  if (s->rstream) cudaStreamDestroy(s->rstream);
  if (s->own_stream) cudaStreamDestroy((cudaStream_t)s->opt.cuda_stream);
  delete s;
}

memd_status memd_server_submit(memd_server* s, const memd_request* q, int64_t* id) {
  if (!s || !q || !id) return MEMD_ERR_INVALID;
  if (q->n < 0 || q->nsteps < 0 || (q->n > 0 && (!q->pos || !q->q)))
    return sfail(s, MEMD_ERR_INVALID, "bad request arrays");
  memd_server::Req r;
  r.id = s->next_id++;
  std::memcpy(r.mesh, q->mesh, sizeof(r.mesh));
  std::memcpy(r.box, q->box, sizeof(r.box));
  r.eps_kind = q->eps.kind;
  r.eps_axis = q->eps.axis;
  std::memcpy(r.eps_params, q->eps.params, sizeof(r.eps_params));
  const int64_t V = (int64_t)q->mesh[0] * q->mesh[1] * q->mesh[2];
  if (q->eps.values) {
    const int64_t cnt = q->eps.kind == MEMD_EPS_LINKS ? 3 * V : V;
    r.eps_values.assign(q->eps.values, q->eps.values + cnt);
  }
  r.c_light = q->c_light;
  r.dt = q->dt;
  const int64_t n = q->n;
  r.pos.assign(q->pos, q->pos + 3 * n);
  r.q.assign(q->q, q->q + n);
  if (q->mass) r.mass.assign(q->mass, q->mass + n);
  if (q->vel) r.vel.assign(q->vel, q->vel + 3 * n);
  r.seed = q->seed;
  r.nsteps = r.remaining = q->nsteps;
  r.footprint = footprint(s->opt, r);
  *id = r.id;
  s->queue.push_back(r.id);
  s->reqs.emplace(r.id, std::move(r));
  return MEMD_OK;
}

memd_status memd_server_pump(memd_server* s, int32_t* n_active, int32_t* n_queued,
                             int32_t* n_done) {
  memd::NvtxRange nvtx_("memd_server_pump");
  if (!s) return MEMD_ERR_INVALID;
  const cudaStream_t sst = (cudaStream_t)s->opt.cuda_stream;
  {
    const memd_status se = start_workers(s);
    if (se != MEMD_OK) return sfail(s, se, "admission workers");
  }
  if (!s->ev_done && (cudaEventCreateWithFlags(&s->ev_done, cudaEventDisableTiming) != cudaSuccess ||
                      cudaStreamCreateWithFlags(&s->rstream, cudaStreamNonBlocking) != cudaSuccess))
    return sfail(s, MEMD_ERR_CUDA, "server events");
  // device time of the quanta that have finished
  auto harvest = [&](bool wait) {
    while (!s->timed.empty()) {
      auto pr = s->timed.front();
      if (wait) cudaEventSynchronize(pr.second);
      if (cudaEventQuery(pr.second) != cudaSuccess) break;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess)
        s->stats.step_gpu_s += 1e-3 * ms;
      s->timed.pop_front();
      s->spare.push_back(pr);
    }
    cudaGetLastError();
  };
  harvest(false);
  // 1. requests whose last steps are in the quantum in flight leave the
  // batch now (the host counted their steps at launch); their results are
  // collected below, once that quantum has finished
  std::vector<int64_t> keep, leaving;
  for (int64_t id : s->active) (s->reqs[id].remaining <= 0 ? leaving : keep).push_back(id);
  // 2. systems whose setup has finished join; queued requests go to the
  // admission workers in arrival order while memory and slots allow (their
  // footprint is reserved from the hand-over on)
  std::vector<std::pair<memd_server::Req*, memd_status>> got;
  int in_flight = 0;
  {
    std::lock_guard<std::mutex> g(s->mu);
    got.swap(s->ready);
    in_flight = s->in_flight;
  }
  bool changed = !leaving.empty();
  for (auto& pr : got) {
    memd_server::Req& r = *pr.first;
    if (pr.second != MEMD_OK) {
      r.state = MEMD_REQ_FAILED;
      s->used -= r.footprint;
      continue;
    }
    r.state = MEMD_REQ_RUNNING;
    keep.push_back(r.id);
    changed = true;
  }
  while (!s->queue.empty() && (int)(keep.size() + leaving.size()) + in_flight < s->opt.max_slots) {
    memd_server::Req& r = s->reqs[s->queue.front()];
    if (r.footprint > s->opt.budget_bytes) {
      r.state = MEMD_REQ_FAILED;
      r.error = "request larger than the memory budget";
      s->queue.pop_front();
      continue;
    }
    if (s->used + r.footprint > s->opt.budget_bytes) break;
    s->queue.pop_front();
    s->used += r.footprint;
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->todo.push_back(&r);
      s->in_flight += 1;
    }
    in_flight += 1;
    s->cv_todo.notify_one();
  }
  // 3. the next quantum, queued behind the one in flight: the batch's tables
  // are updated in place when its membership changed
  s->active.swap(keep);
  bool launched = false;
  if (!s->active.empty()) {
    if (changed || !s->batch) {
      std::vector<memd_ctx*> m;
      for (int64_t id : s->active) m.push_back(s->reqs[id].ctx);
      memd_status st;
      if (!s->batch) {
        st = memd_batch_create_opt((int32_t)m.size(), m.data(), &s->batch, false, MEMD_FIELD_AUTO);
        // the admission workers' setup kernels run beside the quanta: the
        // deposition runs after the field pass, not beside it (512-request
        // stream: p50 2.0-2.2 s -> 1.28 s, stepping 5.1 -> 5.5e10 link
        // updates/s)
        if (st == MEMD_OK) memd_batch_set_overlap(s->batch, false);
        s->stats.rebuilds += 1;
      } else {
        st = memd_batch_update_members(s->batch, (int32_t)m.size(), m.data());
      }
      if (st != MEMD_OK) return sfail(s, st, "batch tables");
      s->stats.table_updates += 1;
    }
    int64_t k = s->opt.quantum;
    for (int64_t id : s->active) k = std::min(k, s->reqs[id].remaining);
    if (k > 0) {
      memd_thermostat th{s->opt.gamma, s->opt.kT};
      std::pair<cudaEvent_t, cudaEvent_t> pr{nullptr, nullptr};
      if (!s->spare.empty()) {
        pr = s->spare.front();
        s->spare.pop_front();
      } else if (cudaEventCreate(&pr.first) != cudaSuccess ||
                 cudaEventCreate(&pr.second) != cudaSuccess) {
        return sfail(s, MEMD_ERR_CUDA, "server events");
      }
      cudaEventRecord(pr.first, sst);
      memd_status st = memd_batch_step(s->batch, k, s->opt.thermostat ? &th : nullptr);
      if (st != MEMD_OK) return sfail(s, st, "batch step failed");
      cudaEventRecord(pr.second, sst);
      s->timed.push_back(pr);
      for (int64_t id : s->active) {
        s->reqs[id].remaining -= k;
        s->stats.link_updates += 3 * k * (int64_t)s->reqs[id].mesh[0] * s->reqs[id].mesh[1] *
                                 s->reqs[id].mesh[2];
        s->stats.particle_steps += k * (int64_t)s->reqs[id].q.size();
      }
      s->stats.steps_rounds += 1;
      launched = true;
    }
  }
  // 4. the quantum before this one has finished once the stream reaches this
  // point; results of the requests that left are copied on the server's
  // second stream meanwhile, so the quantum just queued keeps the GPU busy
  if (!leaving.empty() || (!launched && s->any_launched)) {
    if (cudaStreamSynchronize(s->rstream) != cudaSuccess || cudaEventSynchronize(s->ev_done) != cudaSuccess)
      return sfail(s, MEMD_ERR_CUDA, "waiting for the last quantum");
    for (int64_t id : leaving) {
      memd_server::Req& r = s->reqs[id];
      r.ctx->stream = s->rstream;
      retire(s, r);
    }
  }
  if (launched) {
    cudaEventRecord(s->ev_done, sst);
    s->any_launched = true;
  } else if (s->any_launched) {
    harvest(true);  // the stream has drained
    s->any_launched = false;
  }
  if (s->active.empty() && in_flight > 0) {
    // nothing to step yet: wait a little for a setup to finish
    std::unique_lock<std::mutex> g(s->mu);
    s->cv_ready.wait_for(g, std::chrono::milliseconds(2), [&] { return !s->ready.empty(); });
  }
  s->stats.rounds += 1;
  int64_t resident = 0;
  for (int64_t id : s->active) resident += s->reqs[id].footprint;
  s->stats.budget_use_sum += (double)resident / (double)s->opt.budget_bytes;
  int32_t done = 0;
  for (auto& kv : s->reqs)
    if (kv.second.state == MEMD_REQ_DONE || kv.second.state == MEMD_REQ_FAILED) ++done;
  if (n_active) *n_active = (int32_t)s->active.size();
  if (n_queued) *n_queued = (int32_t)s->queue.size();
  if (n_done) *n_done = done;
  return MEMD_OK;
}

memd_status memd_server_status(memd_server* s, int64_t id, int32_t* state) {
  if (!s || !state) return MEMD_ERR_INVALID;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(s, MEMD_ERR_INVALID, "unknown request");
  *state = it->second.state;
  return MEMD_OK;
}

memd_status memd_server_result(memd_server* s, int64_t id, double* pos, double* vel,
                               int32_t* img, double* forces, memd_energy_terms* e) {
  if (!s) return MEMD_ERR_INVALID;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(s, MEMD_ERR_INVALID, "unknown request");
  memd_server::Req& r = it->second;
  if (r.state == MEMD_REQ_FAILED) return sfail(s, MEMD_ERR_STATE, r.error);
  if (r.state != MEMD_REQ_DONE) return sfail(s, MEMD_ERR_STATE, "request not finished");
  const size_t n3 = r.r_pos.size();
  if (pos && n3) std::memcpy(pos, r.r_pos.data(), n3 * sizeof(double));
  if (vel && n3) std::memcpy(vel, r.r_vel.data(), n3 * sizeof(double));
  if (img && n3) std::memcpy(img, r.r_img.data(), n3 * sizeof(int32_t));
  if (forces && n3) std::memcpy(forces, r.r_f.data(), n3 * sizeof(double));
  if (e) *e = r.r_e;
  return MEMD_OK;
}

memd_status memd_server_release(memd_server* s, int64_t id) {
  if (!s) return MEMD_ERR_INVALID;
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return sfail(s, MEMD_ERR_INVALID, "unknown request");
  if (it->second.state != MEMD_REQ_DONE && it->second.state != MEMD_REQ_FAILED)
    return sfail(s, MEMD_ERR_STATE, "request still queued or running");
  s->reqs.erase(it);
  return MEMD_OK;
}

int64_t memd_server_used_bytes(const memd_server* s) { return s ? s->used : 0; }

memd_status memd_server_get_stats(const memd_server* s, memd_server_stats* out) {
  if (!s || !out) return MEMD_ERR_INVALID;
  *out = s->stats;
  return MEMD_OK;
}

const char* memd_server_last_error(const memd_server* s) {
  return s ? s->last_error.c_str() : "no server";
}

}  // extern "C"
