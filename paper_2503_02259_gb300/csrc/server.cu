// Continuous-batching request server (include/gp.h, "Serving").
//
// One device pool of the HBM budget is reserved at creation and sub-allocated
// first-fit; max_slots worker threads each own one CUDA stream per stream
// priority level.  A free worker admits the queued request with the least work
// (entries x columns) among those whose footprint fits the pool's free space;
// a request that has waited kAgeSeconds or more is admitted first, in arrival
// order, so large requests are not starved.  It runs the request through the
// library's own calls and returns the memory, so requests that arrive while
// others are running join them on the device: the CTAs of all running
// requests' kernels are interleaved on the SMs by the hardware work
// distributor.  A request runs
// on a stream whose priority falls with its work (entries x columns), so the
// tiles of a small request are dispatched ahead of the queued tiles of a large
// one instead of waiting for them.  The paper serves nothing; its stateless
// loss/gradient and prediction calls (§Design and Implementation) are what
// each request runs.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "gp_api_internal.h"
#include "admission.h"

namespace {

using gp::sched::align_up;
using gp::sched::kAlign;
using gp::sched::PoolAllocator;

// Device sub-buffers of one request inside its pool block.
struct JobLayout {
  size_t x, y, xs, mu, alpha, ws, ws_bytes, total;
};

const float* const kSizingX = reinterpret_cast<const float*>(kAlign);  // never dereferenced

gp_solve_opts opts_of(const gp_request& r, bool loss) {
  gp_solve_opts o{};
  o.nprobe = loss ? r.nprobe : 0;
  o.nlanczos = r.nlanczos > 0 ? r.nlanczos : 20;
  o.cg_maxit = r.cg_maxit;
  o.prec = r.prec;
  o.slq_prec = r.slq_prec;
  o.cg_rtol = r.cg_rtol;
  o.seed = r.seed;
  return o;
}

bool layout_of(const gp_request& r, JobLayout* L) {
  if (r.n < 1 || r.d < 1 || r.d > GP_MAX_DIM) return false;
  if (r.kind != 0 && r.kind != 1) return false;
  if (r.kind == 1 && r.m < 1) return false;
  gp_problem prob{kSizingX, r.n, r.d, r.kernel, r.theta};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  L->x = take(sizeof(float) * r.n * r.d);
  L->y = take(sizeof(float) * r.n);
  L->xs = L->mu = L->alpha = 0;
  size_t wsb = 0;
  if (r.kind == 0) {
    const gp_solve_opts o = opts_of(r, true);
    wsb = gp_workspace_bytes(GP_OP_LOSS_GRAD, &prob, 0, &o);
    // A request that may run in a batch gets room for either workspace.
    if (gp::sched::batchable(r))
      wsb = std::max(wsb, gp_workspace_bytes(GP_OP_LOSS_GRAD_BATCH, &prob, 0, &o));
  } else {
    L->xs = take(sizeof(float) * r.m * r.d);
    L->mu = take(sizeof(float) * r.m);
    L->alpha = take(sizeof(float) * r.n);
    const gp_solve_opts o = opts_of(r, false);
    wsb = std::max(gp_workspace_bytes(GP_OP_PCG, &prob, 1, &o),
                   gp_workspace_bytes(GP_OP_PREDICT, &prob, static_cast<int32_t>(r.m), nullptr));
  }
  if (wsb == 0) return false;
  L->ws = take(wsb);
  L->ws_bytes = wsb;
  L->total = off;
  return true;
}

struct Job {
  uint64_t ticket = 0;
  gp_request req{};
  JobLayout lay{};
  double work = 0.0;     // entries x columns of its products (admission order)
  float* hX = nullptr;   // host staging (inputs) and results: a block of the
  float* hy = nullptr;   // pinned staging pool, or pageable memory when the
  float* hXs = nullptr;  // pool is full
  float* hmu = nullptr;
  size_t hoff = 0, hbytes = 0;        // pinned block (hbytes > 0)
  std::unique_ptr<float[]> pageable;  // fallback staging
  gp_result res{};
  bool done = false;
};

double seconds_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct gp_server {
  int device = 0;
  char* pool = nullptr;
  size_t budget = 0;
  std::unique_ptr<PoolAllocator> alloc;
  // Pinned host staging, reserved once (a per-request cudaMallocHost /
  // cudaFreeHost could stall the device); guarded by mu.
  char* hpool = nullptr;
  size_t hbudget = 0;
  std::unique_ptr<PoolAllocator> halloc;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Job>> queue;
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  std::vector<std::thread> workers;
  // Start-up latch: each worker reports whether it created its streams;
  // gp_server_create waits for every report (cv_start).
  int workers_ready = 0, workers_failed = 0;
  std::condition_variable cv_start;
  bool stop = false;
  uint64_t next_ticket = 1;
  int64_t submitted = 0, completed = 0, refused = 0, active = 0, peak_active = 0;
  size_t peak_bytes = 0;
  // Grouped launches: up to max_batch compatible loss + gradient requests run
  // as one gp_loss_and_grad_batch (1: every request alone).
  int max_batch = 1;
  int64_t batches = 0, batched_requests = 0, largest_batch = 0;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
};

namespace {

// Returns a job's staging (its pinned block, or its pageable buffer).
void free_staging(gp_server* srv, Job& j) {
  if (j.hbytes > 0) {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->halloc->release(j.hoff, j.hbytes);
  }
  j.hbytes = 0;
  j.pageable.reset();
  j.hX = j.hy = j.hXs = j.hmu = nullptr;
}

// Run one request on `st` inside its pool block; fills j.res.
void run_job(gp_server* srv, Job& j, char* base, cudaStream_t st) {
  const gp_request& r = j.req;
  float* dX = reinterpret_cast<float*>(base + j.lay.x);
  float* dy = reinterpret_cast<float*>(base + j.lay.y);
  void* ws = base + j.lay.ws;
  gp_status s = GP_OK;
  cudaError_t e = cudaMemcpyAsync(dX, j.hX, sizeof(float) * r.n * r.d, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dy, j.hy, sizeof(float) * r.n, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    j.res.status = GP_ERR_CUDA;
    return;
  }
  gp_problem prob{dX, r.n, r.d, r.kernel, r.theta};
  if (r.kind == 0) {
    const gp_solve_opts o = opts_of(r, true);
    gp_loss_info info{};
    s = gp_loss_and_grad(&prob, dy, &o, &j.res.loss, j.res.grad, &info, ws, j.lay.ws_bytes, st);
    j.res.cg_iters = info.cg_iters;
    j.res.relres = info.relres_max;
  } else {
    float* dXs = reinterpret_cast<float*>(base + j.lay.xs);
    float* dmu = reinterpret_cast<float*>(base + j.lay.mu);
    float* dalpha = reinterpret_cast<float*>(base + j.lay.alpha);
    e = cudaMemcpyAsync(dXs, j.hXs, sizeof(float) * r.m * r.d, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      j.res.status = GP_ERR_CUDA;
      return;
    }
    const gp_solve_opts o = opts_of(r, false);
    int32_t it = 0;
    double rel = 0.0;
    s = gp_pcg_solve(&prob, dy, 1, dalpha, &o, &it, &rel, ws, j.lay.ws_bytes, st);
    j.res.cg_iters = it;
    j.res.relres = rel;
    if (s == GP_OK || s == GP_ERR_NOT_CONVERGED) {
      const gp_status sp = gp_predict_mean(&prob, dalpha, dXs, r.m, dmu, GP_PREC_FP32, ws,
                                           j.lay.ws_bytes, st);
      if (sp != GP_OK) s = sp;
      if (sp == GP_OK) {
        e = cudaMemcpyAsync(j.hmu, dmu, sizeof(float) * r.m, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = GP_ERR_CUDA;
      }
    }
  }
  cudaStreamSynchronize(st);
  j.res.status = s;
  (void)srv;
}

// Run a batch of compatible loss + gradient requests (each in its own pool
// block) as one gp_loss_and_grad_batch on `st`; fills every job's result.
void run_batch(std::vector<std::shared_ptr<Job>>& jobs, const std::vector<char*>& bases,
               cudaStream_t st) {
  const size_t count = jobs.size();
  std::vector<gp_problem> probs(count);
  std::vector<gp_solve_opts> opts(count);
  std::vector<const float*> ys(count);
  std::vector<void*> ws(count);
  std::vector<size_t> wsb(count);
  std::vector<double> loss(count), grad(3 * count);
  std::vector<gp_loss_info> info(count);
  std::vector<int32_t> status(count, GP_ERR_CUDA);
  bool copied = true;
  for (size_t k = 0; k < count; ++k) {
    Job& j = *jobs[k];
    const gp_request& r = j.req;
    float* dX = reinterpret_cast<float*>(bases[k] + j.lay.x);
    float* dy = reinterpret_cast<float*>(bases[k] + j.lay.y);
    copied = copied && cudaMemcpyAsync(dX, j.hX, sizeof(float) * r.n * r.d, cudaMemcpyHostToDevice,
                                       st) == cudaSuccess;
    copied = copied &&
             cudaMemcpyAsync(dy, j.hy, sizeof(float) * r.n, cudaMemcpyHostToDevice, st) == cudaSuccess;
    probs[k] = gp_problem{dX, r.n, r.d, r.kernel, r.theta, nullptr};
    opts[k] = opts_of(r, true);
    ys[k] = dy;
    ws[k] = bases[k] + j.lay.ws;
    wsb[k] = j.lay.ws_bytes;
  }
  gp_status s = GP_ERR_CUDA;
  if (copied)
    s = gp_loss_and_grad_batch(static_cast<int32_t>(count), probs.data(), ys.data(), opts.data(),
                               loss.data(), grad.data(), info.data(), status.data(), ws.data(),
                               wsb.data(), st);
  cudaStreamSynchronize(st);
  for (size_t k = 0; k < count; ++k) {
    gp_result& res = jobs[k]->res;
    // Per-member status when the call ran; the call's own status otherwise.
    const bool ran = s == GP_OK || s == GP_ERR_NOT_CONVERGED;
    res.status = ran ? static_cast<gp_status>(status[k]) : s;
    res.loss = loss[k];
    for (int t = 0; t < 3; ++t) res.grad[t] = grad[3 * k + t];
    res.cg_iters = info[k].cg_iters;
    res.relres = info[k].relres_max;
  }
}

using gp::sched::kAgeSeconds;
using gp::sched::priority_level;
using gp::sched::request_work;

// Called with srv->mu held: picks the next request to admit by the rule of
// gp::sched::pick_next and reserves its pool block (returns false if none can
// start now).
bool admit_next(gp_server* srv, std::shared_ptr<Job>* job, size_t* off) {
  auto& q = srv->queue;
  const long i = gp::sched::pick_next(
      q.size(), seconds_since(srv->t0), *srv->alloc, [&](size_t k) { return q[k]->work; },
      [&](size_t k) { return q[k]->res.t_submit_s; }, [&](size_t k) { return q[k]->lay.total; }, off);
  if (i < 0) return false;
  *job = q[static_cast<size_t>(i)];
  q.erase(q.begin() + i);
  return true;
}

void worker_main(gp_server* srv) {
  cudaSetDevice(srv->device);
  gp::set_thread_cooperative(false);
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) least = greatest = 0;
  const int levels = std::max(1, std::min(8, least - greatest + 1));
  std::vector<cudaStream_t> streams(levels, nullptr);
  bool ok = true;
  for (int i = 0; i < levels && ok; ++i) {
    // Level i has the i-th highest priority (numerically greatest + i).
    if (cudaStreamCreateWithPriority(&streams[i], cudaStreamNonBlocking, greatest + i) != cudaSuccess) {
      cudaGetLastError();
      for (int k = 0; k < i; ++k) cudaStreamDestroy(streams[k]);
      ok = false;
    }
  }
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (ok)
      ++srv->workers_ready;
    else
      ++srv->workers_failed;
  }
  srv->cv_start.notify_all();
  if (!ok) return;   // gp_server_create reports the failure and stops the others
  for (;;) {
    std::vector<std::shared_ptr<Job>> batch;
    std::vector<size_t> offs;
    {
      std::shared_ptr<Job> job;
      size_t off = 0;
      std::unique_lock<std::mutex> lk(srv->mu);
      // Re-check at least every 100 ms, so that a request reaching kAgeSeconds
      // is noticed without another event.
      while (!srv->stop && !admit_next(srv, &job, &off))
        srv->cv_work.wait_for(lk, std::chrono::milliseconds(100));
      if (srv->stop) break;
      batch.push_back(job);
      offs.push_back(off);
      if (srv->max_batch > 1 && gp::sched::batchable(job->req)) {
        auto& q = srv->queue;
        const std::vector<size_t> extra = gp::sched::pick_batch(
            q.size(), job->work, srv->max_batch - 1, *srv->alloc,
            [&](size_t k) { return gp::sched::same_batch(job->req, q[k]->req); },
            [&](size_t k) { return q[k]->work; }, [&](size_t k) { return q[k]->lay.total; }, &offs);
        for (size_t k : extra) batch.push_back(q[k]);
        std::vector<size_t> rm(extra);
        std::sort(rm.rbegin(), rm.rend());
        for (size_t k : rm) q.erase(q.begin() + static_cast<long>(k));
      }
      srv->active += static_cast<int64_t>(batch.size());
      srv->peak_active = std::max(srv->peak_active, srv->active);
      srv->peak_bytes = std::max(srv->peak_bytes, srv->alloc->in_use());
      const double now = seconds_since(srv->t0);
      for (auto& j : batch) j->res.t_start_s = now;
      if (batch.size() > 1) {
        ++srv->batches;
        srv->batched_requests += static_cast<int64_t>(batch.size());
        srv->largest_batch = std::max<int64_t>(srv->largest_batch, static_cast<int64_t>(batch.size()));
      }
    }
    cudaStream_t st = streams[priority_level(batch[0]->req, levels)];
    if (batch.size() == 1) {
      run_job(srv, *batch[0], srv->pool + offs[0], st);
    } else {
      std::vector<char*> bases;
      for (size_t o : offs) bases.push_back(srv->pool + o);
      run_batch(batch, bases, st);
    }
    {
      std::lock_guard<std::mutex> lk(srv->mu);
      const double now = seconds_since(srv->t0);
      for (size_t k = 0; k < batch.size(); ++k) {
        srv->alloc->release(offs[k], batch[k]->lay.total);
        --srv->active;
        ++srv->completed;
        batch[k]->res.t_done_s = now;
        batch[k]->done = true;
      }
    }
    srv->cv_work.notify_all();
    srv->cv_done.notify_all();
  }
  for (cudaStream_t st : streams) cudaStreamDestroy(st);
}

gp_status fail(gp_status st, const char* msg) {
  gp::set_error(msg);
  return st;
}

}  // namespace

extern "C" {

size_t gp_server_footprint(const gp_request* req) {
  JobLayout L;
  if (req == nullptr || !layout_of(*req, &L)) return 0;
  return L.total;
}

gp_status gp_server_destroy(gp_server* srv);

static gp_status server_create(size_t hbm_budget_bytes, int32_t max_slots, int32_t max_batch,
                               gp_server** out);

gp_status gp_server_create(size_t hbm_budget_bytes, int32_t max_slots, gp_server** out) {
  return server_create(hbm_budget_bytes, max_slots, 1, out);
}

gp_status gp_server_create_batched(size_t hbm_budget_bytes, int32_t max_slots, int32_t max_batch,
                                   gp_server** out) {
  if (max_batch < 1 || max_batch > 64)
    return fail(GP_ERR_ARG, "gp_server_create_batched: max_batch must be in [1, 64]");
  return server_create(hbm_budget_bytes, max_slots, max_batch, out);
}

static gp_status server_create(size_t hbm_budget_bytes, int32_t max_slots, int32_t max_batch,
                               gp_server** out) {
  if (out == nullptr || max_slots < 1 || max_slots > 256 || hbm_budget_bytes < (1u << 20))
    return fail(GP_ERR_ARG, "gp_server_create: need out != NULL, 1 <= max_slots <= 256, budget >= 1 MiB");
  auto* srv = new gp_server();
  srv->max_batch = max_batch;
  if (cudaGetDevice(&srv->device) != cudaSuccess) {
    delete srv;
    return fail(GP_ERR_CUDA, "gp_server_create: no current device");
  }
  srv->budget = hbm_budget_bytes & ~(kAlign - 1);
  void* p = nullptr;
  if (cudaMalloc(&p, srv->budget) != cudaSuccess) {
    cudaGetLastError();
    delete srv;
    return fail(GP_ERR_OOM, "gp_server_create: cannot reserve the device pool");
  }
  srv->pool = static_cast<char*>(p);
  srv->alloc = std::make_unique<PoolAllocator>(srv->budget);
  // Pinned staging: 1/8 of the device budget, between 64 MiB and 2 GiB.
  srv->hbudget = std::min<size_t>(std::max<size_t>(srv->budget / 8, size_t(64) << 20),
                                  size_t(2) << 30);
  void* hp = nullptr;
  if (cudaMallocHost(&hp, srv->hbudget) != cudaSuccess) {
    cudaGetLastError();
    srv->hbudget = 0;   // every request uses pageable staging
  }
  srv->hpool = static_cast<char*>(hp);
  srv->halloc = std::make_unique<PoolAllocator>(srv->hbudget);
  for (int i = 0; i < max_slots; ++i) srv->workers.emplace_back(worker_main, srv);
  bool all_ready = false;
  {
    std::unique_lock<std::mutex> lk(srv->mu);
    srv->cv_start.wait_for(lk, std::chrono::seconds(60), [&] {
      return srv->workers_ready + srv->workers_failed == max_slots;
    });
    all_ready = srv->workers_ready == max_slots;
  }
  if (!all_ready) {
    // A worker could not create its streams (or did not report in time): stop
    // the others and release everything, so no request can queue without a
    // worker to run it.
    gp_server_destroy(srv);
    return fail(GP_ERR_CUDA, "gp_server_create: a worker could not create its CUDA streams");
  }
  srv->t0 = std::chrono::steady_clock::now();   // the clock of t_submit_s / t_done_s
  *out = srv;
  return GP_OK;
}

gp_status gp_server_submit(gp_server* srv, const gp_request* req, uint64_t* ticket) {
  if (srv == nullptr || req == nullptr || ticket == nullptr) return fail(GP_ERR_ARG, "NULL argument");
  const gp_request& r = *req;
  if (r.X == nullptr || r.y == nullptr || (r.kind == 1 && r.Xstar == nullptr))
    return fail(GP_ERR_ARG, "gp_server_submit: missing host array");
  auto job = std::make_shared<Job>();
  if (!layout_of(r, &job->lay)) return fail(GP_ERR_ARG, "gp_server_submit: invalid request");
  job->req = r;
  job->work = request_work(r);
  const double t_submit = seconds_since(srv->t0);
  if (job->lay.total > srv->budget) {
    std::lock_guard<std::mutex> lk(srv->mu);
    ++srv->refused;
    return fail(GP_ERR_OOM, "gp_server_submit: request footprint exceeds the server's budget");
  }
  // Staging block: X, y, and for predictions X* and mu, each 256-byte aligned.
  const size_t bx = align_up(sizeof(float) * r.n * r.d), by = align_up(sizeof(float) * r.n);
  const size_t bxs = r.kind == 1 ? align_up(sizeof(float) * r.m * r.d) : 0;
  const size_t bmu = r.kind == 1 ? align_up(sizeof(float) * r.m) : 0;
  const size_t hb = bx + by + bxs + bmu;
  char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    size_t off = 0;
    if (srv->hbudget > 0 && srv->halloc->alloc(hb, &off)) {
      job->hoff = off;
      job->hbytes = hb;
      base = srv->hpool + off;
    }
  }
  if (base == nullptr) {
    job->pageable.reset(new (std::nothrow) float[hb / sizeof(float)]);
    if (!job->pageable) return fail(GP_ERR_OOM, "gp_server_submit: cannot allocate host staging");
    base = reinterpret_cast<char*>(job->pageable.get());
  }
  job->hX = reinterpret_cast<float*>(base);
  job->hy = reinterpret_cast<float*>(base + bx);
  if (r.kind == 1) {
    job->hXs = reinterpret_cast<float*>(base + bx + by);
    job->hmu = reinterpret_cast<float*>(base + bx + by + bxs);
  }
  memcpy(job->hX, r.X, sizeof(float) * r.n * r.d);
  memcpy(job->hy, r.y, sizeof(float) * r.n);
  if (r.kind == 1) memcpy(job->hXs, r.Xstar, sizeof(float) * r.m * r.d);
  job->req.X = job->req.y = job->req.Xstar = nullptr;
  job->res.t_submit_s = t_submit;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    job->ticket = srv->next_ticket++;
    srv->jobs[job->ticket] = job;
    srv->queue.push_back(job);
    ++srv->submitted;
  }
  srv->cv_work.notify_all();
  *ticket = job->ticket;
  return GP_OK;
}

gp_status gp_server_poll(gp_server* srv, uint64_t ticket, gp_result* res) {
  if (srv == nullptr || res == nullptr) return fail(GP_ERR_ARG, "NULL argument");
  std::shared_ptr<Job> job;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(ticket);
    if (it == srv->jobs.end()) return fail(GP_ERR_ARG, "gp_server_poll: unknown ticket");
    if (!it->second->done) return GP_ERR_TIMEOUT;
    job = it->second;
    srv->jobs.erase(it);
  }
  float* user_mu = res->mu;
  *res = job->res;
  res->mu = user_mu;
  if (user_mu != nullptr && job->req.kind == 1 && job->hmu != nullptr)
    memcpy(user_mu, job->hmu, sizeof(float) * job->req.m);
  free_staging(srv, *job);
  return GP_OK;
}

gp_status gp_server_drain(gp_server* srv, double timeout_s) {
  if (srv == nullptr) return fail(GP_ERR_ARG, "NULL server");
  std::unique_lock<std::mutex> lk(srv->mu);
  const bool ok = srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
    return srv->completed >= srv->submitted;
  });
  return ok ? GP_OK : GP_ERR_TIMEOUT;
}

gp_status gp_server_get_stats(gp_server* srv, gp_server_stats* out) {
  if (srv == nullptr || out == nullptr) return fail(GP_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(srv->mu);
  out->submitted = srv->submitted;
  out->completed = srv->completed;
  out->refused = srv->refused;
  out->peak_active = srv->peak_active;
  out->peak_bytes = srv->peak_bytes;
  out->budget_bytes = srv->budget;
  out->batches = srv->batches;
  out->batched_requests = srv->batched_requests;
  out->largest_batch = srv->largest_batch;
  return GP_OK;
}

gp_status gp_server_destroy(gp_server* srv) {
  if (srv == nullptr) return fail(GP_ERR_ARG, "NULL server");
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  for (auto& t : srv->workers) t.join();
  for (auto& kv : srv->jobs) free_staging(srv, *kv.second);
  srv->jobs.clear();
  srv->queue.clear();
  if (srv->pool) cudaFree(srv->pool);
  if (srv->hpool) cudaFreeHost(srv->hpool);
  delete srv;
  return GP_OK;
}

}  // extern "C"
