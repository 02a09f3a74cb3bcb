// Continuous-batching server of independent hydro problems.
//
// Requests (a Sod, Sedov or two-state Riemann problem on a cubic FP64 box,
// advanced a given number of CTU-PPM steps) arrive at any time.  A scheduler
// thread admits them in arrival order as long as their device footprint fits
// the HBM budget and a slot is free and builds their initial state on the
// device.  Every iteration is then one batched CTU-PPM step (hydro_batch_run,
// launched directly: the stepped set changes from iteration to iteration)
// over a set of active boxes, each with its own gamma and CFL time step:
//   - HYDRO_SERVE_ALL: every active request steps every iteration (the GPU is
//     shared evenly per step, so a small request advances only as fast as
//     the largest box in the mix);
//   - HYDRO_SERVE_RESPONSE_RATIO (default): the requests with the highest
//     response ratio (time since submission + remaining work, over remaining
//     work; work = steps left x the measured cost of a step of that size)
//     step, added in that order while the iteration's estimated GPU time stays
//     within a quantum (the first one always steps).  Short requests get
//     through quickly, and a long one's ratio grows while it waits, so it is
//     not starved.  Only the stepped set needs step scratch, so the scratch
//     pool is bounded by the quantum and the largest box, and more requests'
//     states fit the budget.
// Requests that finish are retired (state copied to the caller's host buffer
// if one was given) and their memory is released, so new arrivals join at the
// next iteration.  The paper's analogue is the box iterator feeding a level's
// boxes to the GPU kernel (Sec. 4); serving many small problems concurrently
// is this library's own use of it.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hydro.h"
#include "hydro_api_internal.cuh"

using namespace hydro;
using Clock = std::chrono::steady_clock;

namespace {

// analytic initial state of a request on its grown box (ghosts included)
__global__ void k_init_problem(double* __restrict__ u, int n, int kind, double gamma, double rho_l, double p_l,
                               double rho_r, double p_r, double rho0, double p_amb, double p_dep, double r_dep2) {
  const long long g = n + 2 * NG;
  const long long N = g * g * g;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= N) return;
  const int gi = (int)(t % g), gj = (int)((t / g) % g), gk = (int)(t / (g * g));
  const int i = gi - NG, j = gj - NG, k = gk - NG;
  double rho, p;
  if (kind == HYDRO_PROB_SEDOV) {
    // deposit zones: centre strictly within r_dep of the box centre, in units of dx (exact)
    const double ox = (double)i + 0.5 - n / 2.0, oy = (double)j + 0.5 - n / 2.0, oz = (double)k + 0.5 - n / 2.0;
    const bool in = (ox * ox + oy * oy + oz * oz) < r_dep2;
    rho = rho0;
    p = in ? p_dep : p_amb;
  } else {
    const double dx = 1.0 / n;
    const double x = ((double)i + 0.5) * dx;
    const bool left = x < 0.5;
    rho = left ? rho_l : rho_r;
    p = left ? p_l : p_r;
  }
  u[t] = rho;
  u[N + t] = 0.0;
  u[2 * N + t] = 0.0;
  u[3 * N + t] = 0.0;
  u[4 * N + t] = p / (gamma - 1.0);
}

struct Req {
  uint64_t id = 0;
  hydro_request_t req{};
  double* buf[2] = {nullptr, nullptr};
  int cur = 0;
  int steps_done = 0;
  double t = 0.0, dt = 0.0;
  size_t state_bytes = 0, scratch_bytes = 0;
  Clock::time_point submitted, admitted;
  hydro_result_t result{};
  bool done = false;
  bool cancel = false;  // serve_cancel on an admitted request: retire at the next iteration
};

size_t grown_zones(int n) { return (size_t)(n + 2 * NG) * (n + 2 * NG) * (n + 2 * NG); }

// relative cost of one step of an n^3 box: the tracing and solver stages run
// over (n + 2)^3 to (n + 3)^3 zones
double step_units(int n) { return (double)(n + 3) * (n + 3) * (n + 3); }

// the fastest rate a step can reach, ms per unit (0.5 ns per zone: four
// times the measured single-box rate), used to bound the scratch a quantum
// can need before the rate is measured
constexpr double MIN_MS_PER_UNIT = 5e-7;

hydro_box_t box_of(double* u, int n) {
  hydro_box_t b;
  std::memset(&b, 0, sizeof b);
  b.u = u;
  b.n[0] = b.n[1] = b.n[2] = n;
  b.ng = NG;
  const long long g = n + 2 * NG;
  b.stride[0] = g;
  b.stride[1] = g * g;
  b.stride[2] = g * g * g;
  for (int a = 0; a < 3; ++a) {
    b.dx[a] = 1.0 / n;
    b.bc[a][0] = b.bc[a][1] = HYDRO_BC_OUTFLOW;
  }
  return b;
}

hydro_params_t params_of(const hydro_request_t& r) {
  hydro_params_t p;
  std::memset(&p, 0, sizeof p);
  p.gamma = r.gamma;
  p.cfl = r.cfl;
  p.small_dens = 1e-200;
  p.small_pres = 1e-200;
  p.dim = 3;
  p.flags = 0;
  return p;
}

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct serve {
  int device = 0;
  hydro_ctx_t* ctx = nullptr;
  cudaStream_t stream = nullptr;
  size_t budget = 0;
  size_t states_used = 0;
  int max_slots = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;
  std::vector<Req*> active;
  std::unordered_map<uint64_t, Req*> reqs;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread loop;
  double* dt_dev = nullptr;
  double* dt_next_dev = nullptr;
  // scheduling
  int policy = HYDRO_SERVE_RESPONSE_RATIO;
  // 2.5 ms (200-request prefix at 0.7 x capacity, two runs each: p99
  // slowdown 39 against 59 at 5 ms and 78 at 10 ms, p50 latency 4 % lower
  // than at 5 ms, p99 latency and throughput the same within 1 %)
  double quantum_ms = 2.5;
  double ms_per_unit = 2.1e-6;  // measured cost of a step per step_units (running average)
  // statistics
  long long iterations = 0, zone_updates = 0, admitted = 0, completed = 0, box_steps = 0;
  double busy_ms = 0.0, enqueue_ms = 0.0;
  size_t pool_cached = 0;  // scratch pool size, refreshed by the scheduler thread

  size_t pool_bytes() const { return hydro_batch_pool_bytes(ctx); }
  // scratch the pool may need with the active set plus one more request
  size_t pool_need(size_t scratch_sum, size_t scratch_max) const {
    if (policy == HYDRO_SERVE_ALL) return std::max(pool_bytes(), scratch_sum);
    const double units = quantum_ms / MIN_MS_PER_UNIT;
    const size_t quantum_scratch = (size_t)(units * SCRATCH_FIELDS * sizeof(double));
    return std::max(pool_bytes(), std::min(scratch_sum, scratch_max + quantum_scratch));
  }
  void retire(Req* r, int status);
  void run();
};

void serve::retire(Req* r, int status) {
  if (status == HYDRO_OK && r->req.result_host && r->buf[r->cur]) {
    if (cudaMemcpy(r->req.result_host, r->buf[r->cur], r->state_bytes / 2, cudaMemcpyDeviceToHost) != cudaSuccess)
      status = HYDRO_ECUDA;
  }
  for (double*& b : r->buf)
    if (b) {
      cudaFree(b);
      b = nullptr;
    }
  std::lock_guard<std::mutex> lock(mu);
  states_used -= r->state_bytes;
  const auto now = Clock::now();
  r->result.status = status;
  r->result.steps_done = r->steps_done;
  r->result.t_final = r->t;
  r->result.latency_ms = ms_between(r->submitted, now);
  r->result.queue_ms = ms_between(r->submitted, r->admitted);
  r->result.zone_updates = (long long)r->steps_done * r->req.n * r->req.n * r->req.n;
  r->done = true;
  completed += 1;
  cv_done.notify_all();
}

void serve::run() {
  if (cudaSetDevice(device) != cudaSuccess) return;
  std::vector<hydro_box_t> bin, bout;
  std::vector<hydro_params_t> prm;
  std::vector<double> dts, dtn;
  std::vector<int> bad;
  for (;;) {
    std::vector<Req*> fresh;
    {
      std::unique_lock<std::mutex> lock(mu);
      cv_work.wait(lock, [&] { return stop || !pending.empty() || !active.empty(); });
      if (stop) break;
      // admission in arrival order while the footprint fits the budget
      size_t scratch_sum = 0, scratch_max = 0;
      for (Req* r : active) {
        scratch_sum += r->scratch_bytes;
        scratch_max = std::max(scratch_max, r->scratch_bytes);
      }
      while (!pending.empty() && (int)(active.size() + fresh.size()) < max_slots) {
        Req* r = pending.front();
        size_t scratch_need = pool_need(scratch_sum + r->scratch_bytes, std::max(scratch_max, r->scratch_bytes));
        if (states_used + r->state_bytes + scratch_need > budget) break;
        pending.pop_front();
        states_used += r->state_bytes;
        scratch_sum += r->scratch_bytes;
        scratch_max = std::max(scratch_max, r->scratch_bytes);
        r->admitted = Clock::now();
        admitted += 1;
        fresh.push_back(r);
      }
    }
    // state, initial data and first CFL step of the new requests
    for (Req* r : fresh) {
      const int n = r->req.n;
      int status = HYDRO_OK;
      for (double*& b : r->buf)
        if (cudaMalloc(&b, r->state_bytes / 2) != cudaSuccess) {
          cudaGetLastError();
          b = nullptr;
          status = HYDRO_ENOMEM;
        }
      if (status == HYDRO_OK) {
        const hydro_request_t& q = r->req;
        double p_dep = 0.0;
        if (q.kind == HYDRO_PROB_SEDOV) {
          // deposit zone count (interior zones with centre within 4 dx of the centre)
          long long ndep = 0;
          const int lo = std::max(0, n / 2 - 6), hi = std::min(n, n / 2 + 6);  // the sphere lies inside
          for (int k = lo; k < hi; ++k)
            for (int j = lo; j < hi; ++j)
              for (int i = lo; i < hi; ++i) {
                double ox = i + 0.5 - n / 2.0, oy = j + 0.5 - n / 2.0, oz = k + 0.5 - n / 2.0;
                if (ox * ox + oy * oy + oz * oz < 16.0) ++ndep;
              }
          const double dx = 1.0 / n;
          p_dep = (q.gamma - 1.0) * q.energy / ((double)ndep * (dx * dx * dx));
        }
        const long long N = (long long)grown_zones(n);
        k_init_problem<<<(unsigned)((N + 255) / 256), 256, 0, stream>>>(
            r->buf[0], n, q.kind, q.gamma, q.rho_l, q.p_l, q.rho_r, q.p_r, 1.0, q.p_ambient, p_dep, 16.0);
        hydro_box_t b0 = box_of(r->buf[0], n);
        hydro_params_t p = params_of(q);
        double dt = 0.0;
        status = hydro_dt(ctx, &b0, &p, &dt, stream);
        r->dt = dt;
        r->cur = 0;
      }
      if (status != HYDRO_OK) {
        retire(r, status);
        continue;
      }
      std::lock_guard<std::mutex> lock(mu);
      active.push_back(r);
    }
    // requests cancelled since the last iteration leave before it
    std::vector<Req*> cancelled;
    {
      std::lock_guard<std::mutex> lock(mu);
      std::vector<Req*> still;
      for (Req* r : active) (r->cancel ? cancelled : still).push_back(r);
      active.swap(still);
    }
    for (Req* r : cancelled) retire(r, HYDRO_ECANCELED);
    if (active.empty()) continue;

    // the set that steps this iteration
    const auto t0 = Clock::now();
    std::vector<Req*> step_set;
    if (policy == HYDRO_SERVE_ALL) {
      step_set = active;
    } else {
      std::vector<std::pair<double, Req*>> order;
      for (Req* r : active) {
        const double work = (r->req.steps - r->steps_done) * ms_per_unit * step_units(r->req.n);
        order.push_back({(ms_between(r->submitted, t0) + work) / work, r});
      }
      std::stable_sort(order.begin(), order.end(),
                       [](const std::pair<double, Req*>& a, const std::pair<double, Req*>& b) { return a.first > b.first; });
      size_t scratch_sum = 0, scratch_max = 0;
      for (Req* r : active) {
        scratch_sum += r->scratch_bytes;
        scratch_max = std::max(scratch_max, r->scratch_bytes);
      }
      const size_t scratch_cap = pool_need(scratch_sum, scratch_max);
      double est = 0.0;
      size_t scratch = 0;
      for (auto& o : order) {
        Req* r = o.second;
        const double c = ms_per_unit * step_units(r->req.n);
        if (!step_set.empty() && (est + c > quantum_ms || scratch + r->scratch_bytes > scratch_cap)) continue;
        step_set.push_back(r);
        est += c;
        scratch += r->scratch_bytes;
      }
    }
    const int na = (int)step_set.size();
    bin.resize(na);
    bout.resize(na);
    prm.resize(na);
    dts.resize(na);
    dtn.resize(na);
    bad.assign(na, 0);
    double units = 0.0;
    for (int i = 0; i < na; ++i) {
      Req* r = step_set[i];
      bin[i] = box_of(r->buf[r->cur], r->req.n);
      bout[i] = box_of(r->buf[r->cur ^ 1], r->req.n);
      prm[i] = params_of(r->req);
      dts[i] = r->dt;
      units += step_units(r->req.n);
    }
    int rc = HYDRO_OK;
    const double select_ms = ms_between(t0, Clock::now());
    double enq_ms = 0.0;
    if (cudaMemcpyAsync(dt_dev, dts.data(), na * sizeof(double), cudaMemcpyHostToDevice, stream) != cudaSuccess)
      rc = HYDRO_ECUDA;
    if (rc == HYDRO_OK)
      rc = hydro_batch_run(ctx, bin.data(), bout.data(), na, prm.data(), 1, dt_dev, dt_next_dev, nullptr,
                           bad.data(), stream, nullptr, true, &enq_ms);
    if (rc == HYDRO_OK || rc == HYDRO_EBADSTATE) {
      if (cudaMemcpyAsync(dtn.data(), dt_next_dev, na * sizeof(double), cudaMemcpyDeviceToHost, stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(stream) != cudaSuccess)
        rc = HYDRO_ECUDA;
    }
    std::vector<std::pair<Req*, int>> finished;
    for (int i = 0; i < na; ++i) {
      Req* r = step_set[i];
      if (rc != HYDRO_OK && rc != HYDRO_EBADSTATE) {
        finished.push_back({r, rc});
        continue;
      }
      if (bad[i]) {
        finished.push_back({r, HYDRO_EBADSTATE});
        continue;
      }
      r->cur ^= 1;
      r->t += r->dt;
      r->steps_done += 1;
      r->dt = dtn[i];
      if (r->steps_done >= r->req.steps) finished.push_back({r, HYDRO_OK});
    }
    const auto t1 = Clock::now();
    {
      std::lock_guard<std::mutex> lock(mu);
      iterations += 1;
      box_steps += na;
      for (int i = 0; i < na; ++i)
        if (!bad[i]) zone_updates += (long long)step_set[i]->req.n * step_set[i]->req.n * step_set[i]->req.n;
      const double ms = ms_between(t0, t1);
      busy_ms += ms;
      enqueue_ms += select_ms + enq_ms;
      if (rc == HYDRO_OK && units > 0.0) ms_per_unit = 0.8 * ms_per_unit + 0.2 * (ms / units);
      pool_cached = pool_bytes();
      std::vector<Req*> still;
      for (Req* r : active)
        if (std::find_if(finished.begin(), finished.end(),
                         [r](const std::pair<Req*, int>& f) { return f.first == r; }) == finished.end())
          still.push_back(r);
      active.swap(still);
    }
    for (auto& f : finished) retire(f.first, f.second);
  }
}

extern "C" {

int serve_create(serve_t** out, int device, size_t hbm_budget_bytes, int max_slots) {
  if (!out || max_slots < 1 || max_slots > 4096) return HYDRO_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return HYDRO_ECUDA;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) return HYDRO_ECUDA;
  serve* s = new (std::nothrow) serve();
  if (!s) return HYDRO_ENOMEM;
  s->device = device;
  s->max_slots = max_slots;
  int rc = hydro_ctx_create(&s->ctx, device);
  size_t free_b = 0, total_b = 0;
  if (rc == HYDRO_OK && cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) rc = HYDRO_ECUDA;
  if (rc == HYDRO_OK && (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess ||
                         cudaMalloc(&s->dt_dev, max_slots * sizeof(double)) != cudaSuccess ||
                         cudaMalloc(&s->dt_next_dev, max_slots * sizeof(double)) != cudaSuccess))
    rc = HYDRO_ENOMEM;
  if (rc != HYDRO_OK) {
    cudaGetLastError();
    if (s->dt_dev) cudaFree(s->dt_dev);
    if (s->dt_next_dev) cudaFree(s->dt_next_dev);
    if (s->stream) cudaStreamDestroy(s->stream);
    hydro_ctx_destroy(s->ctx);
    delete s;
    if (prev >= 0) cudaSetDevice(prev);
    return rc;
  }
  s->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.8 * (double)free_b);
  s->loop = std::thread([s] { s->run(); });
  if (prev >= 0) cudaSetDevice(prev);
  *out = s;
  return HYDRO_OK;
}

int serve_submit(serve_t* s, const hydro_request_t* req, uint64_t* id) {
  if (!s || !req || !id) return HYDRO_EINVAL;
  const hydro_request_t& q = *req;
  if (q.kind < HYDRO_PROB_SOD || q.kind > HYDRO_PROB_TWO_STATE) return HYDRO_EINVAL;
  if (q.n < NG || q.n > 1024 || q.steps < 1) return HYDRO_EINVAL;
  if (!(q.gamma > 1.0) || !(q.cfl > 0.0) || !(q.cfl <= 1.0)) return HYDRO_EINVAL;
  if (q.kind != HYDRO_PROB_SEDOV && !(q.rho_l > 0.0 && q.p_l > 0.0 && q.rho_r > 0.0 && q.p_r > 0.0))
    return HYDRO_EINVAL;
  if (q.kind == HYDRO_PROB_SEDOV && !(q.energy > 0.0 && q.p_ambient > 0.0)) return HYDRO_EINVAL;
  Req* r = new (std::nothrow) Req();
  if (!r) return HYDRO_ENOMEM;
  r->req = q;
  r->state_bytes = 2 * 5 * grown_zones(q.n) * sizeof(double);
  int n3[3] = {q.n, q.n, q.n};
  r->scratch_bytes = (size_t)scratch_geom(n3, 3).sc * SCRATCH_FIELDS * sizeof(double);
  r->submitted = Clock::now();
  std::lock_guard<std::mutex> lock(s->mu);
  if (r->state_bytes + r->scratch_bytes > s->budget) {
    delete r;
    return HYDRO_ETOOBIG;
  }
  r->id = s->next_id++;
  s->reqs[r->id] = r;
  s->pending.push_back(r);
  *id = r->id;
  s->cv_work.notify_all();
  return HYDRO_OK;
}

int serve_cancel(serve_t* s, uint64_t id) {
  if (!s) return HYDRO_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return HYDRO_EINVAL;
  Req* r = it->second;
  if (r->done) return HYDRO_OK;  // finished first: the result stands
  auto q = std::find(s->pending.begin(), s->pending.end(), r);
  if (q != s->pending.end()) {  // never admitted: it leaves the queue now
    s->pending.erase(q);
    const auto now = Clock::now();
    r->result.status = HYDRO_ECANCELED;
    r->result.steps_done = 0;
    r->result.t_final = 0.0;
    r->result.latency_ms = ms_between(r->submitted, now);
    r->result.queue_ms = r->result.latency_ms;
    r->result.zone_updates = 0;
    r->done = true;
    s->cv_done.notify_all();
    return HYDRO_OK;
  }
  r->cancel = true;  // admitted: the scheduler retires it before its next iteration
  s->cv_work.notify_all();
  return HYDRO_OK;
}

int serve_poll(serve_t* s, uint64_t id, hydro_result_t* res, int timeout_ms) {
  if (!s || !res) return HYDRO_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return HYDRO_EINVAL;
  Req* r = it->second;
  if (!r->done) {
    if (timeout_ms == 0) return HYDRO_EAGAIN;
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0) s->cv_done.wait(lock, ready);
    else if (!s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), ready)) return HYDRO_ETIMEDOUT;
  }
  *res = r->result;
  s->reqs.erase(it);
  delete r;
  return HYDRO_OK;
}

int serve_set_policy(serve_t* s, int policy, double quantum_ms) {
  if (!s || (policy != HYDRO_SERVE_ALL && policy != HYDRO_SERVE_RESPONSE_RATIO)) return HYDRO_EINVAL;
  if (policy == HYDRO_SERVE_RESPONSE_RATIO && !(quantum_ms > 0.0 && quantum_ms <= 60000.0)) return HYDRO_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  // busy while anything is queued, being admitted or running
  if (!s->pending.empty() || s->admitted != s->completed) return HYDRO_EAGAIN;
  s->policy = policy;
  if (policy == HYDRO_SERVE_RESPONSE_RATIO) s->quantum_ms = quantum_ms;
  return HYDRO_OK;
}

int serve_stats(serve_t* s, hydro_serve_stats_t* st) {
  if (!s || !st) return HYDRO_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  st->queued = (int)s->pending.size();
  st->active = (int)s->active.size();
  st->admitted = s->admitted;
  st->completed = s->completed;
  st->iterations = s->iterations;
  st->zone_updates = s->zone_updates;
  st->busy_ms = s->busy_ms;
  st->hbm_budget = s->budget;
  st->hbm_states = s->states_used;
  st->hbm_scratch_pool = s->pool_cached;
  st->box_steps = s->box_steps;
  st->enqueue_ms = s->enqueue_ms;
  st->ms_per_unit = s->ms_per_unit;
  return HYDRO_OK;
}

void serve_destroy(serve_t* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->loop.joinable()) s->loop.join();
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  cudaStreamSynchronize(s->stream);
  for (auto& kv : s->reqs) {
    for (double* b : kv.second->buf)
      if (b) cudaFree(b);
    delete kv.second;
  }
  cudaFree(s->dt_dev);
  cudaFree(s->dt_next_dev);
  cudaStreamDestroy(s->stream);
  hydro_ctx_destroy(s->ctx);
  if (prev >= 0) cudaSetDevice(prev);
  delete s;
}

}  // extern "C"
