// server.cu -- continuous-batching reconstruction server (ffpat_server_*,
// ffpat_submit, ffpat_poll): many Algorithm-8 solves (Sec. 3.2) of different
// grid sizes in flight on one GPU.
//
// A worker thread owns one CUDA stream.  Requests wait in a FIFO queue and are
// admitted while a slot is free and their device memory (sound speed, data,
// iterate and workspace) fits the HBM budget; each admitted request carries a
// host-side phase machine (power iteration if no step was given, then FB
// iterations: forward W, P + residual (+ Lambda), P^T, adjoint W, update).
// Every "tick" the worker gathers the next leapfrog work of every request that
// is inside a W phase and advances all of them with at most two batched
// launches: one single step for the requests at their start step or last odd
// step (launch_step_batch) and one two-step pass for the others
// (launch_step2_batch); requests whose W phase ended get their projection /
// update kernels queued behind it.  Nothing on this path waits for the GPU
// except a bounded run-ahead (a ring of tick events) and the completion event
// of each request, so requests that arrive while others run join the next
// tick.  A request's kernels see exactly the arithmetic of ffpat_fb_solve, so
// its result does not depend on what else shares the GPU.
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"

struct ffpat_server;

namespace ffpat {
namespace {

using Clock = std::chrono::steady_clock;

enum Phase { kQueued, kFwd, kAdj, kFinish, kDone };

struct Req {
  uint64_t ticket = 0;
  ffpat_problem prob{};
  Plan pl;
  double lambda = 0, step = 0;
  int iters = 0, power_iters = 0;
  // host staging (pinned)
  float* c_h = nullptr;
  float* g_h = nullptr;
  float* out_h = nullptr;
  unsigned char* tab_h = nullptr;
  double* fin_h = nullptr;  // 8 doubles of the last iteration's sums + the step
  // device
  unsigned char* dmem = nullptr;
  size_t dbytes = 0;
  float* c_d = nullptr;
  float* g_d = nullptr;
  float* h_d = nullptr;
  double* step_d = nullptr;
  // progress
  Phase phase = kQueued;
  int it = 0;     // iterations done (power, then FB)
  int wstep = 0;  // leapfrog step inside the current W
  int de = 0;     // which pair of (d, e) buffers holds the current level
  const float* w_in = nullptr;
  const float* cur = nullptr;
  cudaEvent_t done_ev = nullptr;
  Clock::time_point t_submit, t_admit, t_done;
  int status = FFPAT_PENDING;
  bool cancel = false;
  bool admitted = false;  // holds budget (dbytes) while true
};

constexpr int kTickRing = 32;
constexpr size_t kMaxQueue = 4096;

}  // namespace
}  // namespace ffpat

using ffpat::Req;

struct ffpat_server {
  size_t budget = 0, used = 0;
  int max_slots = 1;
  int device = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t ring[ffpat::kTickRing] = {};
  int ring_pos = 0;
  long long ticks = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Req>> queue;
  std::vector<std::shared_ptr<Req>> active;
  std::map<uint64_t, std::shared_ptr<Req>> all;  // every request not yet polled
  std::vector<double> latencies_ms;
  long long failed = 0, cancelled = 0;
  double point_steps = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  int fatal = 0;
  std::thread worker;
  ffpat::Clock::time_point t0;
};

namespace ffpat {
namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t request_bytes(const Plan& pl, size_t ws) {
  return up256(pl.n3 * 4) * 2 + up256(pl.nd * 4) + up256(64 * sizeof(double)) + ws;
}

void release_host(Req& r) {
  if (r.c_h) cudaFreeHost(r.c_h);
  if (r.g_h) cudaFreeHost(r.g_h);
  if (r.tab_h) cudaFreeHost(r.tab_h);
  r.c_h = r.g_h = nullptr;
  r.tab_h = nullptr;
}

// admission: device memory, uploads, wave coefficients; power-iteration start
int admit(ffpat_server* S, Req& r) {
  cudaStream_t st = S->st;
  const size_t ws = ffpat_workspace_bytes(&r.prob);
  if (cudaMallocAsync((void**)&r.dmem, r.dbytes, st) != cudaSuccess) {
    cudaGetLastError();
    return FFPAT_ENOMEM;
  }
  unsigned char* b = r.dmem;
  r.c_d = (float*)b;
  b += up256(r.pl.n3 * 4);
  r.h_d = (float*)b;
  b += up256(r.pl.n3 * 4);
  r.g_d = (float*)b;
  b += up256(r.pl.nd * 4);
  r.step_d = (double*)b;
  b += up256(64 * sizeof(double));
  if (attach(&r.prob, r.pl, b, ws) != FFPAT_OK) return FFPAT_EINVAL;
  if (cudaMemcpyAsync(r.c_d, r.c_h, r.pl.n3 * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(r.g_d, r.g_h, r.pl.nd * 4, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(r.pl.tab, r.tab_h, table_bytes(r.pl.nth), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaMemsetAsync(r.h_d, 0, r.pl.n3 * 4, st) != cudaSuccess)
    return check_launch("server admission copies");
  // c_max on the host from the staged copy (max is exact, so Nt and dt equal
  // what the device reduction of ffpat_fb_solve finds)
  double cmax = 0.0;
  for (size_t i = 0; i < r.pl.n3; ++i) cmax = fmax(cmax, (double)r.c_h[i]);
  if (time_steps(r.pl, cmax, &r.pl.nt, &r.pl.dt) != FFPAT_OK) return FFPAT_EINVAL;
  r.pl.cmax = cmax;
  if (launch_kappa(r.pl, r.c_d, st) != FFPAT_OK) return FFPAT_ECUDA;
  if (r.power_iters > 0) {
    double* sq = r.pl.scal + 8;
    if (launch_hash_fill(r.pl, r.pl.v, 0x5eed1901ull, st) != FFPAT_OK ||
        launch_dot(r.pl, r.pl.n3, r.pl.v, r.pl.v, sq, st) != FFPAT_OK ||
        launch_scale_dev(r.pl, r.pl.n3, r.pl.v, r.pl.v, sq, st) != FFPAT_OK)
      return FFPAT_ECUDA;
  }
  r.phase = kFwd;
  r.wstep = 0;
  r.w_in = (const float*)(r.power_iters > 0 ? r.pl.v : r.h_d);
  r.t_admit = Clock::now();
  return FFPAT_OK;
}

// The state of a request inside a W: p in s[0] / s[1] (alternating), the
// increment d and the Kahan carry e in the pair (s[2], s[3]) or (s[4], s[5])
// (`de`).  A W runs the start step, then two steps per pass while at least two
// remain, then a last single step if one is left -- the sequence of
// ffpat_fb_solve's time loop, so the served result is the same bit for bit.
float* d_buf(const Req& r, int k) { return (float*)r.pl.s[k ? 4 : 2]; }
float* e_buf(const Req& r, int k) { return (float*)r.pl.s[k ? 5 : 3]; }

bool two_steps_next(const Req& r) {
  return r.wstep > 0 && r.pl.nt - r.wstep >= 2 && r.pl.n <= kTwoStepMaxN;
}

// the single step of request r in this tick (start step or the last one)
BatchStep next_step(Req& r) {
  BatchStep b;
  const Plan& pl = r.pl;
  b.start = r.wstep == 0;
  if (b.start) r.de = 0;
  b.p = b.start ? r.w_in : r.cur;
  b.pout = (float*)(b.start ? pl.s[0] : (r.cur == pl.s[0] ? pl.s[1] : pl.s[0]));
  b.d = d_buf(r, r.de);
  b.e = e_buf(r, r.de);
  b.kap = (const float*)pl.kap;
  b.n = pl.n;
  return b;
}

// the two-step pass of request r in this tick (d, e go to the other pair)
BatchStep2 next_pass(const Req& r) {
  BatchStep2 b;
  const Plan& pl = r.pl;
  b.p = r.cur;
  b.pout = (float*)(r.cur == pl.s[0] ? pl.s[1] : pl.s[0]);
  b.d = d_buf(r, r.de);
  b.e = e_buf(r, r.de);
  b.dout = d_buf(r, 1 - r.de);
  b.eout = e_buf(r, 1 - r.de);
  b.kap = (const float*)pl.kap;
  b.n = pl.n;
  return b;
}

// queue the kernels between the end of a W phase and the next phase
int after_wave(ffpat_server* S, Req& r) {
  cudaStream_t st = S->st;
  const Plan& pl = r.pl;
  const bool power = r.it < r.power_iters;
  if (r.phase == kFwd) {
    if (launch_project(pl, r.cur, pl.r, power ? nullptr : r.g_d, st, nullptr, pl.x) != FFPAT_OK)
      return FFPAT_ECUDA;
    const void* lr = pl.r;
    if (pl.precond == FFPAT_PRECOND_RAMP) {
      if (launch_ramp(pl, pl.r, pl.r2, st) != FFPAT_OK) return FFPAT_ECUDA;
      lr = pl.r2;
    }
    if (!power && launch_dot(pl, pl.nd, lr, pl.r, pl.hist, st) != FFPAT_OK) return FFPAT_ECUDA;
    if (launch_backproject(pl, lr, pl.x, pl.kap, st) != FFPAT_OK) return FFPAT_ECUDA;
    r.phase = kAdj;
    r.wstep = 0;
    r.w_in = (const float*)pl.x;
    return FFPAT_OK;
  }
  // end of the adjoint W: update
  if (power) {
    double* sq = pl.scal + 8;
    if (launch_kscale(pl, r.cur, pl.v, false, st) != FFPAT_OK ||
        launch_dot(pl, pl.n3, pl.v, pl.v, sq, st) != FFPAT_OK ||
        launch_scale_dev(pl, pl.n3, pl.v, pl.v, sq, st) != FFPAT_OK)
      return FFPAT_ECUDA;
    if (r.it + 1 == r.power_iters && launch_inv_sqrt(sq, r.step_d, st) != FFPAT_OK)
      return FFPAT_ECUDA;
  } else {
    const double* sdev = r.power_iters > 0 ? r.step_d : nullptr;
    if (launch_fb_update(pl, r.h_d, r.cur, r.step, r.lambda, pl.hist + 2, st, sdev) != FFPAT_OK)
      return FFPAT_ECUDA;
  }
  r.it += 1;
  if (r.it == r.power_iters + r.iters) {
    if (cudaMemcpyAsync(r.out_h, r.h_d, pl.n3 * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(r.fin_h, pl.hist, 6 * sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        (r.power_iters > 0 &&
         cudaMemcpyAsync(r.fin_h + 6, r.step_d, sizeof(double), cudaMemcpyDeviceToHost, st) !=
             cudaSuccess) ||
        cudaEventRecord(r.done_ev, st) != cudaSuccess)
      return check_launch("server completion copies");
    r.phase = kFinish;
    return FFPAT_OK;
  }
  r.phase = kFwd;
  r.wstep = 0;
  r.w_in = (const float*)(r.it < r.power_iters ? pl.v : r.h_d);
  return FFPAT_OK;
}

void finish(ffpat_server* S, Req& r, int status) {
  r.status = status;
  r.t_done = Clock::now();
  if (r.dmem) {
    cudaFreeAsync(r.dmem, S->st);
    r.dmem = nullptr;
  }
  if (r.admitted) S->used -= r.dbytes;
  r.admitted = false;
  release_host(r);
  r.phase = kDone;
  if (status == FFPAT_OK) {
    S->latencies_ms.push_back(
        std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count());
    S->point_steps += 2.0 * (r.power_iters + r.iters) * (double)r.pl.nt * (double)r.pl.n3;
  } else if (status == FFPAT_ECANCELED) {
    S->cancelled += 1;
  } else {
    S->failed += 1;
  }
}

void worker_loop(ffpat_server* S) {
  cudaSetDevice(S->device);
  std::vector<BatchStep> batch;
  std::vector<BatchStep2> batch2;
  std::vector<Req*> in_batch, in_batch2;
  while (true) {
    {
      std::unique_lock<std::mutex> lk(S->mu);
      // retire finished requests, admit new ones
      for (auto it = S->active.begin(); it != S->active.end();) {
        Req& r = **it;
        bool drop = false;
        if (r.cancel) {
          finish(S, r, FFPAT_ECANCELED);
          drop = true;
        } else if (r.phase == kFinish) {
          const cudaError_t q = cudaEventQuery(r.done_ev);
          if (q == cudaSuccess) {
            finish(S, r, FFPAT_OK);
            drop = true;
          } else if (q != cudaErrorNotReady) {
            finish(S, r, FFPAT_ECUDA);
            drop = true;
          }
        }
        it = drop ? S->active.erase(it) : it + 1;
      }
      while (!S->queue.empty()) {
        auto r = S->queue.front();
        if (r->cancel) {
          S->queue.pop_front();
          finish(S, *r, FFPAT_ECANCELED);
          continue;
        }
        if ((int)S->active.size() >= S->max_slots || S->used + r->dbytes > S->budget) break;
        S->queue.pop_front();
        S->used += r->dbytes;
        r->admitted = true;
        const int rc = admit(S, *r);
        if (rc != FFPAT_OK) {
          finish(S, *r, rc);
          continue;
        }
        S->active.push_back(r);
      }
      if (S->stop) break;
      batch.clear();
      batch2.clear();
      in_batch.clear();
      in_batch2.clear();
      bool any_finish = false;
      for (auto& r : S->active) {
        if (r->phase == kFwd || r->phase == kAdj) {
          if (two_steps_next(*r)) {
            batch2.push_back(next_pass(*r));
            in_batch2.push_back(r.get());
          } else {
            batch.push_back(next_step(*r));
            in_batch.push_back(r.get());
          }
        }
        any_finish |= r->phase == kFinish;
      }
      if (batch.empty() && batch2.empty()) {
        S->cv.notify_all();
        if (any_finish) {
          lk.unlock();
          std::this_thread::sleep_for(std::chrono::microseconds(50));
        } else {
          S->cv.wait_for(lk, std::chrono::milliseconds(2));
        }
        continue;
      }
    }
    // bounded run-ahead: at most kTickRing ticks queued on the stream
    cudaEvent_t& ev = S->ring[S->ring_pos];
    cudaEventSynchronize(ev);
    Trace trace_tick("serving tick (batched leapfrog steps)");
    // single steps (start steps, last odd steps) in one launch, two-step
    // passes in another; a request takes part in at most one of them
    int rc = launch_step_batch(batch.data(), (int)batch.size(), S->st);
    if (rc == FFPAT_OK) rc = launch_step2_batch(batch2.data(), (int)batch2.size(), S->st);
    for (size_t i = 0; rc == FFPAT_OK && i < in_batch.size(); ++i) {
      Req& r = *in_batch[i];
      r.cur = batch[i].pout;
      r.wstep += 1;
      if (r.wstep == r.pl.nt) rc = after_wave(S, r);
    }
    for (size_t i = 0; rc == FFPAT_OK && i < in_batch2.size(); ++i) {
      Req& r = *in_batch2[i];
      r.cur = batch2[i].pout;
      r.de = 1 - r.de;
      r.wstep += 2;
      if (r.wstep == r.pl.nt) rc = after_wave(S, r);
    }
    cudaEventRecord(ev, S->st);
    S->ring_pos = (S->ring_pos + 1) % kTickRing;
    S->ticks += 1;
    if (rc != FFPAT_OK) {
      std::lock_guard<std::mutex> g(S->mu);
      S->fatal = rc;
      for (auto& r : S->active) finish(S, *r, rc);
      S->active.clear();
    }
  }
  cudaStreamSynchronize(S->st);
}

}  // namespace
}  // namespace ffpat

using namespace ffpat;

extern "C" {

int ffpat_server_create(size_t hbm_budget_bytes, int32_t max_slots, ffpat_server** out) {
  if (!out) return report(FFPAT_EINVAL, "out is NULL");
  if (max_slots < 1 || max_slots > kMaxBatchRequests)
    return report(FFPAT_EINVAL, "max_slots = %d outside [1, %d]", max_slots, kMaxBatchRequests);
  if (hbm_budget_bytes == 0) return report(FFPAT_EINVAL, "HBM budget is 0");
  auto* S = new ffpat_server();
  S->budget = hbm_budget_bytes;
  S->max_slots = max_slots;
  cudaGetDevice(&S->device);
  if (cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) != cudaSuccess) {
    delete S;
    return check_launch("server stream");
  }
  for (auto& e : S->ring) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  S->t0 = Clock::now();
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return FFPAT_OK;
}

int ffpat_submit(ffpat_server* S, const ffpat_problem* problem, const void* c_host,
                 const void* g_host, double lambda, double step, int32_t iters, uint64_t* ticket) {
  if (!S || !problem || !c_host || !g_host || !ticket) return report(FFPAT_EINVAL, "NULL argument");
  auto r = std::make_shared<Req>();
  r->prob = *problem;
  const size_t ws = ffpat_workspace_bytes(problem);
  if (ws == 0) return FFPAT_EINVAL;
  if (problem->precision != FFPAT_FP32_KAHAN || problem->n % 4 != 0 || problem->pad != 0)
    return report(FFPAT_EINVAL, "served problems are FFPAT_FP32_KAHAN with N %% 4 == 0 and pad = 0");
  if (iters < 1 || iters > kMaxHist) return report(FFPAT_EINVAL, "iters = %d", iters);
  if (!(lambda >= 0.0) || !isfinite(lambda) || !isfinite(step))
    return report(FFPAT_EINVAL, "lambda / step not finite");
  Plan probe;
  if (attach(problem, probe, (void*)256, ws) != FFPAT_OK) return FFPAT_EINVAL;
  r->pl = probe;
  r->dbytes = request_bytes(probe, ws);
  if (r->dbytes > S->budget)
    return report(FFPAT_EINVAL, "request needs %zu bytes > HBM budget %zu", r->dbytes, S->budget);
  r->lambda = lambda;
  r->step = step;
  r->iters = iters;
  r->power_iters = step > 0.0 ? 0 : 20;
  if (cudaMallocHost((void**)&r->c_h, probe.n3 * 4) != cudaSuccess ||
      cudaMallocHost((void**)&r->g_h, probe.nd * 4) != cudaSuccess ||
      cudaMallocHost((void**)&r->out_h, probe.n3 * 4) != cudaSuccess ||
      cudaMallocHost((void**)&r->tab_h, table_bytes(probe.nth)) != cudaSuccess ||
      cudaMallocHost((void**)&r->fin_h, 8 * sizeof(double)) != cudaSuccess) {
    release_host(*r);
    if (r->out_h) cudaFreeHost(r->out_h);
    if (r->fin_h) cudaFreeHost(r->fin_h);
    cudaGetLastError();
    return report(FFPAT_ENOMEM, "pinned host staging");
  }
  memcpy(r->c_h, c_host, probe.n3 * 4);
  memcpy(r->g_h, g_host, probe.nd * 4);
  fill_tables_host(probe.nth, r->tab_h);
  memset(r->fin_h, 0, 8 * sizeof(double));
  cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
  r->t_submit = Clock::now();
  std::lock_guard<std::mutex> g(S->mu);
  if (S->queue.size() >= kMaxQueue) {
    release_host(*r);
    cudaFreeHost(r->out_h);
    cudaFreeHost(r->fin_h);
    cudaEventDestroy(r->done_ev);
    return report(FFPAT_EBUSY, "server queue full (%zu requests)", kMaxQueue);
  }
  r->ticket = S->next_ticket++;
  S->queue.push_back(r);
  S->all[r->ticket] = r;
  *ticket = r->ticket;
  S->cv.notify_all();
  return FFPAT_OK;
}

int ffpat_poll(ffpat_server* S, uint64_t ticket, void* h_out_host, ffpat_fb_stats* stats) {
  if (!S) return report(FFPAT_EINVAL, "server is NULL");
  std::shared_ptr<Req> r;
  {
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return report(FFPAT_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
    r = it->second;
    if (r->phase != kDone) return FFPAT_PENDING;
    S->all.erase(it);
  }
  const int status = r->status;
  if (status == FFPAT_OK) {
    if (h_out_host) memcpy(h_out_host, r->out_h, r->pl.n3 * 4);
    if (stats) {
      const double* q = r->fin_h;
      memset(stats, 0, sizeof *stats);
      stats->iters_done = r->iters;
      stats->objective = 0.5 * q[0] + r->lambda * q[2];
      stats->resid_norm = sqrt(q[1]);
      stats->rel_change = sqrt(q[4]) / fmax(sqrt(q[3]), 1e-300);
      stats->step = r->power_iters > 0 ? q[6] : r->step;
      stats->opnorm_sq = r->power_iters > 0 ? 1.0 / q[6] : 0.0;
    }
  }
  cudaFreeHost(r->out_h);
  cudaFreeHost(r->fin_h);
  cudaEventDestroy(r->done_ev);
  r->out_h = nullptr;
  r->fin_h = nullptr;
  if (status == FFPAT_ECANCELED) return report(FFPAT_ECANCELED, "request %llu was cancelled", (unsigned long long)ticket);
  if (status != FFPAT_OK) return report(status, "request %llu failed", (unsigned long long)ticket);
  return FFPAT_OK;
}

int ffpat_cancel(ffpat_server* S, uint64_t ticket) {
  if (!S) return report(FFPAT_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return report(FFPAT_EINVAL, "unknown ticket");
  it->second->cancel = true;
  S->cv.notify_all();
  return FFPAT_OK;
}

int ffpat_server_stats(ffpat_server* S, ffpat_serving_stats* out) {
  if (!S || !out) return report(FFPAT_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> g(S->mu);
  memset(out, 0, sizeof *out);
  std::vector<double> l = S->latencies_ms;
  std::sort(l.begin(), l.end());
  auto pct = [&](double p) {
    if (l.empty()) return 0.0;
    const size_t i = (size_t)std::min<double>((double)l.size() - 1, ceil(p * l.size()) - 1);
    return l[i];
  };
  out->completed = (int64_t)l.size();
  out->failed = S->failed;
  out->cancelled = S->cancelled;
  out->p50_ms = pct(0.50);
  out->p99_ms = pct(0.99);
  double sum = 0;
  for (double v : l) sum += v;
  out->mean_ms = l.empty() ? 0.0 : sum / l.size();
  out->max_ms = l.empty() ? 0.0 : l.back();
  out->point_steps = S->point_steps;
  out->ticks = S->ticks;
  out->active = (int32_t)S->active.size();
  out->queued = (int32_t)S->queue.size();
  out->hbm_in_use = S->used;
  return S->fatal;
}

int ffpat_server_destroy(ffpat_server* S) {
  if (!S) return FFPAT_OK;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
    for (auto& r : S->queue) r->cancel = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto& r : S->active) finish(S, *r, FFPAT_ECANCELED);
  for (auto& r : S->queue) finish(S, *r, FFPAT_ECANCELED);
  cudaStreamSynchronize(S->st);
  for (auto& kv : S->all) {
    Req& r = *kv.second;
    release_host(r);
    if (r.out_h) cudaFreeHost(r.out_h);
    if (r.fin_h) cudaFreeHost(r.fin_h);
    if (r.done_ev) cudaEventDestroy(r.done_ev);
  }
  for (auto& e : S->ring) cudaEventDestroy(e);
  cudaStreamDestroy(S->st);
  delete S;
  return FFPAT_OK;
}

}  // extern "C"
