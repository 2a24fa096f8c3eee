// Continuous-batching solve server: a persistent host loop that runs many GNP-FGMRES
// solves at once on one GPU.  Each request brings its own matrix, model, right-hand
// side and solution buffer.  Requests wait in a FIFO queue and are admitted as slots and
// device memory free up; an admitted request gets its own Krylov workspace, GNP scratch
// (the model's weights and A_hat are shared read-only) and stream, and its restart cycle
// is captured once as a CUDA graph.  Each running request has one cycle in flight on its
// stream: the graph, then a copy of its solver state to pinned host memory and an event.
// The loop polls the events; the moment a request's cycle ends it applies that request's
// stopping rules and either launches its next cycle or retires it, freeing its slot for
// the queue, so no request waits for another's cycle (the requests' work overlaps on the
// device).  A request's result does not depend on what else runs: every kernel reads
// only its own request's data and all reductions have a fixed order.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "solver.h"

namespace gnp {

using Clock = std::chrono::steady_clock;

struct Request {
  long long ticket = 0;
  gnp_mat* A = nullptr;
  gnp_model* M = nullptr;
  const double* b = nullptr;
  double* x = nullptr;
  double rtol = 1e-8;
  int maxiters = 1000;
  int m = 30;
  size_t footprint = 0;
  Clock::time_point t_submit;
  // running state
  Solver* S = nullptr;
  ApplyWs ws;
  cudaGraph_t cycle = nullptr;
  cudaGraphExec_t exec = nullptr;  // the instantiated cycle
  cudaStream_t stream = nullptr;   // the request's own stream
  cudaEvent_t ev = nullptr;        // recorded after each cycle's state copy
  CycleCtl ctl;
  DevState* mirror = nullptr;  // pinned copy of the device state, written after each cycle
  double beta = 0.0;
  // result: `result` is set by the loop thread, `status` (read by poll/wait) only under
  // the server lock when the request is published as finished
  int result = GNP_OK;
  int status = -1;
  gnp_solve_info info{};
};

struct Server {
  gnp_server_config cfg{};
  int device = 0;
  std::thread loop;
  std::mutex mu;
  std::condition_variable cv;       // wakes the loop
  std::condition_variable done_cv;  // wakes waiters
  std::deque<Request*> queue;
  std::vector<Request*> running;      // loop thread only
  int n_active = 0;                   // running.size(), published under the lock
  std::map<long long, Request*> all;  // every request not yet collected by poll/wait
  long long next_ticket = 1;
  size_t used_bytes = 0;
  bool stop = false;
  // statistics (`rounds`: restart cycles launched)
  long long rounds = 0, completed = 0, admitted = 0, max_active_seen = 0;
  int error = GNP_OK;
  char errmsg[256] = {0};
};

static size_t request_footprint(const gnp_mat* A, int m, int maxiters) {
  return solver_bytes(A->n, m, maxiters) + apply_ws_bytes(A->n);
}

static void release(Request* r) {
  if (r->exec) cudaGraphExecDestroy(r->exec);
  r->exec = nullptr;
  if (r->cycle) cudaGraphDestroy(r->cycle);
  r->cycle = nullptr;
  if (r->ev) cudaEventDestroy(r->ev);
  r->ev = nullptr;
  if (r->stream) cudaStreamDestroy(r->stream);
  r->stream = nullptr;
  solver_free(r->S);
  r->S = nullptr;
  apply_ws_free(r->ws);
  if (r->mirror) cudaFreeHost(r->mirror);
  r->mirror = nullptr;
}

// Loop thread: the request ended with `status` (published later under the lock).
static void finish(Server* sv, Request* r, int status) {
  (void)sv;
  r->result = status;
  r->info.status = status;
  r->info.seconds = std::chrono::duration<double>(Clock::now() - r->t_submit).count();
}

// Allocate the request's workspace and stream, run its initial residual, capture and
// instantiate its cycle graph.  Returns true when the request is still running afterwards.
static bool setup(Server* sv, Request* r) {
  (void)sv;
  int s = GNP_OK;
  if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) {
    set_error("server: stream or event creation failed");
    s = GNP_ERR_CUDA;
  }
  if (s == GNP_OK) s = solver_create(r->A->n, r->m, r->maxiters, &r->S);
  if (s == GNP_OK && r->M) s = apply_ws_alloc(r->ws, r->A->n);
  if (s == GNP_OK && cudaMallocHost(reinterpret_cast<void**>(&r->mirror), sizeof(DevState)) != cudaSuccess) {
    set_error("server: cudaMallocHost failed");
    s = GNP_ERR_OOM;
  }
  cudaStream_t st = r->stream;
  if (s == GNP_OK && r->M) s = apply_prepare(r->M);
  if (s == GNP_OK) s = solve_init_launch(r->A, r->S, r->b, r->x, r->rtol, r->maxiters, r->m, 0.0, st);
  if (s == GNP_OK && cudaMemcpyAsync(r->mirror, r->S->st, sizeof(DevState), cudaMemcpyDeviceToHost, st) !=
                         cudaSuccess)
    s = GNP_ERR_CUDA;
  if (s == GNP_OK && cudaStreamSynchronize(st) != cudaSuccess) {
    set_error("server: %s", cudaGetErrorString(cudaGetLastError()));
    s = GNP_ERR_CUDA;
  }
  if (s != GNP_OK) {
    finish(sv, r, s);
    return false;
  }
  const DevState& hs = *r->mirror;
  r->beta = hs.beta;
  r->info.iters = 0;
  if (hs.bnorm == 0.0) {
    cudaMemsetAsync(r->x, 0, sizeof(double) * r->A->n, st);
    cudaStreamSynchronize(st);
    finish(sv, r, GNP_OK);
    return false;
  }
  if (!std::isfinite(hs.beta) || !std::isfinite(hs.bnorm)) {
    finish(sv, r, GNP_ERR_NAN);
    return false;
  }
  if (hs.beta <= hs.tol) {
    r->info.rel_res_true = hs.beta / hs.bnorm;
    finish(sv, r, GNP_OK);
    return false;
  }
  if (r->maxiters == 0) {
    finish(sv, r, GNP_ERR_NOT_CONVERGED);
    return false;
  }
  // capture the restart cycle once; its device-side step state makes it replayable
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    set_error("server: begin capture failed");
    finish(sv, r, GNP_ERR_CUDA);
    return false;
  }
  Prec P;
  P.kind = r->M ? GNP_PRECOND_GNP : GNP_PRECOND_IDENTITY;
  P.M = r->M;
  P.key = r->M;
  s = launch_cycle(r->A, r->S, P, r->m, r->b, r->x, st, false, r->M ? &r->ws : nullptr);
  cudaError_t ce = cudaStreamEndCapture(st, &r->cycle);
  if (ce == cudaSuccess && s == GNP_OK) ce = cudaGraphInstantiate(&r->exec, r->cycle, 0);
  if (s != GNP_OK || ce != cudaSuccess) {
    if (ce != cudaSuccess) set_error("server: capture or instantiation failed: %s", cudaGetErrorString(ce));
    finish(sv, r, s != GNP_OK ? s : GNP_ERR_CUDA);
    return false;
  }
  return true;
}

// Start the request's next restart cycle on its stream: the cycle, the copy of its state to
// pinned memory, the event the loop polls.
static int launch_next(Server* sv, Request* r) {
  if (cudaGraphLaunch(r->exec, r->stream) != cudaSuccess ||
      cudaMemcpyAsync(r->mirror, r->S->st, sizeof(DevState), cudaMemcpyDeviceToHost, r->stream) != cudaSuccess ||
      cudaEventRecord(r->ev, r->stream) != cudaSuccess) {
    set_error("server: cycle launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return GNP_ERR_CUDA;
  }
  ++sv->rounds;
  return GNP_OK;
}

static void fill_result(Request* r) {
  if (!r->mirror) return;
  const DevState& hs = *r->mirror;
  r->info.iters = hs.iters;
  r->info.restarts = r->ctl.restarts;
  r->info.cycles = r->ctl.cycles;
  const double bn = hs.bnorm > 0.0 ? hs.bnorm : 1.0;
  r->info.rel_res_true = hs.beta / bn;
  r->info.rel_res_est = hs.res_est / bn;
}

static void server_loop(Server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    // admission (under the lock): FIFO, by slot count and device-memory footprint
    std::vector<Request*> fresh, ended;
    while (!sv->queue.empty() && (int)(sv->running.size() + fresh.size()) < sv->cfg.max_active) {
      Request* r = sv->queue.front();
      if (r->footprint > sv->cfg.max_bytes) {
        sv->queue.pop_front();
        r->status = GNP_ERR_OOM;
        r->info.status = GNP_ERR_OOM;
        ++sv->completed;
        sv->done_cv.notify_all();
        continue;
      }
      if (sv->used_bytes + r->footprint > sv->cfg.max_bytes) break;
      sv->queue.pop_front();
      sv->used_bytes += r->footprint;
      fresh.push_back(r);
    }
    if (sv->stop && sv->queue.empty() && sv->running.empty() && fresh.empty()) break;
    if (sv->running.empty() && fresh.empty()) {
      sv->cv.wait_for(lk, std::chrono::milliseconds(50));
      continue;
    }
    lk.unlock();
    bool progressed = !fresh.empty();
    for (Request* r : fresh) {
      ++sv->admitted;
      if (setup(sv, r) && launch_next(sv, r) == GNP_OK) {
        sv->running.push_back(r);
      } else {
        if (r->result == GNP_OK && r->exec) finish(sv, r, GNP_ERR_CUDA);  // the first launch failed
        fill_result(r);
        ended.push_back(r);
      }
    }
    sv->max_active_seen = std::max<long long>(sv->max_active_seen, (long long)sv->running.size());
    // every request whose cycle has ended: stopping rules, then its next cycle or retirement
    std::vector<Request*> still;
    for (Request* r : sv->running) {
      const cudaError_t q = cudaEventQuery(r->ev);
      if (q == cudaErrorNotReady) {
        still.push_back(r);
        continue;
      }
      progressed = true;
      int status = GNP_OK;
      bool end = true;
      if (q != cudaSuccess) {
        set_error("server: cycle failed: %s", cudaGetErrorString(q));
        status = GNP_ERR_CUDA;
      } else {
        ++r->ctl.cycles;
        const DevState& hs = *r->mirror;
        const double beta_prev = r->beta;
        end = cycle_after(hs, beta_prev, r->maxiters, r->ctl, &status);
        r->beta = hs.beta;
        if (!end && launch_next(sv, r) != GNP_OK) {
          status = GNP_ERR_CUDA;
          end = true;
        }
      }
      if (end) {
        fill_result(r);
        finish(sv, r, status);
        ended.push_back(r);
      } else {
        still.push_back(r);
      }
    }
    sv->running.swap(still);
    for (Request* r : ended) release(r);
    lk.lock();
    for (Request* r : ended) {
      sv->used_bytes -= r->footprint;
      r->status = r->result;
      ++sv->completed;
    }
    sv->n_active = (int)sv->running.size();
    if (!ended.empty()) sv->done_cv.notify_all();
    if (!progressed) {
      // no cycle ended and nothing was admitted: wait a little (new requests wake the loop)
      sv->cv.wait_for(lk, std::chrono::microseconds(50));
    }
  }
}

}  // namespace gnp

struct gnp_server {
  gnp::Server* s;
};

using namespace gnp;

extern "C" {

int gnp_server_create(const gnp_server_config* cfg, gnp_server** out) {
  GNP_REQUIRE(cfg && out, "gnp_server_create: null argument");
  *out = nullptr;
  GNP_REQUIRE(cfg->max_active >= 1, "gnp_server_create: max_active must be >= 1");
  GNP_REQUIRE(cfg->restart >= 1 && cfg->restart <= GNP_MAX_RESTART, "gnp_server_create: bad restart");
  Server* sv = new Server();
  sv->cfg = *cfg;
  cudaGetDevice(&sv->device);
  sv->loop = std::thread(server_loop, sv);
  *out = new gnp_server{sv};
  return GNP_OK;
}

int gnp_server_submit(gnp_server* h, gnp_mat* A, gnp_model* M, const double* b_dev, double* x_dev,
                      double rtol, int maxiters, long long* ticket) {
  GNP_REQUIRE(h && A && b_dev && x_dev && ticket, "gnp_server_submit: null argument");
  GNP_REQUIRE(!M || M->A == A, "gnp_server_submit: the preconditioner was built for another matrix");
  GNP_REQUIRE(maxiters >= 0 && rtol >= 0.0, "gnp_server_submit: bad maxiters/rtol");
  Server* sv = h->s;
  Request* r = new Request();
  r->A = A;
  r->M = M;
  r->b = b_dev;
  r->x = x_dev;
  r->rtol = rtol;
  r->maxiters = maxiters;
  r->m = sv->cfg.restart;
  r->footprint = request_footprint(A, r->m, maxiters);
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    GNP_REQUIRE(!sv->stop, "gnp_server_submit: server is shutting down");
    r->ticket = sv->next_ticket++;
    sv->queue.push_back(r);
    sv->all[r->ticket] = r;
  }
  sv->cv.notify_one();
  *ticket = r->ticket;
  return GNP_OK;
}

static int collect(Server* sv, std::map<long long, Request*>::iterator it, gnp_solve_info* info) {
  Request* r = it->second;
  const int st = r->status;
  if (info) {
    double* hist = info->res_history;
    double* hess = info->hessenberg;
    double* times = info->time_history;
    *info = r->info;
    info->res_history = hist;
    info->hessenberg = hess;
    info->time_history = times;
    info->res_history_len = 0;
    info->hessenberg_cols = 0;
  }
  sv->all.erase(it);
  delete r;
  return st;
}

int gnp_server_poll(gnp_server* h, long long ticket, gnp_solve_info* info) {
  GNP_REQUIRE(h, "gnp_server_poll: null server");
  Server* sv = h->s;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  GNP_REQUIRE(it != sv->all.end(), "gnp_server_poll: unknown ticket %lld", ticket);
  if (it->second->status < 0) return GNP_ERR_BUSY;
  return collect(sv, it, info);
}

int gnp_server_wait(gnp_server* h, long long ticket, double timeout_s, gnp_solve_info* info) {
  GNP_REQUIRE(h, "gnp_server_wait: null server");
  Server* sv = h->s;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  GNP_REQUIRE(it != sv->all.end(), "gnp_server_wait: unknown ticket %lld", ticket);
  Request* r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s));
  while (r->status < 0) {
    if (sv->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && r->status < 0) {
      set_error("gnp_server_wait: ticket %lld still running after %.3f s", ticket, timeout_s);
      return GNP_ERR_TIMEOUT;
    }
  }
  return collect(sv, sv->all.find(ticket), info);
}

int gnp_server_stats(gnp_server* h, gnp_server_stats_t* out) {
  GNP_REQUIRE(h && out, "gnp_server_stats: null argument");
  Server* sv = h->s;
  std::lock_guard<std::mutex> lk(sv->mu);
  out->queued = (int)sv->queue.size();
  out->active = sv->n_active;
  out->used_bytes = sv->used_bytes;
  out->rounds = sv->rounds;
  out->completed = sv->completed;
  out->max_active_seen = sv->max_active_seen;
  return GNP_OK;
}

void gnp_server_destroy(gnp_server* h) {
  if (!h) return;
  Server* sv = h->s;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    // requests still queued are abandoned: they finish with GNP_ERR_TIMEOUT
    for (Request* r : sv->queue) {
      r->status = GNP_ERR_TIMEOUT;
      r->info.status = GNP_ERR_TIMEOUT;
    }
    sv->queue.clear();
  }
  sv->cv.notify_all();
  if (sv->loop.joinable()) sv->loop.join();
  for (auto& kv : sv->all) {
    release(kv.second);
    delete kv.second;
  }
  delete sv;
  delete h;
}

}  // extern "C"
