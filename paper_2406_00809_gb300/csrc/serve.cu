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
//
// Grouped steps (gnp_server_config::grouped): requests whose GNP runs on the short-row
// layer kernels share one stream and advance one FGMRES step per round, every kernel of
// the step launched once for all of them over a work table (each request's own grid,
// GTable; its data, GSlot).  A round is the encoder, the L Res-GCONV layers, the two CGS2
// passes and the cycle end (x update, residual) of every grouped request; the cycle-end
// kernels act only for the requests whose cycle ends in that round, and the residual's
// last block applies the stopping rules on the device (GCtl), so rounds need no host.
// GROUP_ROUNDS rounds are captured as one CUDA graph per set of grouped requests, and at
// most two launches of it are in flight.  After each launch the loop reads the control
// blocks (pinned copy + event).  A request that is done has its final x and state (its
// kernels do nothing from then on): its result is read at once, and its memory is freed
// once every launch that still names it has completed.  A waiting request is set up on a
// second stream and its slot filled, the rounds captured again on that stream while the
// launches in flight run: admission every GROUP_ROUNDS steps, without draining the GPU.
// The grouped step follows the two-pass CGS2 schedule of fgmres_solve (GNP_ORTHO=cgs2),
// kernel for kernel.
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
  // grouped steps: the request's slot, and the stopping rules' outcome (read from its
  // control block; the request is released at the next rebuild)
  bool grouped = false;
  int slot = -1;
  bool retire = false;
  int end_status = GNP_OK;
};

// Rounds (FGMRES steps of every grouped request) per launch of the captured graph.
constexpr int GROUP_ROUNDS = 8;

// The grouped requests: the rounds' stream and a second one (set-up and capture), the
// device slot array and control blocks, the graph of GROUP_ROUNDS rounds, the launches in
// flight (each followed by a copy of the control blocks to pinned memory and an event),
// and the released requests and graphs that launches in flight may still name.
struct Group {
  cudaStream_t stream = nullptr, aux = nullptr;
  GSlot* d_slots = nullptr;
  GCtl* d_ctl = nullptr;
  GCtl* h_ctl = nullptr;  // pinned
  GSlot h_slots[GT_MAX] = {};
  Request* req[GT_MAX] = {};
  bool busy[GT_MAX] = {};  // released, but a launch in flight may still name the slot
  cudaGraphExec_t exec = nullptr;
  std::deque<cudaEvent_t> launches;
  std::deque<unsigned long long> launch_seq;  // the launches' numbers (1, 2, ...)
  unsigned long long seq = 0;                 // launches issued
  unsigned long long since[GT_MAX] = {};      // the first launch after slot k was filled
  struct Grave {
    cudaEvent_t ev;  // recorded after the last launch that may name these
    std::vector<Request*> reqs;
    std::vector<int> slots;
    cudaGraphExec_t exec;
  };
  std::deque<Grave> graves;
  std::vector<cudaEvent_t> pool;
  int live() const {
    int c = 0;
    for (Request* r : req) c += r != nullptr;
    return c;
  }
  int used() const {
    int c = 0;
    for (int k = 0; k < GT_MAX; ++k) c += req[k] != nullptr || busy[k];
    return c;
  }
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
  // statistics (`rounds`: restart cycles run; a grouped request's are counted when it ends)
  long long rounds = 0, completed = 0, admitted = 0, max_active_seen = 0;
  int error = GNP_OK;
  char errmsg[256] = {0};
  Group grp;  // loop thread only (besides its slot count, grp_used, published under the lock)
  int grp_used = 0;
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

// Allocate the request's workspace, run its initial residual on `st` and apply the checks
// that can end a solve before its first cycle.  Returns true when the request still runs.
static bool prepare(Server* sv, Request* r, int s, cudaStream_t st) {
  if (s == GNP_OK) s = solver_create(r->A->n, r->m, r->maxiters, &r->S);
  if (s == GNP_OK && r->M) s = apply_ws_alloc(r->ws, r->A->n);
  if (s == GNP_OK && cudaMallocHost(reinterpret_cast<void**>(&r->mirror), sizeof(DevState)) != cudaSuccess) {
    set_error("server: cudaMallocHost failed");
    s = GNP_ERR_OOM;
  }
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
  return true;
}

// Allocate the request's workspace and stream, run its initial residual, capture and
// instantiate its cycle graph.  Returns true when the request is still running afterwards.
static bool setup(Server* sv, Request* r) {
  int s = GNP_OK;
  if (cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess) {
    set_error("server: stream or event creation failed");
    s = GNP_ERR_CUDA;
  }
  cudaStream_t st = r->stream;
  if (!prepare(sv, r, s, st)) return false;
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

// ---------------------------------------------------------------- grouped steps

static cudaEvent_t group_event(Group& G) {
  cudaEvent_t e = nullptr;
  if (!G.pool.empty()) {
    e = G.pool.back();
    G.pool.pop_back();
  } else if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
    e = nullptr;
  }
  return e;
}

// Every grouped request ends with `status` (a launch or the device failed).
static void group_fail_all(Server* sv, int status) {
  for (Request* r : sv->grp.req)
    if (r && !r->retire) {
      r->retire = true;
      r->end_status = status;
    }
}

// Read the launches that have completed (blocking: all of them): requests whose control
// block says done are to be released.  Returns whether any launch completed.
static bool group_poll(Server* sv, bool block) {
  Group& G = sv->grp;
  bool any = false;
  while (!G.launches.empty()) {
    const cudaError_t q = block ? cudaEventSynchronize(G.launches.front()) : cudaEventQuery(G.launches.front());
    if (q == cudaErrorNotReady) break;
    const unsigned long long s = G.launch_seq.front();
    G.pool.push_back(G.launches.front());
    G.launches.pop_front();
    G.launch_seq.pop_front();
    any = true;
    if (q != cudaSuccess) {
      set_error("server: grouped round failed: %s", cudaGetErrorString(q));
      group_fail_all(sv, GNP_ERR_CUDA);
      continue;
    }
    // h_ctl holds the copy of launch s or a later one (done never reverts); a slot filled
    // after launch s was issued may still hold its previous request's block there
    for (int k = 0; k < GT_MAX; ++k) {
      Request* r = G.req[k];
      if (r && !r->retire && s >= G.since[k] && G.h_ctl[k].done) {
        r->retire = true;
        r->end_status = G.h_ctl[k].status;
      }
    }
  }
  return any;
}

// Free what no launch in flight names any more (blocking: everything); the released
// requests' results are then published (`ended`).
static void group_bury(Server* sv, std::vector<Request*>& ended, bool block) {
  Group& G = sv->grp;
  while (!G.graves.empty()) {
    Group::Grave& g = G.graves.front();
    const cudaError_t q = block ? cudaEventSynchronize(g.ev) : cudaEventQuery(g.ev);
    if (q == cudaErrorNotReady) break;
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (int k : g.slots) G.busy[k] = false;
    for (Request* r : g.reqs) {
      finish(sv, r, r->end_status);
      ended.push_back(r);
    }
    G.pool.push_back(g.ev);
    G.graves.pop_front();
  }
}

// Capture GROUP_ROUNDS rounds for the current grouped requests on the second stream: per
// class of hidden precision and layer form the GNP application, then the CGS2 passes and
// the cycle end of all of them.  The previous graph goes to the graveyard with `grave`.
static int group_capture(Server* sv, Group::Grave& grave) {
  Group& G = sv->grp;
  grave.exec = G.exec;
  G.exec = nullptr;
  std::vector<GHost> all;
  std::vector<std::vector<GHost>> cls(4);
  int m = 0;
  for (int k = 0; k < GT_MAX; ++k) {
    Request* r = G.req[k];
    if (!r) continue;
    const GHost h{k, r->A->n, r->M};
    all.push_back(h);
    cls[(r->M->hprec == GNP_H_BF16 ? 2 : 0) + (r->M->cfg.form == GNP_LAYER_PAPER ? 0 : 1)].push_back(h);
    m = r->m;
  }
  if (all.empty()) return GNP_OK;
  GNP_TRY_CUDA(cudaStreamBeginCapture(G.aux, cudaStreamCaptureModeThreadLocal));
  int s = GNP_OK;
  for (int round = 0; round < GROUP_ROUNDS && s == GNP_OK; ++round) {
    for (const auto& c : cls)
      if (s == GNP_OK) s = grouped_apply_launch(c, G.d_slots, G.aux);
    if (s == GNP_OK) s = grouped_krylov_launch(all, G.d_slots, G.aux);
    if (s == GNP_OK) s = grouped_cycle_end_launch(all, m, G.d_slots, G.aux);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(G.aux, &graph);
  if (s != GNP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (ce == cudaSuccess) ce = cudaGraphInstantiate(&G.exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    set_error("server: capture of the grouped rounds failed: %s", cudaGetErrorString(ce));
    G.exec = nullptr;
    return GNP_ERR_CUDA;
  }
  return GNP_OK;
}

// Fill slot k for request r (set up already): its GSlot and a fresh control block.
static int group_fill(Group& G, int k, Request* r) {
  const GCtl c0{-1, 0, GNP_OK, 0, 0, 0, 0, 0};
  Solver* S = r->S;
  GSlot d{};
  d.gc = G.d_ctl + k;
  d.m = r->m;
  d.rp = r->A->rp;
  d.col = r->A->col;
  d.val = r->A->val;
  d.valhat = r->M->valhat;
  d.n = r->A->n;
  d.L = r->M->cfg.L;
  d.noscale = r->M->cfg.no_scale ? 1 : 0;
  d.sqrt_n = std::sqrt((double)r->A->n);
  d.Hh[0] = r->ws.H[0];
  d.Hh[1] = r->ws.H[1];
  d.tau = r->ws.tau;
  d.V = S->V;
  d.Z = S->Z;
  d.w = S->w;
  d.st = S->st;
  d.Hb = S->H;
  d.R = S->R;
  d.cs = S->cs;
  d.sn = S->sn;
  d.g = S->g;
  d.h1 = S->h1;
  d.h2 = S->h2;
  d.hf = S->hf;
  d.hist = S->hist;
  d.thist = S->thist;
  d.partials = S->red.partials;
  d.counter = S->red.counter;
  d.b = r->b;
  d.x = r->x;
  G.h_slots[k] = d;
  // the launches in flight do not name slot k (it is neither live nor busy): write its entries
  GNP_TRY_CUDA(cudaMemcpyAsync(G.d_slots + k, &G.h_slots[k], sizeof(GSlot), cudaMemcpyHostToDevice, G.aux));
  GNP_TRY_CUDA(cudaMemcpyAsync(G.d_ctl + k, &c0, sizeof(GCtl), cudaMemcpyHostToDevice, G.aux));
  GNP_TRY_CUDA(cudaStreamSynchronize(G.aux));
  r->slot = k;
  G.req[k] = r;
  G.since[k] = G.seq + 1;
  return GNP_OK;
}

// Release the requests that are done (their results read now, their memory freed once no
// launch in flight names them) and admit `fresh` (grouped requests from the queue), then
// capture the rounds again.  Requests that end at set-up go to `ended`.
static void group_rebuild(Server* sv, std::vector<Request*>& fresh, std::vector<Request*>& ended) {
  Group& G = sv->grp;
  if (!G.stream) {
    int e = GNP_OK;
    if (cudaStreamCreateWithFlags(&G.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&G.aux, cudaStreamNonBlocking) != cudaSuccess)
      e = GNP_ERR_CUDA;
    if (e == GNP_OK) e = dev_alloc(&G.d_slots, (size_t)GT_MAX);
    if (e == GNP_OK) e = dev_alloc(&G.d_ctl, (size_t)GT_MAX);
    if (e == GNP_OK && cudaMallocHost(reinterpret_cast<void**>(&G.h_ctl), sizeof(GCtl) * GT_MAX) != cudaSuccess)
      e = GNP_ERR_OOM;
    if (e != GNP_OK) {
      set_error("server: grouped streams, slot array or control blocks");
      for (Request* r : fresh) {
        finish(sv, r, GNP_ERR_CUDA);
        ended.push_back(r);
      }
      fresh.clear();
      return;
    }
  }
  Group::Grave grave{nullptr, {}, {}, nullptr};
  for (int k = 0; k < GT_MAX; ++k) {
    Request* r = G.req[k];
    if (!r || !r->retire) continue;
    // a done request's kernels no longer write its state or x: read its result now
    GCtl c{};
    if (cudaMemcpy(&c, G.d_ctl + k, sizeof(GCtl), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(r->mirror, r->S->st, sizeof(DevState), cudaMemcpyDeviceToHost) != cudaSuccess) {
      if (r->end_status == GNP_OK) r->end_status = GNP_ERR_CUDA;
    } else if (c.done && r->end_status != GNP_ERR_CUDA) {
      r->end_status = c.status;  // the pinned copy read by the loop may have been in flight
    }
    r->ctl.stagn = c.stagn;
    r->ctl.mism = c.mism;
    r->ctl.restarts = c.restarts;
    r->ctl.cycles = c.cycles;
    sv->rounds += c.cycles;
    fill_result(r);
    grave.reqs.push_back(r);
    grave.slots.push_back(k);
    G.busy[k] = true;
    G.req[k] = nullptr;
  }
  for (Request* r : fresh) {
    ++sv->admitted;
    if (!prepare(sv, r, GNP_OK, G.aux)) {
      fill_result(r);
      ended.push_back(r);
      continue;
    }
    int k = 0;
    while (G.req[k] || G.busy[k]) ++k;  // admission left a free slot for every grouped request
    if (group_fill(G, k, r) != GNP_OK) {
      finish(sv, r, GNP_ERR_CUDA);
      ended.push_back(r);
    }
  }
  fresh.clear();
  const int cs = group_capture(sv, grave);
  grave.ev = group_event(G);
  if (!grave.ev || cudaEventRecord(grave.ev, G.stream) != cudaSuccess) {
    // no event: wait for the launches in flight here instead
    cudaStreamSynchronize(G.stream);
    if (grave.ev) G.pool.push_back(grave.ev);
    grave.ev = group_event(G);
    if (grave.ev) cudaEventRecord(grave.ev, G.stream);
  }
  if (grave.ev) G.graves.push_back(grave);
  if (cs != GNP_OK) group_fail_all(sv, GNP_ERR_CUDA);
}

// Launch the captured rounds again unless two launches are still in flight; then the copy
// of the control blocks and an event.  Returns whether it launched.
static bool group_launch(Server* sv) {
  Group& G = sv->grp;
  if (!G.exec || G.launches.size() >= 2) return false;
  cudaEvent_t ev = group_event(G);
  if (!ev || cudaGraphLaunch(G.exec, G.stream) != cudaSuccess ||
      cudaMemcpyAsync(G.h_ctl, G.d_ctl, sizeof(GCtl) * GT_MAX, cudaMemcpyDeviceToHost, G.stream) != cudaSuccess ||
      cudaEventRecord(ev, G.stream) != cudaSuccess) {
    set_error("server: grouped round launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    if (ev) G.pool.push_back(ev);
    group_fail_all(sv, GNP_ERR_CUDA);
    return false;
  }
  G.launches.push_back(ev);
  G.launch_seq.push_back(++G.seq);
  return true;
}

static void group_destroy(Group& G) {
  if (G.stream) cudaStreamSynchronize(G.stream);
  if (G.aux) cudaStreamSynchronize(G.aux);
  if (G.exec) cudaGraphExecDestroy(G.exec);
  for (auto& g : G.graves) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    G.pool.push_back(g.ev);
  }
  G.graves.clear();
  for (cudaEvent_t e : G.launches) G.pool.push_back(e);
  for (cudaEvent_t e : G.pool) cudaEventDestroy(e);
  G.pool.clear();
  G.launches.clear();
  G.launch_seq.clear();
  if (G.stream) cudaStreamDestroy(G.stream);
  if (G.aux) cudaStreamDestroy(G.aux);
  dev_free(G.d_slots);
  dev_free(G.d_ctl);
  if (G.h_ctl) cudaFreeHost(G.h_ctl);
  G.h_ctl = nullptr;
  G.exec = nullptr;
  G.stream = G.aux = nullptr;
}

static void server_loop(Server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    // admission (under the lock): FIFO, by slot count and device-memory footprint
    std::vector<Request*> fresh, gfresh, ended;
    while (!sv->queue.empty() &&
           (int)(sv->running.size() + sv->grp_used + fresh.size() + gfresh.size()) < sv->cfg.max_active) {
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
      // a request that can run in grouped steps always does (its result must not depend on
      // the load), so it waits for a grouped slot
      const bool grp = sv->cfg.grouped && grouped_ok(r->M);
      if (grp && sv->grp_used + (int)gfresh.size() >= GT_MAX) break;
      sv->queue.pop_front();
      sv->used_bytes += r->footprint;
      r->grouped = grp;
      (grp ? gfresh : fresh).push_back(r);
    }
    if (sv->stop && sv->queue.empty() && sv->running.empty() && sv->grp_used == 0 && fresh.empty() &&
        gfresh.empty())
      break;
    if (sv->running.empty() && sv->grp_used == 0 && fresh.empty() && gfresh.empty()) {
      sv->cv.wait_for(lk, std::chrono::milliseconds(50));
      continue;
    }
    lk.unlock();
    bool progressed = !fresh.empty() || !gfresh.empty();
    // grouped requests: read finished cycle ends; release and admit (rebuilding the round)
    progressed |= group_poll(sv, false);
    const size_t buried = ended.size();
    group_bury(sv, ended, false);
    progressed |= ended.size() > buried;
    bool rebuild = !gfresh.empty();
    for (Request* r : sv->grp.req) rebuild |= r && r->retire;
    if (rebuild) group_rebuild(sv, gfresh, ended);
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
    const int glive = sv->grp.live();
    sv->max_active_seen = std::max<long long>(sv->max_active_seen, (long long)(sv->running.size() + glive));
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
    if (glive > 0) progressed |= group_launch(sv);
    for (Request* r : ended) release(r);
    lk.lock();
    for (Request* r : ended) {
      sv->used_bytes -= r->footprint;
      r->status = r->result;
      ++sv->completed;
    }
    sv->grp_used = sv->grp.used();
    sv->n_active = (int)sv->running.size() + glive;
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
  group_destroy(sv->grp);
  for (auto& kv : sv->all) {
    release(kv.second);
    delete kv.second;
  }
  delete sv;
  delete h;
}

}  // extern "C"
