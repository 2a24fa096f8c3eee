// FGMRES device state and workspace (krylov.cu), shared with the solve server (serve.cu).
#pragma once

#include <vector>

#include <algorithm>
#include <cstdlib>

#include "internal.h"

namespace gnp {

enum : int {
  FL_EST_CONV = 1,
  FL_BREAKDOWN = 2,
  FL_DROPPED = 4,
  FL_NAN = 8,
  FL_MAXIT = 16,
  FL_FULL = 32,
  FL_TIMEOUT = 64,
};

struct DevState {
  int j;        // current Arnoldi step within the cycle   (ctl[0])
  int active;   // 1 while the cycle runs                    (ctl[1])
  int iters;    // Arnoldi steps so far
  int maxiters;
  int m;        // restart length
  int jj;       // columns used by the cycle-end update
  int flags;
  int last_flags;  // flags of the cycle that just ended (kept by k_residual)
  int last_jj;     // columns that cycle used
  int jv;          // step j whose basis vector k_vnext forms (set by k_cgs<4>)
  double bnorm, tol, rtol, beta, vscale, wnorm0, hn, res_est;
  double w1sq;     // ||w1||^2 of step jv (k_cgs<4>)
  unsigned long long t0;          // %globaltimer (ns) when the solve began
  unsigned long long timeout_ns;  // 0: no time limit
};

// Device clock in nanoseconds (the PTX %globaltimer register, common to all SMs).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr double BREAKDOWN_REL = 1e-14;

// Grid of the CGS2 kernels: one block per SM while the rows are few enough that L2
// latency, not bandwidth, bounds the basis reads (each block then reduces once per
// column chunk, and the float64 pipes of all SMs share the work evenly); up to four per
// SM on larger systems for memory parallelism.  Never more than red_blocks(n), the
// capacity of the partial-sum scratch.
// GNP_DOT_BLOCKS_PER_SM=1..4 in the environment forces the blocks per SM (for tuning).
inline int dot_blocks(int n) {
  static const char* e = getenv("GNP_DOT_BLOCKS_PER_SM");
  static const int forced = e ? atoi(e) : 0;
  const int per = (n + NUM_SMS_GB300 * RED_THREADS * 2 - 1) / (NUM_SMS_GB300 * RED_THREADS * 2);
  const int bps = (forced >= 1 && forced <= 4) ? forced : std::max(1, std::min(4, per));
  return std::min(red_blocks(n), NUM_SMS_GB300 * bps);
}

constexpr int KC = 8;  // basis columns per register chunk
constexpr int RSTRIDE = RED_THREADS + 8;  // row stride of the reduction transpose (doubles)
static_assert(RED_THREADS == TILE && RED_THREADS / 32 == KC, "one warp per chunk column");

// Block-wide sums of KC values per thread (256 threads): the values are transposed
// through shared memory (sh: KC * RSTRIDE doubles) so that warp w adds column w's 256
// values with 8 sequential adds per lane and one 5-level shuffle tree, instead of one
// tree per value per warp.  GB300 executes float64 adds at 2 per SM per cycle, so
// the number of tree levels, not the memory traffic, decides these kernels' cost.
// ACC: dst[w] += sum (shared accumulators); else dst[w] = sum.  Fixed order.
template <bool ACC>
__device__ __forceinline__ void block_reduce_kc(const double (&a)[KC], double* sh, double* dst, int kvalid) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
#pragma unroll
  for (int kc = 0; kc < KC; ++kc) sh[kc * RSTRIDE + t] = a[kc];
  __syncthreads();
  if (w < kvalid) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < RED_THREADS / 32; ++i) s += sh[w * RSTRIDE + lane + 32 * i];
    s = warp_sum(s);
    if (lane == 0) {
      if (ACC) dst[w] += s;
      else dst[w] = s;
    }
  }
  __syncthreads();
}


// One thread finishes Arnoldi step j of its system (Sec. 2.1, Algorithm 1): col[0..j]
// holds h_{0..j,j} (it is rotated in place, col needs j+2 entries), hn = h_{j+1,j};
// scs/ssn are the previous rotations.  Stores column j of H_bar, applies the previous
// Givens rotations and the new one (rho = hypot(a, b), c = a/rho, s = b/rho; rho = 0
// gives c = 1, s = 0), updates g and the residual estimate |g_{j+1}| (Sec. 4), records
// the iteration's residual and device time, and decides whether the cycle continues.
__device__ __forceinline__ void arnoldi_step_finish(DevState* st, int j, double* col, double hn,
                                                    const double* scs, const double* ssn, double* H,
                                                    double* R, double* cs, double* sn, double* g,
                                                    double* hist, unsigned long long* thist) {
  // one serial thread: the state and g_j come in with one batch of loads and go back at
  // the end, so that no store to H or R forces a reload of a state field in between
  DevState s = *st;
  const double gj = g[j];
  const int m = s.m;
  const int ldh = m + 1;
  s.hn = hn;
  bool finite = isfinite(hn);
  for (int i = 0; i <= j; ++i) H[(size_t)j * ldh + i] = col[i];
  col[j + 1] = hn;
  H[(size_t)j * ldh + j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double t = scs[i] * col[i] + ssn[i] * col[i + 1];
    col[i + 1] = -ssn[i] * col[i] + scs[i] * col[i + 1];
    col[i] = t;
  }
  for (int i = 0; i <= j + 1; ++i) finite = finite && isfinite(col[i]);
  const double a = col[j], b = col[j + 1];
  const double rho = hypot(a, b);
  double c = 1.0, sv = 0.0;
  if (rho != 0.0) {
    c = a / rho;
    sv = b / rho;
  }
  const int iters = s.iters + 1;
  s.iters = iters;
  const unsigned long long elapsed = global_ns() - s.t0;
  thist[iters] = elapsed;
  const double wn0 = s.wnorm0;
  int flags = 0;
  int jj;
  if (!finite || !isfinite(rho)) {
    flags |= FL_NAN;
    jj = j;
  } else if (rho <= BREAKDOWN_REL * wn0) {
    hist[iters] = fabs(gj) / s.bnorm;
    flags |= FL_DROPPED;
    jj = j;
  } else {
    cs[j] = c;
    sn[j] = sv;
    col[j] = rho;
    col[j + 1] = 0.0;
    for (int i = 0; i <= j + 1; ++i) R[(size_t)j * ldh + i] = col[i];
    g[j + 1] = -sv * gj;
    g[j] = c * gj;
    jj = j + 1;
    const double res = fabs(-sv * gj);
    s.res_est = res;
    hist[iters] = res / s.bnorm;
    if (hn <= BREAKDOWN_REL * wn0) flags |= FL_BREAKDOWN;
    else if (res <= s.tol) flags |= FL_EST_CONV;
    else if (iters >= s.maxiters) flags |= FL_MAXIT;
    else if (s.timeout_ns != 0ull && elapsed >= s.timeout_ns) flags |= FL_TIMEOUT;
    else if (j + 1 >= m) flags |= FL_FULL;
  }
  s.jj = jj;
  s.flags = flags;
  if (flags) {
    s.active = 0;
  } else {
    s.j = j + 1;
    s.vscale = hn;
  }
  *st = s;
}


struct Solver {
  int n = 0, m_cap = 0, maxit_cap = -1;
  double* V = nullptr;   // [n*(m+1)] column-major basis
  float* Z = nullptr;    // [n*m] preconditioned directions
  double* w = nullptr;   // [n]
  DevState* st = nullptr;
  DevState* st_host = nullptr;  // pinned mirror
  double* H = nullptr;   // [(m+1)*m] unrotated H_bar of the current cycle
  double* R = nullptr;   // [(m+1)*m] rotated (upper triangular part used)
  double* cs = nullptr;
  double* sn = nullptr;
  double* g = nullptr;   // [m+1]
  double* h1 = nullptr;  // [m+2]
  double* h2 = nullptr;  // [m+2]
  double* Zd = nullptr;   // [n*m] float64 directions (Jacobi and inner-GMRES preconditioners)
  int zd_m = 0;
  double* hist = nullptr;  // [maxiters+1]
  unsigned long long* thist = nullptr;  // [maxiters+1] ns since DevState::t0 at each iteration
  RedScratch red;
  // captured restart cycle
  cudaGraphExec_t gexec = nullptr;
  const void* g_model = nullptr;  // the preconditioner the graph was captured for
  int g_kind = -1;
  unsigned long long g_version = 0;
  int g_m = 0, g_hprec = -1;
  const double* g_b = nullptr;
  double* g_x = nullptr;
  cudaStream_t g_stream = nullptr;
  cudaStream_t own = nullptr;  // used when the caller passes the legacy default stream
  // optional timing of the Res-GCONV launches: events[(j*L + l)*2 + {0,1}]
  std::vector<cudaEvent_t> events;
  int ev_L = 0, ev_m = 0;
  bool g_prof = false;
};


// Inner GMRES used as a preconditioner (Sec. 3 "Compared methods"): one cycle of at most
// `iters` Arnoldi steps from x0 = 0, ended early when the Givens estimate reaches
// rtol * ||v||.  Owns its Krylov workspace, so it can run inside an outer FGMRES step.
struct InnerGmres {
  Solver* S = nullptr;
  double* b = nullptr;  // [n] right-hand side (the outer basis vector)
  double* x = nullptr;  // [n] iterate
  int iters = 10;
  double rtol = 1e-6;
};

// The right preconditioner of a solve.
struct Prec {
  int kind = GNP_PRECOND_IDENTITY;
  gnp_model* M = nullptr;         // GNP
  const double* dinv = nullptr;   // Jacobi: 1 / a_ii (1 where a_ii = 0)
  InnerGmres* inner = nullptr;    // GMRES
  const void* key = nullptr;      // identity of the object (graph cache)
};

// z = P(v) for P = Jacobi: v (read through ColPtr) is first divided by outer->vscale and
// written back when outer is non-null (the outer step's normalisation of v_j); every
// kernel returns at once when outer->active == 0.  z: float64 column.
int jacobi_launch(const double* dinv, ColPtr v, DevState* outer, ColPtr z, int n, cudaStream_t st);
// The same for P = inner GMRES (krylov.cu).
int inner_gmres_launch(gnp_mat* A, InnerGmres* G, ColPtr v, DevState* outer, ColPtr z, cudaStream_t st);
int inner_gmres_create(int n, int iters, double rtol, InnerGmres** out);
void inner_gmres_free(InnerGmres* G);

// The solver-side view of a gnp_precond handle (precond.cu).
Prec precond_view(gnp_precond* P);
const gnp_mat* precond_matrix(const gnp_precond* P);

// Enqueue ||b||, the initial residual and the state reset of a solve on `st`.
int solve_init_launch(const gnp_mat* A, Solver* S, const double* b, double* x, double rtol, int maxiters,
                      int m, double timeout_s, cudaStream_t st);
// Enqueue one restart cycle (m Arnoldi steps, x update, residual).
int launch_cycle(gnp_mat* A, Solver* S, const Prec& P, int m, const double* b, double* x,
                 cudaStream_t st, bool prof, const ApplyWs* ws);
// Float64 direction storage for the Jacobi / inner-GMRES preconditioners.
int solver_ensure_zd(Solver* S, int m);

// Host bookkeeping between cycles (the stopping rules of the oracle's documentation).
struct CycleCtl {
  int stagn = 0, mism = 0, restarts = 0, cycles = 0;
};
// After a cycle whose state is hs and whose starting residual was beta_prev: returns true
// when the solve ends, with *status set.
bool cycle_after(const DevState& hs, double beta_prev, int maxiters, CycleCtl& c, int* status);

}  // namespace gnp
