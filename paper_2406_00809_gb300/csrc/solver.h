// FGMRES device state and workspace (krylov.cu), shared with the solve server (serve.cu).
#pragma once

#include <vector>

#include <algorithm>
#include <cstdlib>
#include <cstring>

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
  // Overlapped CGS2 (delayed reorthogonalisation): the first pass of step jd wrote
  int jd;          // the step whose first pass finished last
  double rho;      // the normalisation of v'_{s+1}: max(rho_s, RHO_FLOOR ||w_s||)
  double rho_est;  // rho_s = ||w_s - V_s h_s|| by the first pass (Pythagorean)
  double rho_inv;  // 1 / rho (0 after a breakdown)
  double nu_inv;   // 1 / nu_s, nu_s = ||v'_s - V_{s-1} a_s|| (the second pass of step s)
  int fresh;       // 1 from a cycle's restart (k_residual) until the first pass of its first
                   // step (k_spmv_dot_row): tells the grouped encoder which body to run
};

// Device clock in nanoseconds (the PTX %globaltimer register, common to all SMs).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr double BREAKDOWN_REL = 1e-14;

// The overlapped CGS2 schedule of the GNP-preconditioned step (the default; GNP_ORTHO=cgs2
// in the environment selects CGS2 with both passes after the SpMV).  Read at every cycle
// launch; the captured cycle graphs are keyed on it.
inline bool ortho_overlapped() {
  const char* e = getenv("GNP_ORTHO");
  return !(e && strcmp(e, "cgs2") == 0);
}

// The Pythagorean rho_s = sqrt(||w_s||^2 - ||h_s||^2) of the overlapped schedule loses its
// digits to cancellation once rho_s / ||w_s|| falls below about sqrt(eps); v'_{s+1} is
// normalised by max(rho_s, RHO_FLOOR ||w_s||) (see krylov.cu).
constexpr double RHO_FLOOR = 1e-7;

// Grid of the CGS2 kernels: about one row per thread, from one block per SM (small
// systems) up to four per SM on larger ones.  The float64 pipes of all SMs share the
// work evenly; a second block per SM hides part of the latency of the other's block
// reduction (65,536 rows: 100.4 against 101.2 us per FGMRES step with one block per SM).
// Capped at red_blocks(n), one row per thread: a grid of whole blocks per SM instead
// (304 blocks of 216 rows at 65,536 rows, not 256 of 256) measured slower, 92 against
// 89 us per step.  GNP_DOT_BLOCKS_PER_SM=1..4 in the environment forces the blocks per SM
// (for tuning).
inline int dot_blocks(int n) {
  static const char* e = getenv("GNP_DOT_BLOCKS_PER_SM");
  static const int forced = e ? atoi(e) : 0;
  const int per = (n + NUM_SMS_GB300 * RED_THREADS - 1) / (NUM_SMS_GB300 * RED_THREADS);
  const int bps = (forced >= 1 && forced <= 4) ? forced : std::max(1, std::min(4, per));
  return forced >= 1 && forced <= 4 ? NUM_SMS_GB300 * bps : std::min(red_blocks(n), NUM_SMS_GB300 * bps);
}

constexpr int KC = 8;  // basis columns per register chunk
constexpr int RED_SH = 32 * (RED_THREADS / 32);  // shared doubles of block_reduce_w
static_assert(KC == 8 && RED_THREADS == TILE && RED_THREADS % 32 == 0, "block_reduce_kc: 8 columns, whole warps");

// Block-wide sums of KW = 8, 16 or 32 values per thread (RED_THREADS threads), in a
// fixed order.  GB300 executes float64 adds at 2 per SM per cycle, so the number of
// warp-wide float64 instructions decides the cost.  Each warp first reduces its 32 lanes
// with a transposing butterfly: at the xor-16 step a lane keeps half of its columns and
// hands the other half to its partner, at xor 8 a quarter, and so on until one column is
// left (KW - 1 adds in all), then the remaining xor steps finish the sum: every lane
// holds the warp total of column (lane >> (5 - log2 KW)) & (KW - 1), for KW + 4 - log2 KW
// adds where a tree per column would take 5 KW.  The warp totals of each column meet in
// shared memory (sh: KW * RED_THREADS / 32 doubles) and are added in warp order.
// ACC: dst[k] += sum (shared accumulators); else dst[k] = sum, for k < kvalid.
template <int KW, bool ACC>
__device__ __forceinline__ void block_reduce_w(const double (&a)[KW], double* sh, double* dst, int kvalid) {
  static_assert(KW == 8 || KW == 16 || KW == 32, "8, 16 or 32 columns");
  constexpr int LV = KW == 8 ? 3 : (KW == 16 ? 4 : 5);  // transposing steps
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  double v[KW];
#pragma unroll
  for (int q = 0; q < KW; ++q) v[q] = a[q];
#pragma unroll
  for (int lv = 0; lv < LV; ++lv) {
    const int m = 16 >> lv;
    const int h = KW >> (lv + 1);
    const bool hi = (lane & m) != 0;
#pragma unroll
    for (int q = 0; q < h; ++q) {
      const double keep = hi ? v[h + q] : v[q];
      const double send = hi ? v[q] : v[h + q];
      v[q] = keep + __shfl_xor_sync(0xffffffffu, send, m);
    }
  }
  double x = v[0];
#pragma unroll
  for (int m = 16 >> LV; m >= 1; m >>= 1) x += __shfl_xor_sync(0xffffffffu, x, m);
  if ((lane & ((1 << (5 - LV)) - 1)) == 0) sh[w * KW + ((lane >> (5 - LV)) & (KW - 1))] = x;
  __syncthreads();
  if (t < kvalid) {
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < RED_THREADS / 32; ++i) s += sh[i * KW + t];
    if (ACC) dst[t] += s;
    else dst[t] = s;
  }
  __syncthreads();
}

template <bool ACC>
__device__ __forceinline__ void block_reduce_kc(const double (&a)[KC], double* sh, double* dst, int kvalid) {
  block_reduce_w<KC, ACC>(a, sh, dst, kvalid);
}

// Per-block partial sums of the dots  sum_i V[k][i] y_i  for k < K over the rows
// i = blockIdx.x * blockDim.x + threadIdx.x + c * gridDim.x * blockDim.x (y = w; column
// `normk`, if any, is y itself, giving ||y||^2) -> part[k], KW columns per pass: one
// pass for up to 32 columns, so that the basis loads of a row are in flight together and
// the block reduces once.
template <int KW>
__device__ __forceinline__ void block_dots_w(VGrid gr, const double* __restrict__ V, const double* __restrict__ w,
                                             int n, int K, int normk, double* sh, double* part) {
  const size_t ld = (size_t)n;
  const int gtid = gr.bid * blockDim.x + threadIdx.x;
  const int gstride = gr.nblk * blockDim.x;
  for (int k0 = 0; k0 < K; k0 += KW) {
    double acc[KW];
#pragma unroll
    for (int kc = 0; kc < KW; ++kc) acc[kc] = 0.0;
    for (int i = gtid; i < n; i += gstride) {
      const double y = w[i];
#pragma unroll
      for (int kc = 0; kc < KW; ++kc) {
        const int k = k0 + kc;
        if (k < K) {
          const double vk = (k == normk) ? y : V[k * ld + i];
          acc[kc] += vk * y;
        }
      }
    }
    block_reduce_w<KW, false>(acc, sh, part + k0, min(KW, K - k0));
  }
}

__device__ __forceinline__ void block_dots(VGrid gr, const double* __restrict__ V, const double* __restrict__ w,
                                           int n, int K, int normk, double* sh, double* part) {
  if (K <= 8) block_dots_w<8>(gr, V, w, n, K, normk, sh, part);
  else if (K <= 16) block_dots_w<16>(gr, V, w, n, K, normk, sh, part);
  else block_dots_w<32>(gr, V, w, n, K, normk, sh, part);
}
__device__ __forceinline__ void block_dots(const double* __restrict__ V, const double* __restrict__ w, int n,
                                           int K, int normk, double* sh, double* part) {
  block_dots(hw_grid(), V, w, n, K, normk, sh, part);
}


// The new Givens rotation of Arnoldi step j and what follows it (one thread): a = the
// rotated entry j of column j, b = h_{j+1,j} = hn; `finite` = every other rotated entry
// of the column is finite.  rho = hypot(a, b), c = a/rho, s = b/rho (rho = 0 gives c = 1,
// s = 0); R[j, j] = rho (entries above j are already stored), g and the residual
// estimate |g_{j+1}| (Sec. 4), the iteration's residual and device time, and whether the
// cycle continues.  The state and g_j come in with one batch of loads and go back at the
// end, so that no store to R, g or the histories forces a reload of a state field.
// lagged (one-reduction CGS2): column j is finished one step late, so the step counter
// (advanced by the reduction) and vscale are left alone and wn0 is the column's own ||w||;
// otherwise wn0 < 0 takes st->wnorm0.
__device__ __forceinline__ void arnoldi_step_decide(DevState* st, int j, double a, double hn, bool finite,
                                                    double* R, double* cs, double* sn, double* g,
                                                    double* hist, unsigned long long* thist,
                                                    bool lagged = false, double wn0_in = -1.0) {
  DevState s = *st;
  const double gj = g[j];
  const int m = s.m;
  const int ldh = m + 1;
  s.hn = hn;
  finite = finite && isfinite(hn) && isfinite(a);
  const double rho = hypot(a, hn);
  double c = 1.0, sv = 0.0;
  if (rho != 0.0) {
    c = a / rho;
    sv = hn / rho;
  }
  const int iters = s.iters + 1;
  s.iters = iters;
  const unsigned long long elapsed = global_ns() - s.t0;
  thist[iters] = elapsed;
  const double wn0 = wn0_in >= 0.0 ? wn0_in : s.wnorm0;
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
    R[(size_t)j * ldh + j] = rho;
    R[(size_t)j * ldh + j + 1] = 0.0;
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
  } else if (!lagged) {
    s.j = j + 1;
    s.vscale = hn;
  }
  *st = s;
}

// One thread finishes Arnoldi step j of its system (Sec. 2.1, Algorithm 1): col[0..j]
// holds h_{0..j,j} (it is rotated in place, col needs j+2 entries), hn = h_{j+1,j};
// scs/ssn are the previous rotations.  Stores column j of H_bar, applies the previous
// Givens rotations (entries above j go to R at once: column j of R is read only when the
// step is kept) and then arnoldi_step_decide.
__device__ __forceinline__ void arnoldi_step_finish(DevState* st, int j, double* col, double hn,
                                                    const double* scs, const double* ssn, double* H,
                                                    double* R, double* cs, double* sn, double* g,
                                                    double* hist, unsigned long long* thist,
                                                    bool lagged = false, double wn0 = -1.0) {
  const int ldh = st->m + 1;
  for (int i = 0; i <= j; ++i) H[(size_t)j * ldh + i] = col[i];
  H[(size_t)j * ldh + j + 1] = hn;
  bool finite = true;
  for (int i = 0; i < j; ++i) {
    const double t = scs[i] * col[i] + ssn[i] * col[i + 1];
    col[i + 1] = -ssn[i] * col[i] + scs[i] * col[i + 1];
    col[i] = t;
    R[(size_t)j * ldh + i] = t;
    finite = finite && isfinite(t);
  }
  arnoldi_step_decide(st, j, col[j], hn, finite, R, cs, sn, g, hist, thist, lagged, wn0);
}

// arnoldi_step_finish with the whole block (every thread calls it; col, scs, ssn, xs and
// bs in shared memory, xs and bs with room for j+1 entries).  Applying the previous
// rotations to column j is the recurrence x_{i+1} = -s_i x_i + c_i col_{i+1} (x_0 =
// col_0; x_i is entry i after rotations 0..i-1), whose products c_i col_{i+1} do not
// depend on it: the threads form those products, thread 0 runs the recurrence with one
// fused multiply-add per step, then the threads form the rotated entries
// c_i x_i + s_i col_{i+1} and store them; thread 0 decides.  On GB300 a dependent
// float64 operation costs tens of cycles, so the serial chain is what this shortens.
__device__ __forceinline__ void arnoldi_step_finish_block(DevState* st, int j, const double* col, double hn,
                                                          const double* scs, const double* ssn, double* xs,
                                                          double* bs, double* H, double* R, double* cs,
                                                          double* sn, double* g, double* hist,
                                                          unsigned long long* thist, bool lagged = false,
                                                          double wn0 = -1.0) {
  const int t = threadIdx.x;
  const int ldh = st->m + 1;
  for (int i = t; i <= j; i += blockDim.x) H[(size_t)j * ldh + i] = col[i];
  if (t == 0) H[(size_t)j * ldh + j + 1] = hn;
  for (int i = t; i < j; i += blockDim.x) bs[i] = scs[i] * col[i + 1];
  __syncthreads();
  if (t == 0) {
    double x = col[0];
    xs[0] = x;
    for (int i = 0; i < j; ++i) {
      x = fma(-ssn[i], x, bs[i]);
      xs[i + 1] = x;
    }
  }
  __syncthreads();
  bool bad = false;
  for (int i = t; i < j; i += blockDim.x) {
    const double ti = fma(scs[i], xs[i], ssn[i] * col[i + 1]);
    R[(size_t)j * ldh + i] = ti;
    bad = bad || !isfinite(ti);
  }
  bad = __syncthreads_or(bad) != 0;
  if (t == 0) arnoldi_step_decide(st, j, xs[j], hn, !bad, R, cs, sn, g, hist, thist, lagged, wn0);
}


// h_{j+1,j} = ||w1 - V h2|| = sqrt(||w1||^2 - ||h2||^2) of step j = st->jv after
// k_cgs<4>: V has orthonormal columns to working precision and h2 = V^T w1; ||h2|| is
// O(eps ||w||) after the first pass, so nothing cancels unless w1 itself is at the
// breakdown level, where the step ends anyway.  Warp 0 of the calling block sums ||h2||^2
// lane-strided with a fixed shuffle tree (the same bits in every block); the result is in
// *out (shared) after the caller's next __syncthreads.
__device__ __forceinline__ void vnext_hnorm(const double* __restrict__ h2, int j, double w1sq, double* out) {
  if (threadIdx.x < 32) {
    double q = 0.0;
    for (int i = threadIdx.x; i <= j; i += 32) q = fma(h2[i], h2[i], q);
    q = warp_sum(q);
    if (threadIdx.x == 0) *out = sqrt(fmax(w1sq - q, 0.0));
  }
}

// Finish step j = st->jv with the whole block: column j of H_bar = h1 + h2 and h_{j+1,j},
// the Givens update and the continue decision (arnoldi_step_finish_block).
__device__ __forceinline__ void vnext_finish(const VNext& a) {
  __shared__ double shh[GNP_MAX_RESTART + 4];
  __shared__ double scs[GNP_MAX_RESTART + 4];
  __shared__ double ssn[GNP_MAX_RESTART + 4];
  __shared__ double sxs[GNP_MAX_RESTART + 4];
  __shared__ double sbs[GNP_MAX_RESTART + 4];
  __shared__ double shn;
  DevState* st = a.st;
  if (!st->active) return;
  const int j = st->jv;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) shh[i] = a.h1[i] + a.h2[i];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    scs[i] = a.cs[i];
    ssn[i] = a.sn[i];
  }
  vnext_hnorm(a.h2, j, st->w1sq, &shn);
  __syncthreads();
  arnoldi_step_finish_block(st, j, shh, shn, scs, ssn, sxs, sbs, a.H, a.R, a.cs, a.sn, a.g, a.hist, a.thist);
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
  double* hf = nullptr;  // [m+2] overlapped CGS2: the finished column s-1
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
  bool g_dcgs = false;
  // overlapped CGS2: the reorthogonalisation stream and its fork/join events
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
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

// Host bookkeeping between cycles: the stopping rules stated with fgmres_solve in gnp.h
// (true residual at rtol -> OK; two consecutive cycles without decrease -> STAGNATION;
// three consecutive cycles whose estimate met rtol but not the true residual ->
// RESIDUAL_MISMATCH; non-finite -> NAN; maxiters -> NOT_CONVERGED).
struct CycleCtl {
  int stagn = 0, mism = 0, restarts = 0, cycles = 0;
};
// After a cycle whose state is hs and whose starting residual was beta_prev: returns true
// when the solve ends, with *status set.  The stopping rules of fgmres_solve (host, after
// every cycle) and of the solve server's grouped steps (device, at every cycle end).
__host__ __device__ inline bool cycle_after(const DevState& hs, double beta_prev, int maxiters, CycleCtl& c,
                                            int* status) {
  if ((hs.last_flags & FL_NAN) || !isfinite(hs.beta)) {
    *status = GNP_ERR_NAN;
    return true;
  }
  if (hs.beta <= hs.tol) {
    *status = GNP_OK;
    return true;
  }
  if (hs.last_flags & FL_TIMEOUT) {
    *status = GNP_ERR_TIMEOUT;
    return true;
  }
  c.mism = (hs.last_flags & FL_EST_CONV) ? c.mism + 1 : 0;
  c.stagn = (hs.beta >= beta_prev) ? c.stagn + 1 : 0;
  if (c.mism >= 3) {
    *status = GNP_ERR_RESIDUAL_MISMATCH;
    return true;
  }
  if (c.stagn >= 2) {
    *status = GNP_ERR_STAGNATION;
    return true;
  }
  ++c.restarts;
  if (hs.iters >= maxiters) {
    *status = GNP_ERR_NOT_CONVERGED;
    return true;
  }
  return false;
}

}  // namespace gnp
