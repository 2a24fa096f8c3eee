// FGMRES device state and workspace (krylov.cu), shared with the solve server (serve.cu).
#pragma once

#include <vector>

#include "internal.h"

namespace gnp {

enum : int {
  FL_EST_CONV = 1,
  FL_BREAKDOWN = 2,
  FL_DROPPED = 4,
  FL_NAN = 8,
  FL_MAXIT = 16,
  FL_FULL = 32,
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
  int pad;
  double bnorm, tol, rtol, beta, vscale, wnorm0, hn, res_est;
};

constexpr double BREAKDOWN_REL = 1e-14;

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
  double* hist = nullptr;  // [maxiters+1]
  RedScratch red;
  // captured restart cycle
  cudaGraphExec_t gexec = nullptr;
  const void* g_model = nullptr;
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


// Enqueue ||b||, the initial residual and the state reset of a solve on `st`.
int solve_init_launch(const gnp_mat* A, Solver* S, const double* b, double* x, double rtol, int maxiters,
                      int m, cudaStream_t st);
// Enqueue one restart cycle (m Arnoldi steps, x update, residual).
int launch_cycle(gnp_mat* A, Solver* S, gnp_model* M, int m, const double* b, double* x,
                 cudaStream_t st, bool prof, const ApplyWs* ws);

// Host bookkeeping between cycles (the stopping rules of the oracle's documentation).
struct CycleCtl {
  int stagn = 0, mism = 0, restarts = 0, cycles = 0;
};
// After a cycle whose state is hs and whose starting residual was beta_prev: returns true
// when the solve ends, with *status set.
bool cycle_after(const DevState& hs, double beta_prev, int maxiters, CycleCtl& c, int* status);

}  // namespace gnp
