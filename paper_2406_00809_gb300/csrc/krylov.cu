// Restarted flexible GMRES with a nonlinear right preconditioner (Sec. 2.1, Eq. 1,
// Algorithm 1), float64 throughout except the preconditioner output z_j (float32).
//
// One Arnoldi step j (all on the device, no host round trip):
//   [M]    z_j = M(v_j): the preconditioner's first kernel turns the stored w into
//          v_j = w / h_{j,j-1} (or r / beta) in place (k_vscale for M = I, the Jacobi and
//          inner-GMRES kernels), then writes Z[:, j].  The GNP encoder does more from step
//          1 on: it forms v_j = (w1 - V h2) / h_{j,j-1} itself from the previous step's
//          CGS2 output, while one of its blocks finishes that step (k_encode_vn, gconv.cu),
//          so k_vnext runs only after the cycle's last step.
//   k_spmv_dot    w = A z_j (tile gather, float64 values) fused with CGS2 pass 1:
//                 h1 = V_j^T w and ||w||^2 (the breakdown reference).
//   k_cgs<4>      w1 = w - V_j h1 (in place), h2 = V_j^T w1 and ||w1||^2.
//   k_vnext       block 0 forms column j of H_bar (h1 + h2 and h_{j+1,j} =
//                 sqrt(||w1||^2 - ||h2||^2)), applies the previous Givens rotations and
//                 the new one, updates g and the residual estimate |g_{j+1}| (Sec. 4),
//                 and decides whether the cycle continues; meanwhile the other blocks form
//                 V[:, j+1] = w1 - V_j h2 (normalised by the next step's first kernel).
// The Arnoldi process of the training sampler (arnoldi_basis) keeps the explicit third
// pass: k_spmv_tile, k_cgs<1> (h1, ||w||^2), k_cgs<2> (w1, h2), k_cgs<3> (w2 -> V[:, j+1],
// ||w2||, the same last-block update).
// Cycle end: k_xupdate (y = R^{-1} g by back substitution, x += Z y) and k_residual
// (r = b - A x, beta = ||r||, which restarts the cycle).  Every kernel reads the step
// index j and an `active` flag from device memory, so one captured CUDA graph replays a
// whole restart cycle; steps after an early exit return at once.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "solver.h"

namespace gnp {

static bool g_profile_gconv = false;

__device__ __forceinline__ void* colptr_k(const ColPtr& p) {
  const int j = p.jptr ? *p.jptr : 0;
  return static_cast<char*>(p.base) + (size_t)(j + p.off) * p.stride;
}

static int ensure_events(Solver* S, int m, int L) {
  if ((int)S->events.size() >= 2 * m * L && S->ev_L == L) return GNP_OK;
  for (cudaEvent_t e : S->events) cudaEventDestroy(e);
  S->events.assign((size_t)2 * m * L, nullptr);
  for (auto& e : S->events) GNP_TRY_CUDA(cudaEventCreate(&e));
  S->ev_L = L;
  S->ev_m = m;
  return GNP_OK;
}

void solver_free(Solver* s) {
  if (!s) return;
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  if (s->own) cudaStreamDestroy(s->own);
  for (cudaEvent_t e : s->events) cudaEventDestroy(e);
  dev_free(s->V);
  dev_free(s->Z);
  dev_free(s->w);
  dev_free(s->st);
  if (s->st_host) cudaFreeHost(s->st_host);
  dev_free(s->H);
  dev_free(s->R);
  dev_free(s->cs);
  dev_free(s->sn);
  dev_free(s->g);
  dev_free(s->h1);
  dev_free(s->h2);
  dev_free(s->hf);
  dev_free(s->hist);
  dev_free(s->thist);
  red_free(s->red);
  if (s->side) cudaStreamDestroy(s->side);
  if (s->fork) cudaEventDestroy(s->fork);
  if (s->join) cudaEventDestroy(s->join);
  delete s;
}

size_t solver_bytes(int n, int m, int maxiters) {
  const size_t maxb = (size_t)std::max(4 * NUM_SMS_GB300, (n + TILE - 1) / TILE);
  return (size_t)n * (m + 1) * 8 + (size_t)n * m * 4 + (size_t)n * 8 + sizeof(DevState) +
         (size_t)(m + 1) * m * 8 * 2 + (size_t)(5 * m + 10) * 8 + (size_t)(maxiters + 1) * 16 +
         maxb * (m + 2) * 8 + 8;
}

template <class ZT>
__global__ void k_xupdate(const ZT* __restrict__ Z, double* __restrict__ x, int n, const DevState* st,
                          const double* __restrict__ R, const double* __restrict__ g);

static int xupdate_attrs() {
  static bool done = false;
  if (done) return GNP_OK;
  const int bytes = (int)sizeof(double) * GNP_MAX_RESTART * GNP_MAX_RESTART;
  GNP_TRY_CUDA(cudaFuncSetAttribute(k_xupdate<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  GNP_TRY_CUDA(cudaFuncSetAttribute(k_xupdate<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  done = true;
  return GNP_OK;
}

int solver_create(int n, int m, int maxiters, Solver** out) {
  *out = nullptr;
  GNP_TRY(xupdate_attrs());
  Solver* s = new Solver();
  s->n = n;
  int e = GNP_OK;
  do {
    if ((e = dev_alloc(&s->V, (size_t)n * (m + 1))) != GNP_OK) break;
    if ((e = dev_alloc(&s->Z, (size_t)n * m)) != GNP_OK) break;
    if ((e = dev_alloc(&s->w, (size_t)n)) != GNP_OK) break;
    if ((e = dev_alloc(&s->st, 1)) != GNP_OK) break;
    if ((e = dev_alloc(&s->H, (size_t)(m + 1) * m)) != GNP_OK) break;
    if ((e = dev_alloc(&s->R, (size_t)(m + 1) * m)) != GNP_OK) break;
    if ((e = dev_alloc(&s->cs, (size_t)m)) != GNP_OK) break;
    if ((e = dev_alloc(&s->sn, (size_t)m)) != GNP_OK) break;
    if ((e = dev_alloc(&s->g, (size_t)m + 1)) != GNP_OK) break;
    if ((e = dev_alloc(&s->h1, (size_t)m + 2)) != GNP_OK) break;
    if ((e = dev_alloc(&s->h2, (size_t)m + 2)) != GNP_OK) break;
    if ((e = dev_alloc(&s->hf, (size_t)m + 2)) != GNP_OK) break;
    if ((e = dev_alloc(&s->hist, (size_t)maxiters + 1)) != GNP_OK) break;
    if ((e = dev_alloc(&s->thist, (size_t)maxiters + 1)) != GNP_OK) break;
    const int maxb = std::max(4 * NUM_SMS_GB300, (n + TILE - 1) / TILE);  // >= dot_blocks(n)
    if ((e = red_alloc(s->red, maxb, m + 2)) != GNP_OK) break;
    if (cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("cudaStreamCreate failed");
      e = GNP_ERR_CUDA;
      break;
    }
    if (cudaMallocHost(reinterpret_cast<void**>(&s->st_host), sizeof(DevState)) != cudaSuccess) {
      set_error("cudaMallocHost failed");
      e = GNP_ERR_OOM;
      break;
    }
  } while (0);
  if (e != GNP_OK) {
    solver_free(s);
    return e;
  }
  s->m_cap = m;
  s->maxit_cap = maxiters;
  *out = s;
  return GNP_OK;
}

static int solver_ensure(gnp_mat* A, int m, int maxiters) {
  Solver* s = A->solver;
  if (s && s->m_cap >= m && s->maxit_cap >= maxiters) return GNP_OK;
  const int m_new = std::max(m, s ? s->m_cap : 0);
  const int it_new = std::max(maxiters, s ? s->maxit_cap : 0);
  solver_free(s);
  A->solver = nullptr;
  return solver_create(A->n, m_new, it_new, &A->solver);
}

// ---------------------------------------------------------------- SpMV traits

template <class XT>
struct TrSpmv {
  static constexpr int G = 1, NV = 1, STRIDE = 1;
  using acc = double;
  using val_t = double;
  using x_t = XT;
  __device__ __forceinline__ static void load(const XT* X, int c, int, double (&h)[1]) {
    h[0] = (double)__ldg(X + c);
  }
};

// y = A x.  x: float64 or float32 column (ColPtr); y float64.
template <class XT>
__global__ void __launch_bounds__(TILE)
k_spmv_tile(const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
            ColPtr xp, double* __restrict__ y, int n, const int* __restrict__ ctl) {
  if (ctl && !ctl[1]) return;
  using TR = TrSpmv<XT>;
  __shared__ TileSmem<TR> sm;
  const XT* x = static_cast<const XT*>(colptr_k(xp));
  const int r0 = blockIdx.x * TILE;
  const int rows = min(TILE, n - r0);
  tile_load_rp<TR>(sm, rp, r0, rows);
  __syncthreads();
  tile_gather<TR>(sm, rows, col, val, x);
  __syncthreads();
  if (threadIdx.x < rows) {
    double s[1];
    tile_row_sum<TR, 1>(sm, threadIdx.x, 0, s);
    y[r0 + threadIdx.x] = s[0];
  }
}

// w = A z (tile gather) fused with CGS2 pass 1: h1 = V_j^T w and ||w||^2.  Blocks loop
// over tiles and keep their dot sums in shared memory, so the partials stay one row
// per block (at most 4 per SM) however large n is.
template <class XT>
__global__ void __launch_bounds__(TILE)
k_spmv_dot(const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
           ColPtr xp, double* __restrict__ w, const double* __restrict__ V, int n, DevState* st,
           double* __restrict__ h1, double* __restrict__ partials, unsigned* counter) {
  if (!st->active) return;
  using TR = TrSpmv<XT>;
  __shared__ TileSmem<TR> sm;
  __shared__ double sacc[GNP_MAX_RESTART + 2];
  __shared__ double sred[RED_SH];
  const int j = st->j;
  const int K = j + 2;  // h1[0..j] and ||w||^2
  const size_t ld = (size_t)n;
  const XT* x = static_cast<const XT*>(colptr_k(xp));
  for (int k = threadIdx.x; k < K; k += blockDim.x) sacc[k] = 0.0;
  const int nt = (n + TILE - 1) / TILE;
  for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const int r0 = tile * TILE;
    const int rows = min(TILE, n - r0);
    __syncthreads();
    tile_load_rp<TR>(sm, rp, r0, rows);
    __syncthreads();
    tile_gather<TR>(sm, rows, col, val, x);
    __syncthreads();
    const int t = threadIdx.x;
    double wr = 0.0;
    if (t < rows) {
      double s1[1];
      tile_row_sum<TR, 1>(sm, t, 0, s1);
      wr = s1[0];
      w[r0 + t] = wr;
    }
    for (int k0 = 0; k0 < K; k0 += 8) {
      double a[8];
#pragma unroll
      for (int kc = 0; kc < 8; ++kc) {
        const int k = k0 + kc;
        double vk = 0.0;
        if (t < rows && k < K) vk = (k == j + 1) ? wr : V[k * ld + r0 + t];
        a[kc] = vk * wr;
      }
      block_reduce_kc<true>(a, sred, sacc + k0, min(8, K - k0));
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < K; k += blockDim.x) partials[(size_t)blockIdx.x * K + k] = sacc[k];
  if (!last_block_arrive(counter)) return;
  __shared__ double shtot[GNP_MAX_RESTART + 2];
  reduce_partials(partials, gridDim.x, K, shtot);
  if (threadIdx.x == 0) {
    for (int k = 0; k <= j; ++k) h1[k] = shtot[k];
    st->wnorm0 = sqrt(shtot[j + 1]);
    *counter = 0;
  }
}

// k_spmv_dot for matrices whose rows are all short (at most SPMV_ROW_DMAX nonzeros): one
// thread per row computes w_i = sum_j a_ij x_j in column order (no slot bookkeeping), then
// the block forms its share of h1 = V_j^T w and ||w||^2 over its rows, KC columns at a
// time, as k_cgs<1> does.  Same result layout and last-block reduction as k_spmv_dot.
constexpr int SPMV_ROW_DMAX = 32;

// w_i = sum_j a_ij x_j for the rows i = blockIdx.x * blockDim.x + threadIdx.x + c * gridDim.x
// * blockDim.x, one thread per row, in column order with eight nonzeros' loads in flight.
template <class XT>
__device__ __forceinline__ void row_spmv(VGrid gr, const int* __restrict__ rp, const int* __restrict__ col,
                                         const double* __restrict__ val, const XT* __restrict__ x,
                                         double* __restrict__ w, int n) {
  const int gtid = gr.bid * blockDim.x + threadIdx.x;
  const int gstride = gr.nblk * blockDim.x;
  for (int i = gtid; i < n; i += gstride) {
    const int rs = __ldg(rp + i), re = __ldg(rp + i + 1);
    double s = 0.0;
    for (int e0 = rs; e0 < re; e0 += 8) {
      int c[8];
      double v[8];
      XT xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const bool ok = e0 + u < re;
        c[u] = ok ? __ldg(col + e0 + u) : 0;
        v[u] = ok ? __ldg(val + e0 + u) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) xv[u] = (e0 + u < re) ? x[c[u]] : XT(0);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (e0 + u < re) s = fma(v[u], (double)xv[u], s);
    }
    w[i] = s;
  }
}

template <class XT>
__device__ __forceinline__ void spmv_dot_row_body(VGrid gr, const int* __restrict__ rp, const int* __restrict__ col,
                                                  const double* __restrict__ val, ColPtr xp, double* __restrict__ w,
                                                  const double* __restrict__ V, int n, DevState* st,
                                                  double* __restrict__ h1, double* __restrict__ partials,
                                                  unsigned* counter) {
  if (!st->active) return;
  __shared__ double sred[RED_SH];
  __shared__ double shtot[GNP_MAX_RESTART + 2];
  const int j = st->j;
  const int K = j + 2;  // h1[0..j] and ||w||^2
  row_spmv(gr, rp, col, val, static_cast<const XT*>(colptr_k(xp)), w, n);
  block_dots(gr, V, w, n, K, j + 1, sred, partials + (size_t)gr.bid * K);
  if (!last_block_arrive(counter, gr.nblk)) return;
  reduce_partials(partials, gr.nblk, K, shtot);
  if (threadIdx.x == 0) {
    for (int k = 0; k <= j; ++k) h1[k] = shtot[k];
    st->wnorm0 = sqrt(shtot[j + 1]);
    st->fresh = 0;
    *counter = 0;
  }
}

template <class XT>
__global__ void __launch_bounds__(RED_THREADS)
k_spmv_dot_row(const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
               ColPtr xp, double* __restrict__ w, const double* __restrict__ V, int n, DevState* st,
               double* __restrict__ h1, double* __restrict__ partials, unsigned* counter) {
  spmv_dot_row_body<XT>(hw_grid(), rp, col, val, xp, w, V, n, st, h1, partials, counter);
}

// ---------------------------------------------------------------- overlapped CGS2
//
// CGS2 with delayed reorthogonalisation (Bielich, Langou, Thomas, Swirydowicz, Yamazaki,
// Boman 2022), arranged so that the second pass runs beside the GNP.  The encoder of step
// s forms v'_s, the first-pass (once orthogonalised, Pythagorean-normalised) vector, and
// z_s = M(v'_s): FGMRES needs only A Z = V_{m+1} H_bar (Sec. 2.1), so any z_s is a valid
// direction.  While the Res-GCONV layers of step s run (float32, on the L2), a second
// stream takes the float64 second pass of v'_s:
//   k_reorth_dots:   a_s = V_{s-1}^T v'_s, beta = ||v'_s||^2 (one grid reduction), nu_s =
//                    sqrt(beta - ||a_s||^2); as v'_s = V_{s-1} a_s + nu_s v_s, column s-1 of
//                    H_bar is [h_{s-1} + rho_{s-1} a_s; rho_{s-1} nu_s]: its Givens update
//                    and the continue decision follow in the same last block;
//   k_reorth_update: v_s = (v'_s - V_{s-1} a_s) / nu_s, in place.
// The main stream then joins it: k_spmv_rdot(_row) forms w_s = A z_s and the first pass
// against the final V_s, h_s = V_s^T w_s and ||w_s||^2 (one grid reduction), rho_s =
// sqrt(||w_s||^2 - ||h_s||^2); the encoder of step s+1 forms v'_{s+1} = (w_s - V_s h_s) /
// rho_s.  The critical path keeps one grid reduction and the first pass; the other half
// of the float64 work overlaps the float32 layers.  The last column of a cycle keeps its
// first-pass values [h_{m-1}; rho_{m-1}] (v'_m is never used; the cycle ends with the
// true residual), finished by k_dfinish.  In exact arithmetic a_s = 0 and nu_s = 1, so
// the steps are those of CGS2; only rounding differs.

// The Pythagorean rho_s loses its digits to cancellation once rho_s / ||w_s|| falls below
// about sqrt(eps) (it can clamp to 0 where the true value is 1e-10 ||w_s||).  Any
// normalisation of v'_{s+1} keeps w_s = V_s h_s + rho v'_{s+1} exact, so v'_{s+1} is divided
// by max(rho_s, RHO_FLOOR ||w_s||) (solver.h), and nu_{s+1} (an explicit norm after
// reorthogonalisation) gives the true subdiagonal rho nu_{s+1} of column s: an exact
// breakdown shows there, one step later, instead of restarting the cycle early on noise.

// Finish column j of H_bar (col: j+1 entries, global; hn its subdiagonal) with the whole
// block, in lagged form (the step counter belongs to the reductions).
__device__ __forceinline__ void finish_col(const VNext& a, int j, const double* col, double hn, double wn0) {
  __shared__ double scol[GNP_MAX_RESTART + 4];
  __shared__ double scs[GNP_MAX_RESTART + 4];
  __shared__ double ssn[GNP_MAX_RESTART + 4];
  __shared__ double sxs[GNP_MAX_RESTART + 4];
  __shared__ double sbs[GNP_MAX_RESTART + 4];
  for (int i = threadIdx.x; i <= j; i += blockDim.x) scol[i] = col[i];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    scs[i] = a.cs[i];
    ssn[i] = a.sn[i];
  }
  __syncthreads();
  arnoldi_step_finish_block(a.st, j, scol, hn, scs, ssn, sxs, sbs, a.H, a.R, a.cs, a.sn, a.g, a.hist, a.thist, true,
                            wn0);
}

// The last block of the first pass of step s: h_s (-> a.h2), rho_s and the state the next
// encoder reads.  The step breaks down only when w_s = 0 or something is not finite;
// column s is then finished at once with its first-pass values (column s-1 was finished
// by the reorthogonalisation branch before this kernel started), which ends the cycle.
__device__ __forceinline__ void rdot_tail(const VNext& a, const double* partials, int nblocks, int s,
                                          unsigned* counter) {
  __shared__ double tot[GNP_MAX_RESTART + 4];
  __shared__ int s_brk;
  DevState* st = a.st;
  const int K = s + 2;  // h_s[0..s] and ||w_s||^2
  reduce_partials(partials, nblocks, K, tot);
  if (threadIdx.x < 32) {
    double bb = 0.0;
    for (int k = threadIdx.x; k <= s; k += 32) bb = fma(tot[k], tot[k], bb);
    bb = warp_sum(bb);
    if (threadIdx.x == 0) {
      const double omega = tot[s + 1];
      const double rho = sqrt(fmax(omega - bb, 0.0));
      const double wn = sqrt(omega);
      const double rho_n = fmax(rho, RHO_FLOOR * wn);  // the normalisation of v'_{s+1}
      const bool brk = !(rho_n > 0.0) || !isfinite(rho_n) || !isfinite(bb);
      st->rho = rho_n;
      st->rho_est = rho;
      st->rho_inv = brk ? 0.0 : 1.0 / rho_n;
      st->wnorm0 = wn;
      st->jd = s;
      st->j = s + 1;
      s_brk = brk ? 1 : 0;
      *counter = 0;
    }
  }
  double* h2 = const_cast<double*>(a.h2);
  for (int k = threadIdx.x; k <= s; k += blockDim.x) h2[k] = tot[k];
  __syncthreads();
  if (s_brk && st->active) finish_col(a, s, a.h2, st->rho_est, st->wnorm0);
}

// w = A z and the first pass of step s = st->j (short rows: one thread per row).
template <class XT>
__global__ void __launch_bounds__(RED_THREADS)
k_spmv_rdot_row(const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val, ColPtr xp,
                int n, const VNext a, double* __restrict__ partials, unsigned* counter) {
  if (!a.st->active) return;
  __shared__ double sred[RED_SH];
  const int s = a.st->j;
  const int K = s + 2;
  double* w = const_cast<double*>(a.w);
  row_spmv(hw_grid(), rp, col, val, static_cast<const XT*>(colptr_k(xp)), w, n);
  block_dots(a.V, w, n, K, s + 1, sred, partials + (size_t)blockIdx.x * K);
  if (!last_block_arrive(counter)) return;
  rdot_tail(a, partials, gridDim.x, s, counter);
}

// The same with the tile gather (any row lengths): blocks loop over tiles of TILE rows,
// thread t owning row r0 + t, so that the dots see the rows this thread wrote.
template <class XT>
__global__ void __launch_bounds__(TILE)
k_spmv_rdot(const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val, ColPtr xp,
            int n, const VNext a, double* __restrict__ partials, unsigned* counter) {
  static_assert(TILE == RED_THREADS, "tile rows = reduction threads");
  if (!a.st->active) return;
  using TR = TrSpmv<XT>;
  __shared__ TileSmem<TR> sm;
  __shared__ double sred[RED_SH];
  const int s = a.st->j;
  const int K = s + 2;
  double* w = const_cast<double*>(a.w);
  const XT* x = static_cast<const XT*>(colptr_k(xp));
  const int nt = (n + TILE - 1) / TILE;
  for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const int r0 = tile * TILE;
    const int rows = min(TILE, n - r0);
    __syncthreads();
    tile_load_rp<TR>(sm, rp, r0, rows);
    __syncthreads();
    tile_gather<TR>(sm, rows, col, val, x);
    __syncthreads();
    if (threadIdx.x < rows) {
      double s1[1];
      tile_row_sum<TR, 1>(sm, threadIdx.x, 0, s1);
      w[r0 + threadIdx.x] = s1[0];
    }
  }
  block_dots(a.V, w, n, K, s + 1, sred, partials + (size_t)blockIdx.x * K);
  if (!last_block_arrive(counter)) return;
  rdot_tail(a, partials, gridDim.x, s, counter);
}

// Second pass of step s = st->j >= 1 (reorthogonalisation branch): a_s, nu_s, the finished
// column s-1 and its Givens update (last block).
__global__ void __launch_bounds__(RED_THREADS)
k_reorth_dots(int n, const VNext a, double* __restrict__ partials, unsigned* counter) {
  DevState* st = a.st;
  if (!st->active) return;
  __shared__ double sred[RED_SH];
  __shared__ double tot[GNP_MAX_RESTART + 4];
  __shared__ double s_nu;
  const int s = st->j;
  const int K = s + 1;  // a_s[0..s-1] and ||v'_s||^2
  const size_t ld = (size_t)n;
  block_dots(a.V, a.V + (size_t)s * ld, n, K, s, sred, partials + (size_t)blockIdx.x * K);
  if (!last_block_arrive(counter)) return;
  reduce_partials(partials, gridDim.x, K, tot);
  if (threadIdx.x < 32) {
    double aa = 0.0;
    for (int k = threadIdx.x; k < s; k += 32) aa = fma(tot[k], tot[k], aa);
    aa = warp_sum(aa);
    if (threadIdx.x == 0) {
      const double nu = sqrt(fmax(tot[s] - aa, 0.0));
      s_nu = nu;
      st->nu_inv = 1.0 / nu;
      *counter = 0;
    }
  }
  __syncthreads();
  const double rp = st->rho;  // rho_{s-1}, the normalisation of v'_s
  double* hf = const_cast<double*>(a.hf);
  double* ha = const_cast<double*>(a.h1);
  for (int k = threadIdx.x; k < s; k += blockDim.x) {
    ha[k] = tot[k];
    hf[k] = fma(rp, tot[k], a.h2[k]);  // h_{s-1}[k] + rho_{s-1} a_k
  }
  __syncthreads();
  finish_col(a, s - 1, hf, rp * s_nu, st->wnorm0);
}

// v_s = (v'_s - V_{s-1} a_s) / nu_s in place (s = st->j >= 1), after k_reorth_dots.
__global__ void __launch_bounds__(RED_THREADS)
k_reorth_update(int n, const VNext a) {
  const DevState* st = a.st;
  if (!st->active) return;
  __shared__ double sa[GNP_MAX_RESTART + 4];
  __shared__ double s_inv;
  const int s = st->j;
  for (int k = threadIdx.x; k < s; k += blockDim.x) sa[k] = a.h1[k];
  if (threadIdx.x == 0) s_inv = st->nu_inv;
  __syncthreads();
  const double inv = s_inv;
  const size_t ld = (size_t)n;
  double* V = a.V;
  double* vs = V + (size_t)s * ld;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double x = vs[i];
#pragma unroll 8
    for (int k = 0; k < s; ++k) x -= V[k * ld + i] * sa[k];
    vs[i] = x * inv;
  }
}

// End of an overlapped cycle: the last column, [h_{m-1}; rho_{m-1}] (one block).
__global__ void __launch_bounds__(RED_THREADS) k_dfinish(const VNext a) {
  DevState* st = a.st;
  if (!st->active) return;
  finish_col(a, st->jd, a.h2, st->rho_est, st->wnorm0);
}

// r = b - A x -> V[:, 0], beta = ||r||; the last block restarts the cycle state.
__device__ __forceinline__ void residual_body(VGrid gr, const int* __restrict__ rp, const int* __restrict__ col,
                                              const double* __restrict__ val, const double* __restrict__ x,
                                              const double* __restrict__ b, double* __restrict__ V0, int n,
                                              DevState* st, double* __restrict__ g, double* __restrict__ hist,
                                              unsigned long long* __restrict__ thist, double* __restrict__ partials,
                                              unsigned* counter, GCtl* gc = nullptr) {
  using TR = TrSpmv<double>;
  __shared__ TileSmem<TR> sm;
  __shared__ double sh[32];
  const int r0 = gr.bid * TILE;
  const int rows = min(TILE, n - r0);
  tile_load_rp<TR>(sm, rp, r0, rows);
  __syncthreads();
  tile_gather<TR>(sm, rows, col, val, x);
  __syncthreads();
  double acc = 0.0;
  if (threadIdx.x < rows) {
    double s[1];
    tile_row_sum<TR, 1>(sm, threadIdx.x, 0, s);
    double r = b[r0 + threadIdx.x] - s[0];
    V0[r0 + threadIdx.x] = r;
    acc = r * r;
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[gr.bid] = t;
  if (last_block_arrive(counter, gr.nblk)) {
    __shared__ double tot[1];
    reduce_partials(partials, gr.nblk, 1, tot);
    if (threadIdx.x == 0) {
      const double beta = sqrt(tot[0]);
      const double beta_prev = st->beta;  // the residual this cycle began from
      st->beta = beta;
      if (st->iters == 0) {
        hist[0] = beta / st->bnorm;
        thist[0] = global_ns() - st->t0;
      }
      st->last_flags = st->flags;
      st->last_jj = st->jj;
      st->j = 0;
      st->jj = 0;
      st->flags = 0;
      st->vscale = beta;
      st->fresh = 1;
      g[0] = beta;
      st->active = (isfinite(beta) && beta > st->tol && st->iters < st->maxiters) ? 1 : 0;
      if (gc) {  // grouped steps: the stopping rules here, so the next cycle needs no host
        CycleCtl c;
        c.stagn = gc->stagn;
        c.mism = gc->mism;
        c.restarts = gc->restarts;
        c.cycles = ++gc->cycles;
        int status = GNP_OK;
        if (cycle_after(*st, beta_prev, st->maxiters, c, &status)) {
          gc->done = 1;
          gc->status = status;
          st->active = 0;
        }
        gc->stagn = c.stagn;
        gc->mism = c.mism;
        gc->restarts = c.restarts;
      }
      *counter = 0;
    }
  }
}

__global__ void __launch_bounds__(TILE)
k_residual(const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
           const double* __restrict__ x, const double* __restrict__ b, double* __restrict__ V0, int n,
           DevState* st, double* __restrict__ g, double* __restrict__ hist,
           unsigned long long* __restrict__ thist, double* __restrict__ partials, unsigned* counter) {
  residual_body(hw_grid(), rp, col, val, x, b, V0, n, st, g, hist, thist, partials, counter);
}

// ||b|| and tol = rtol ||b||.
__global__ void __launch_bounds__(RED_THREADS)
k_bnorm(const double* __restrict__ b, int n, DevState* st, double* __restrict__ partials, unsigned* counter) {
  __shared__ double sh[32];
  if (blockIdx.x == 0 && threadIdx.x == 0) st->t0 = global_ns();  // the solve's clock starts here
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc += b[i] * b[i];
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
  if (last_block_arrive(counter)) {
    __shared__ double tot[1];
    reduce_partials(partials, gridDim.x, 1, tot);
    if (threadIdx.x == 0) {
      st->bnorm = sqrt(tot[0]);
      st->tol = st->rtol * st->bnorm;
      *counter = 0;
    }
  }
}

// v_j <- v_j / vscale (M = identity, Jacobi, inner GMRES: the normalisation that the GNP
// encoder does in its own first pass).
__global__ void __launch_bounds__(RED_THREADS)
k_vscale(double* __restrict__ V, int n, const DevState* st) {
  if (!st->active) return;
  __shared__ double s_inv;
  if (threadIdx.x == 0) s_inv = 1.0 / st->vscale;  // once per block: float64 division is slow
  __syncthreads();
  double* v = V + (size_t)st->j * n;
  const double inv = s_inv;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = v[i] * inv;
}

// ---------------------------------------------------------------- CGS2 passes

template <int PASS>
__device__ __forceinline__ void cgs_body(VGrid gr, double* __restrict__ V, int n, double* __restrict__ w,
                                         DevState* st, double* __restrict__ h1, double* __restrict__ h2,
                                         double* __restrict__ H, double* __restrict__ R, double* __restrict__ cs,
                                         double* __restrict__ sn, double* __restrict__ g, double* __restrict__ hist,
                                         unsigned long long* __restrict__ thist, double* __restrict__ partials,
                                         unsigned* counter) {
  if (!st->active) return;
  constexpr bool NORM = PASS == 1 || PASS == 4;  // the dots also give ||w||^2 (entry j+1)
  __shared__ double shh[GNP_MAX_RESTART + 2];
  __shared__ double shred[KC][32];  // KC*32 = 256 >= GNP_MAX_RESTART: reused for sines
  __shared__ double sred[PASS == 3 ? 1 : RED_SH];
  __shared__ double shtot[GNP_MAX_RESTART + 4];
  __shared__ double sx[PASS == 4 ? 2 * (GNP_MAX_RESTART + 4) : 1];
  const int j = st->j;
  const size_t ld = (size_t)n;
  const int gtid = gr.bid * blockDim.x + threadIdx.x;
  const int gstride = gr.nblk * blockDim.x;
  if (PASS >= 2) {
    const double* hp = (PASS == 3) ? h2 : h1;
    for (int k = threadIdx.x; k <= j; k += blockDim.x) shh[k] = hp[k];
    __syncthreads();
  }
  if (PASS == 3) {
    // w2 = w1 - V h2 -> V[:, j+1]; ||w2||^2
    double acc = 0.0;
    double* vout = V + (size_t)(j + 1) * ld;
    for (int i = gtid; i < n; i += gstride) {
      double x = w[i];
#pragma unroll 8
      for (int k = 0; k <= j; ++k) x -= V[k * ld + i] * shh[k];
      vout[i] = x;
      acc += x * x;
    }
    double t = block_sum(acc, shred[0]);
    if (threadIdx.x == 0) partials[gr.bid] = t;
  } else {
    if (PASS == 2 || PASS == 4) {
      for (int i = gtid; i < n; i += gstride) {
        double x = w[i];
#pragma unroll 8
        for (int k = 0; k <= j; ++k) x -= V[k * ld + i] * shh[k];
        w[i] = x;
      }
    }
    const int K = NORM ? j + 2 : j + 1;  // passes 1 and 4 also ||w||^2 as entry j+1
    block_dots(gr, V, w, n, K, NORM ? j + 1 : -1, sred, partials + (size_t)gr.bid * K);
  }
  if (!last_block_arrive(counter, gr.nblk)) return;
  const int K = NORM ? j + 2 : (PASS == 2 ? j + 1 : 1);
  reduce_partials(partials, gr.nblk, K, shtot);
  if (PASS == 4) {
    // h2 and ||w1||^2 go out; k_vnext finishes the step (Givens update in its block 0)
    for (int i = threadIdx.x; i <= j; i += blockDim.x) h2[i] = shtot[i];
    if (threadIdx.x == 0) {
      st->w1sq = shtot[j + 1];
      st->jv = j;
      *counter = 0;
    }
    return;
  }
  if (PASS == 3) {
    // stage the Givens inputs with all threads: column j = h1 + h2, the previous
    // rotations (reuse shh for the cosines, shred for the sines)
    double* scs = shh;
    double* ssn = &shred[0][0];
    for (int i = threadIdx.x; i <= j; i += blockDim.x) shtot[1 + i] = h1[i] + h2[i];
    for (int i = threadIdx.x; i < j; i += blockDim.x) {
      scs[i] = cs[i];
      ssn[i] = sn[i];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  *counter = 0;
  if (PASS == 1) {
    for (int k = 0; k <= j; ++k) h1[k] = shtot[k];
    st->wnorm0 = sqrt(shtot[j + 1]);
    return;
  }
  if (PASS == 2) {
    for (int k = 0; k <= j; ++k) h2[k] = shtot[k];
    return;
  }
  // PASS 3: column j of H_bar and the Givens update of the least-squares problem
  const double hn = sqrt(shtot[0]);
  arnoldi_step_finish(st, j, shtot + 1, hn, shh, &shred[0][0], H, R, cs, sn, g, hist, thist);
}

template <int PASS>
__global__ void __launch_bounds__(RED_THREADS)
k_cgs(double* __restrict__ V, int n, double* __restrict__ w, DevState* st, double* __restrict__ h1,
      double* __restrict__ h2, double* __restrict__ H, double* __restrict__ R, double* __restrict__ cs,
      double* __restrict__ sn, double* __restrict__ g, double* __restrict__ hist,
      unsigned long long* __restrict__ thist, double* __restrict__ partials, unsigned* counter) {
  cgs_body<PASS>(hw_grid(), V, n, w, st, h1, h2, H, R, cs, sn, g, hist, thist, partials, counter);
}

// After k_cgs<4>, for step j = st->jv.  Block 0 finishes the step while the others form
// the next basis vector, so the serial Givens update is off the critical path:
//   block 0: column j of H_bar = h1 + h2, h_{j+1,j} = ||w1 - V h2|| =
//     sqrt(||w1||^2 - ||h2||^2) (V has orthonormal columns to working precision and
//     h2 = V^T w1; ||h2|| is O(eps ||w||) after the first pass, so nothing cancels unless
//     w1 itself is at the breakdown level, where the step ends anyway), then
//     arnoldi_step_finish (rotations, g, residual estimate, the continue decision).
//   blocks 1..: V[:, j+1] = w1 - V_j h2 (not yet normalised: the next step's first kernel
//     divides by st->vscale = h_{j+1,j}).  The column is formed even when block 0 ends the
//     cycle (V has m+1 columns; an unused column is harmless); these blocks read only jv,
//     which block 0 does not write.
__global__ void __launch_bounds__(RED_THREADS)
k_vnext(const VNext a, int n) {
  if (blockIdx.x == 0) {
    vnext_finish(a);
    return;
  }
  __shared__ double shh[GNP_MAX_RESTART + 4];
  const DevState* st = a.st;
  if (!st->active) return;
  const int j = st->jv;
  const size_t ld = (size_t)n;
  const double* __restrict__ V = a.V;
  const double* __restrict__ w = a.w;
  for (int k = threadIdx.x; k <= j; k += blockDim.x) shh[k] = a.h2[k];
  __syncthreads();
  double* vout = a.V + (size_t)(j + 1) * ld;
  for (int i = (blockIdx.x - 1) * blockDim.x + threadIdx.x; i < n; i += (gridDim.x - 1) * blockDim.x) {
    double x = w[i];
#pragma unroll 8
    for (int k = 0; k <= j; ++k) x -= V[k * ld + i] * shh[k];
    vout[i] = x;
  }
}

// y = R^{-1} g (back substitution, redundantly in every block), x += Z[:, :jj] y.
// The substitution runs by columns: y_i = g_i / R_ii, then every lane removes y_i's part
// from its own entries of g (g_k -= R_ki y_i, k < i).  Per step the serial chain is one
// multiply and one fused multiply-add (the reciprocals of the diagonal are formed in
// parallel first) instead of a five-level shuffle tree and a division: float64 operations
// that depend on one another cost tens of cycles each on GB300.
// sR: jj x jj doubles of dynamic shared memory (the upper triangle of R, column-major).
template <class ZT>
__device__ __forceinline__ void xupdate_body(VGrid gr, const ZT* __restrict__ Z, double* __restrict__ x, int n,
                                             const DevState* st, const double* __restrict__ R,
                                             const double* __restrict__ g, double* sR) {
  __shared__ double y[GNP_MAX_RESTART];
  __shared__ double sg[GNP_MAX_RESTART];
  __shared__ double rinv[GNP_MAX_RESTART];
  const int jj = st->jj;
  if (jj == 0) return;
  const int ldh = st->m + 1;
  // stage R, g and 1/R_ii with all threads, then one warp back-substitutes
  for (int t = threadIdx.x; t < jj * jj; t += blockDim.x) {
    const int c = t / jj, r = t % jj;
    sR[t] = (r <= c) ? R[(size_t)c * ldh + r] : 0.0;
  }
  for (int t = threadIdx.x; t < jj; t += blockDim.x) {
    sg[t] = g[t];
    rinv[t] = 1.0 / R[(size_t)t * ldh + t];
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int i = jj - 1; i >= 0; --i) {
      const double yi = sg[i] * rinv[i];  // sg[i] is final: its last update was in step i+1
      if (lane == 0) y[i] = yi;
      for (int k = lane; k < i; k += 32) sg[k] -= sR[i * jj + k] * yi;
      __syncwarp();
    }
  }
  __syncthreads();
  const size_t ld = (size_t)n;
  for (int i = gr.bid * blockDim.x + threadIdx.x; i < n; i += gr.nblk * blockDim.x) {
    double acc = x[i];
    for (int k = 0; k < jj; ++k) acc += (double)Z[k * ld + i] * y[k];
    x[i] = acc;
  }
}

template <class ZT>
__global__ void __launch_bounds__(RED_THREADS)
k_xupdate(const ZT* __restrict__ Z, double* __restrict__ x, int n, const DevState* st,
          const double* __restrict__ R, const double* __restrict__ g) {
  extern __shared__ double sR[];
  xupdate_body<ZT>(hw_grid(), Z, x, n, st, R, g, sR);
}

// ---------------------------------------------------------------- grouped steps (serving)
//
// The same bodies for several requests per launch (GTable: each request's stand-alone
// grid; GSlot: its data).  The GNP-preconditioned step of the two-pass CGS2 schedule:
// w = A z with pass 1, pass 2 (the Givens update of the step follows in the next step's
// encoder); the cycle end x += Z y and the restart r = b - A x.
__global__ void __launch_bounds__(RED_THREADS) kg_spmv_dot_row(const __grid_constant__ GTable t, const GSlot* sl) {
  VGrid g;
  const GSlot& d = sl[t.slot[gt_entry(t, g)]];
  const ColPtr z{d.Z, sizeof(float) * (size_t)d.n, reinterpret_cast<const int*>(d.st), 0};
  spmv_dot_row_body<float>(g, d.rp, d.col, d.val, z, d.w, d.V, d.n, d.st, d.h1, d.partials, d.counter);
}

__global__ void __launch_bounds__(RED_THREADS) kg_cgs2(const __grid_constant__ GTable t, const GSlot* sl) {
  VGrid g;
  const GSlot& d = sl[t.slot[gt_entry(t, g)]];
  cgs_body<4>(g, d.V, d.n, d.w, d.st, d.h1, d.h2, d.Hb, d.R, d.cs, d.sn, d.g, d.hist, d.thist, d.partials,
              d.counter);
}

// Every grouped step launches the cycle end for every request; only those at phase m (whose
// encoder finished step m-1 earlier in the same grouped step) and not done run it.  The
// residual's last block applies the stopping rules (cycle_after) and either restarts the cycle or marks the
// request done (active = 0: its later rounds do nothing, x stays as the deciding cycle
// left it).
__global__ void __launch_bounds__(RED_THREADS) kg_xupdate(const __grid_constant__ GTable t, const GSlot* sl) {
  extern __shared__ double sR[];
  VGrid g;
  const GSlot& d = sl[t.slot[gt_entry(t, g)]];
  if (d.gc->phase != d.m || d.gc->done) return;
  xupdate_body<float>(g, d.Z, d.x, d.n, d.st, d.R, d.g, sR);
}

__global__ void __launch_bounds__(TILE) kg_residual(const __grid_constant__ GTable t, const GSlot* sl) {
  VGrid g;
  const GSlot& d = sl[t.slot[gt_entry(t, g)]];
  if (d.gc->phase != d.m || d.gc->done) return;
  residual_body(g, d.rp, d.col, d.val, d.x, d.b, d.V, d.n, d.st, d.g, d.hist, d.thist, d.partials, d.counter,
                d.gc);
}

// ---------------------------------------------------------------- host side

int spmv_launch(const gnp_mat* A, const double* x, const float* xf, double* y, cudaStream_t st) {
  const int nt = (A->n + TILE - 1) / TILE;
  if (xf) {
    ColPtr xp{const_cast<float*>(xf), 0, nullptr, 0};
    k_spmv_tile<float><<<nt, TILE, 0, st>>>(A->rp, A->col, A->val, xp, y, A->n, nullptr);
  } else {
    ColPtr xp{const_cast<double*>(x), 0, nullptr, 0};
    k_spmv_tile<double><<<nt, TILE, 0, st>>>(A->rp, A->col, A->val, xp, y, A->n, nullptr);
  }
  return check_launch("k_spmv_tile");
}

int solver_ensure_zd(Solver* S, int m) {
  if (S->Zd && S->zd_m >= m) return GNP_OK;
  dev_free(S->Zd);
  S->zd_m = 0;
  GNP_TRY(dev_alloc(&S->Zd, (size_t)S->n * m));
  S->zd_m = m;
  return GNP_OK;
}

int grouped_krylov_launch(const std::vector<GHost>& reqs, const GSlot* d_slots, cudaStream_t st) {
  std::vector<std::pair<int, int>> e;
  for (const GHost& q : reqs) e.push_back({q.slot, dot_blocks(q.n)});
  const std::vector<GTable> tabs = gt_build(e, GT_MAX);
  for (const GTable& t : tabs) kg_spmv_dot_row<<<t.start[t.count], RED_THREADS, 0, st>>>(t, d_slots);
  for (const GTable& t : tabs) kg_cgs2<<<t.start[t.count], RED_THREADS, 0, st>>>(t, d_slots);
  return check_launch("grouped FGMRES step");
}

int grouped_cycle_end_launch(const std::vector<GHost>& reqs, int m, const GSlot* d_slots, cudaStream_t st) {
  // (every request of the round: the kernels pick the ones at the end of their cycle)
  std::vector<std::pair<int, int>> ex, er;
  for (const GHost& q : reqs) {
    ex.push_back({q.slot, red_blocks(q.n)});
    er.push_back({q.slot, (q.n + TILE - 1) / TILE});
  }
  const int xsm = (int)sizeof(double) * m * m;
  for (const GTable& t : gt_build(ex, GT_MAX)) kg_xupdate<<<t.start[t.count], RED_THREADS, xsm, st>>>(t, d_slots);
  for (const GTable& t : gt_build(er, GT_MAX)) kg_residual<<<t.start[t.count], TILE, 0, st>>>(t, d_slots);
  return check_launch("grouped FGMRES cycle end");
}

// The reorthogonalisation stream (highest priority, so that its short kernels take SM
// slots as the layers' blocks retire; GNP_SIDE_PRIORITY=low in the environment gives it
// the lowest, for tuning) and the fork/join events, made on first use.
static int solver_side(Solver* S) {
  if (S->side) return GNP_OK;
  int lo = 0, hi = 0;
  GNP_TRY_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  const char* e = getenv("GNP_SIDE_PRIORITY");
  const bool low = e && strcmp(e, "low") == 0;
  GNP_TRY_CUDA(cudaStreamCreateWithPriority(&S->side, cudaStreamNonBlocking, low ? lo : hi));
  GNP_TRY_CUDA(cudaEventCreateWithFlags(&S->fork, cudaEventDisableTiming));
  GNP_TRY_CUDA(cudaEventCreateWithFlags(&S->join, cudaEventDisableTiming));
  return GNP_OK;
}

static VNext vnext_args(Solver* S, int dcgs = 0) {
  return VNext{S->V, S->w, S->h1, S->h2, S->st, S->H, S->R, S->cs, S->sn, S->g, S->hist, S->thist, S->hf, dcgs};
}

// The GNP step's orthogonalisation (ortho_overlapped, solver.h): the overlapped schedule
// takes 78.8 against 88.8 us per step at 65,536 rows.
static bool dcgs_enabled() { return ortho_overlapped(); }

// Row-per-thread SpMV for matrices without long rows (GNP_SPMV_ROWK=0 in the environment
// forces the tile kernel, for tuning).
static bool spmv_short_rows(const gnp_mat* A) {
  static const char* e = getenv("GNP_SPMV_ROWK");
  static const bool on = !(e && e[0] == '0');
  return on && A->max_deg <= SPMV_ROW_DMAX;
}

// w = A x (x float64) with CGS2 pass 1, on the kernel that suits the row lengths.
static void spmv_dot_f64(const gnp_mat* A, ColPtr x, Solver* S, int ndot, int ncg, bool short_rows,
                         cudaStream_t st) {
  if (short_rows)
    k_spmv_dot_row<double><<<ncg, RED_THREADS, 0, st>>>(A->rp, A->col, A->val, x, S->w, S->V, A->n, S->st,
                                                        S->h1, S->red.partials, S->red.counter);
  else
    k_spmv_dot<double><<<ndot, TILE, 0, st>>>(A->rp, A->col, A->val, x, S->w, S->V, A->n, S->st, S->h1,
                                              S->red.partials, S->red.counter);
}

// Enqueue one restart cycle: m Arnoldi steps, x update, residual.
int launch_cycle(gnp_mat* A, Solver* S, const Prec& P, int m, const double* b, double* x,
                 cudaStream_t st, bool prof, const ApplyWs* ws) {
  const int n = A->n;
  const int nt = (n + TILE - 1) / TILE;
  const int nb = red_blocks(n);
  const int ncg = dot_blocks(n);
  const int ndot = std::min(nt, 4 * NUM_SMS_GB300);
  const int* ctl = reinterpret_cast<const int*>(S->st);
  const int* jptr = ctl;
  const bool short_rows = spmv_short_rows(A);
  const bool f64z = P.kind == GNP_PRECOND_JACOBI || P.kind == GNP_PRECOND_GMRES;
  if (f64z) GNP_REQUIRE(S->Zd && S->zd_m >= m, "launch_cycle: float64 directions not allocated");
  if (P.kind == GNP_PRECOND_GNP && dcgs_enabled()) {
    // overlapped CGS2 (see the kernels above): the second pass of v'_j runs on S->side
    // beside the layers of step j
    GNP_TRY(solver_side(S));
    gnp_model* M = P.M;
    const VNext vd = vnext_args(S, 1);
    for (int j = 0; j < m; ++j) {
      ColPtr v{S->V, sizeof(double) * (size_t)n, jptr, 0};
      ColPtr z{S->Z, sizeof(float) * (size_t)n, jptr, 0};
      cudaEvent_t* ev = prof ? S->events.data() + (size_t)2 * j * M->cfg.L : nullptr;
      GNP_TRY(apply_launch(M, v, &S->st->vscale, z, nullptr, ctl, st, ev, ws, j > 0 ? &vd : nullptr,
                           j > 0 ? S->fork : nullptr, S->side));
      if (j > 0) {
        k_reorth_dots<<<ncg, RED_THREADS, 0, S->side>>>(n, vd, S->red.partials, S->red.counter);
        k_reorth_update<<<nb, RED_THREADS, 0, S->side>>>(n, vd);
        GNP_TRY_CUDA(cudaEventRecord(S->join, S->side));
        GNP_TRY_CUDA(cudaStreamWaitEvent(st, S->join, 0));
      }
      if (short_rows)
        k_spmv_rdot_row<float><<<ncg, RED_THREADS, 0, st>>>(A->rp, A->col, A->val, z, n, vd, S->red.partials,
                                                            S->red.counter);
      else
        k_spmv_rdot<float><<<ndot, TILE, 0, st>>>(A->rp, A->col, A->val, z, n, vd, S->red.partials, S->red.counter);
    }
    k_dfinish<<<1, RED_THREADS, 0, st>>>(vd);
    k_xupdate<float><<<nb, RED_THREADS, (int)sizeof(double) * m * m, st>>>(S->Z, x, n, S->st, S->R, S->g);
    k_residual<<<nt, TILE, 0, st>>>(A->rp, A->col, A->val, x, b, S->V, n, S->st, S->g, S->hist, S->thist,
                                    S->red.partials, S->red.counter);
    return check_launch("fgmres cycle (overlapped CGS2)");
  }
  for (int j = 0; j < m; ++j) {
    ColPtr v{S->V, sizeof(double) * (size_t)n, jptr, 0};
    if (P.kind == GNP_PRECOND_GNP) {
      gnp_model* M = P.M;
      ColPtr z{S->Z, sizeof(float) * (size_t)n, jptr, 0};
      cudaEvent_t* ev = prof ? S->events.data() + (size_t)2 * j * M->cfg.L : nullptr;
      // from step 1 on the encoder forms v_j itself (and a block of it finishes step j-1)
      const VNext vn = vnext_args(S);
      GNP_TRY(apply_launch(M, v, &S->st->vscale, z, nullptr, ctl, st, ev, ws, j > 0 ? &vn : nullptr));
      if (short_rows)
        k_spmv_dot_row<float><<<ncg, RED_THREADS, 0, st>>>(A->rp, A->col, A->val, z, S->w, S->V, n, S->st,
                                                           S->h1, S->red.partials, S->red.counter);
      else
        k_spmv_dot<float><<<ndot, TILE, 0, st>>>(A->rp, A->col, A->val, z, S->w, S->V, n, S->st, S->h1,
                                                 S->red.partials, S->red.counter);
    } else if (f64z) {
      ColPtr z{S->Zd, sizeof(double) * (size_t)n, jptr, 0};
      if (P.kind == GNP_PRECOND_JACOBI)
        GNP_TRY(jacobi_launch(P.dinv, v, S->st, z, n, st));
      else
        GNP_TRY(inner_gmres_launch(A, P.inner, v, S->st, z, st));
      spmv_dot_f64(A, z, S, ndot, ncg, short_rows, st);
    } else {
      k_vscale<<<nb, RED_THREADS, 0, st>>>(S->V, n, S->st);
      spmv_dot_f64(A, v, S, ndot, ncg, short_rows, st);
    }
    k_cgs<4><<<ncg, RED_THREADS, 0, st>>>(S->V, n, S->w, S->st, S->h1, S->h2, S->H, S->R, S->cs, S->sn,
                                         S->g, S->hist, S->thist, S->red.partials, S->red.counter);
    if (P.kind != GNP_PRECOND_GNP)
      k_vnext<<<1 + nb, RED_THREADS, 0, st>>>(vnext_args(S), n);
    else if (j == m - 1)
      k_vnext<<<1, RED_THREADS, 0, st>>>(vnext_args(S), n);  // the last step's finish only
  }
  const int xsm = (int)sizeof(double) * m * m;
  if (P.kind == GNP_PRECOND_GNP)
    k_xupdate<float><<<nb, RED_THREADS, xsm, st>>>(S->Z, x, n, S->st, S->R, S->g);
  else
    k_xupdate<double><<<nb, RED_THREADS, xsm, st>>>(f64z ? S->Zd : S->V, x, n, S->st, S->R, S->g);
  k_residual<<<nt, TILE, 0, st>>>(A->rp, A->col, A->val, x, b, S->V, n, S->st, S->g, S->hist,
                                  S->thist, S->red.partials, S->red.counter);
  return check_launch("fgmres cycle");
}

// ---------------------------------------------------------------- inner GMRES

// Start of one inner solve: b = v (divided by outer->vscale and written back when an
// outer FGMRES step owns v), x = 0, and the inner state reset.  When the outer step is
// inactive the inner solve gets maxiters = 0, so all its kernels fall through.
__global__ void __launch_bounds__(RED_THREADS)
k_inner_begin(ColPtr vp, DevState* outer, double* __restrict__ b, double* __restrict__ x, int n,
              DevState* st, int iters, double rtol) {
  const bool act = outer == nullptr || outer->active;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->j = 0;
    st->active = 0;
    st->iters = 0;
    st->maxiters = act ? iters : 0;
    st->m = iters;
    st->jj = 0;
    st->flags = 0;
    st->rtol = rtol;
    st->timeout_ns = 0ull;
  }
  if (!act) return;
  double* v = static_cast<double*>(colptr_k(vp));
  const double s = outer ? outer->vscale : 1.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double t = v[i];
    if (outer) {
      t = t / s;
      v[i] = t;
    }
    b[i] = t;
    x[i] = 0.0;
  }
}

// z = x at the end of the inner solve (skipped when the outer step is inactive).
__global__ void __launch_bounds__(RED_THREADS)
k_inner_end(const double* __restrict__ x, const DevState* outer, ColPtr zp, int n) {
  if (outer && !outer->active) return;
  double* z = static_cast<double*>(colptr_k(zp));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) z[i] = x[i];
}

int inner_gmres_create(int n, int iters, double rtol, InnerGmres** out) {
  *out = nullptr;
  InnerGmres* G = new InnerGmres();
  G->iters = iters;
  G->rtol = rtol;
  int e = solver_create(n, iters, iters, &G->S);
  if (e == GNP_OK) e = dev_alloc(&G->b, (size_t)n);
  if (e == GNP_OK) e = dev_alloc(&G->x, (size_t)n);
  if (e != GNP_OK) {
    inner_gmres_free(G);
    return e;
  }
  *out = G;
  return GNP_OK;
}

void inner_gmres_free(InnerGmres* G) {
  if (!G) return;
  solver_free(G->S);
  dev_free(G->b);
  dev_free(G->x);
  delete G;
}

int inner_gmres_launch(gnp_mat* A, InnerGmres* G, ColPtr v, DevState* outer, ColPtr z, cudaStream_t st) {
  Solver* S = G->S;
  const int n = A->n;
  const int k = G->iters;
  const int nt = (n + TILE - 1) / TILE;
  const int nb = red_blocks(n);
  const int ncg = dot_blocks(n);
  const int ndot = std::min(nt, 4 * NUM_SMS_GB300);
  const int* jptr = reinterpret_cast<const int*>(S->st);
  k_inner_begin<<<nb, RED_THREADS, 0, st>>>(v, outer, G->b, G->x, n, S->st, k, G->rtol);
  k_bnorm<<<nb, RED_THREADS, 0, st>>>(G->b, n, S->st, S->red.partials, S->red.counter);
  k_residual<<<nt, TILE, 0, st>>>(A->rp, A->col, A->val, G->x, G->b, S->V, n, S->st, S->g, S->hist,
                                  S->thist, S->red.partials, S->red.counter);
  for (int j = 0; j < k; ++j) {
    k_vscale<<<nb, RED_THREADS, 0, st>>>(S->V, n, S->st);
    ColPtr vj{S->V, sizeof(double) * (size_t)n, jptr, 0};
    spmv_dot_f64(A, vj, S, ndot, ncg, spmv_short_rows(A), st);
    k_cgs<4><<<ncg, RED_THREADS, 0, st>>>(S->V, n, S->w, S->st, S->h1, S->h2, S->H, S->R, S->cs, S->sn,
                                         S->g, S->hist, S->thist, S->red.partials, S->red.counter);
    k_vnext<<<1 + nb, RED_THREADS, 0, st>>>(vnext_args(S), n);
  }
  k_xupdate<double><<<nb, RED_THREADS, (int)sizeof(double) * k * k, st>>>(S->V, G->x, n, S->st, S->R, S->g);
  k_inner_end<<<nb, RED_THREADS, 0, st>>>(G->x, outer, z, n);
  return check_launch("inner gmres");
}

static int read_state(Solver* S, cudaStream_t st) {
  GNP_TRY_CUDA(cudaMemcpyAsync(S->st_host, S->st, sizeof(DevState), cudaMemcpyDeviceToHost, st));
  GNP_TRY_CUDA(cudaStreamSynchronize(st));
  return GNP_OK;
}

// The unpreconditioned m-step Arnoldi process (Eq. 4) from v1 (not necessarily
// normalised), CGS2 as in the solver: V_out receives the k+1 basis vectors (k <= m, k
// < m only at a breakdown), Hbar_host the (m+1) x m column-major H_bar (first k
// columns valid).  Runs on `st` and synchronises it.
int arnoldi_basis(gnp_mat* A, const double* v1, int m, double* V_out, double* Hbar_host, int* k_out,
                  cudaStream_t st) {
  GNP_TRY(solver_ensure(A, m, m));
  Solver* S = A->solver;
  if (st == nullptr || st == cudaStreamLegacy) {
    GNP_TRY_CUDA(cudaStreamSynchronize(st));
    st = S->own;
  }
  const int n = A->n;
  const int nt = (n + TILE - 1) / TILE;
  const int nb = red_blocks(n);
  const int ncg = dot_blocks(n);
  DevState init{};
  init.maxiters = m;
  init.m = m;
  init.rtol = 0.0;
  memcpy(S->st_host, &init, sizeof(DevState));
  GNP_TRY_CUDA(cudaMemcpyAsync(S->st, S->st_host, sizeof(DevState), cudaMemcpyHostToDevice, st));
  GNP_TRY_CUDA(cudaMemsetAsync(S->w, 0, sizeof(double) * n, st));  // x0 = 0
  // entries of H_bar below the subdiagonal are never written: clear stale values
  GNP_TRY_CUDA(cudaMemsetAsync(S->H, 0, sizeof(double) * (size_t)(m + 1) * m, st));
  k_bnorm<<<nb, RED_THREADS, 0, st>>>(v1, n, S->st, S->red.partials, S->red.counter);
  k_residual<<<nt, TILE, 0, st>>>(A->rp, A->col, A->val, S->w, v1, S->V, n, S->st, S->g, S->hist,
                                  S->thist, S->red.partials, S->red.counter);
  const int* jptr = reinterpret_cast<const int*>(S->st);
  for (int j = 0; j < m; ++j) {
    k_vscale<<<nb, RED_THREADS, 0, st>>>(S->V, n, S->st);
    ColPtr v{S->V, sizeof(double) * (size_t)n, jptr, 0};
    k_spmv_tile<double><<<nt, TILE, 0, st>>>(A->rp, A->col, A->val, v, S->w, n, jptr);
    k_cgs<1><<<ncg, RED_THREADS, 0, st>>>(S->V, n, S->w, S->st, S->h1, S->h2, S->H, S->R, S->cs, S->sn,
                                         S->g, S->hist, S->thist, S->red.partials, S->red.counter);
    k_cgs<2><<<ncg, RED_THREADS, 0, st>>>(S->V, n, S->w, S->st, S->h1, S->h2, S->H, S->R, S->cs, S->sn,
                                         S->g, S->hist, S->thist, S->red.partials, S->red.counter);
    k_cgs<3><<<ncg, RED_THREADS, 0, st>>>(S->V, n, S->w, S->st, S->h1, S->h2, S->H, S->R, S->cs, S->sn,
                                         S->g, S->hist, S->thist, S->red.partials, S->red.counter);
  }
  GNP_TRY(check_launch("arnoldi"));
  GNP_TRY(read_state(S, st));
  const DevState hs = *S->st_host;
  if (hs.flags & FL_NAN) {
    set_error("arnoldi: NaN in the basis");
    return GNP_ERR_NAN;
  }
  int k = hs.jj;
  // a breakdown keeps column j (jj = j + 1); the basis has k + 1 vectors unless the
  // last one was never formed
  GNP_TRY_CUDA(cudaMemcpyAsync(V_out, S->V, sizeof(double) * (size_t)n * (k + 1), cudaMemcpyDeviceToDevice, st));
  GNP_TRY_CUDA(cudaMemcpyAsync(Hbar_host, S->H, sizeof(double) * (size_t)(m + 1) * m, cudaMemcpyDeviceToHost, st));
  GNP_TRY_CUDA(cudaStreamSynchronize(st));
  *k_out = k;
  return GNP_OK;
}

int solve_init_launch(const gnp_mat* A, Solver* S, const double* b, double* x, double rtol, int maxiters,
                      int m, double timeout_s, cudaStream_t st) {
  const int n = A->n;
  const int nt = (n + TILE - 1) / TILE;
  const int nb = red_blocks(n);
  DevState init{};
  init.maxiters = maxiters;
  init.m = m;
  init.rtol = rtol;
  init.timeout_ns = timeout_s > 0.0 ? (unsigned long long)std::max(1.0, timeout_s * 1e9) : 0ull;
  memcpy(S->st_host, &init, sizeof(DevState));
  GNP_TRY_CUDA(cudaMemcpyAsync(S->st, S->st_host, sizeof(DevState), cudaMemcpyHostToDevice, st));
  // entries of H_bar below the subdiagonal are never written: clear stale values
  GNP_TRY_CUDA(cudaMemsetAsync(S->H, 0, sizeof(double) * (size_t)(m + 1) * m, st));
  k_bnorm<<<nb, RED_THREADS, 0, st>>>(b, n, S->st, S->red.partials, S->red.counter);
  k_residual<<<nt, TILE, 0, st>>>(A->rp, A->col, A->val, x, b, S->V, n, S->st, S->g, S->hist,
                                  S->thist, S->red.partials, S->red.counter);
  return check_launch("solve init");
}

static bool graphs_enabled() {
  const char* e = getenv("GNP_NO_GRAPH");
  return !(e && e[0] == '1');
}

}  // namespace gnp

using namespace gnp;

extern "C" int gnp_profile_gconv(int on) {
  gnp::g_profile_gconv = on != 0;
  return GNP_OK;
}

namespace gnp {

static int solve_impl(gnp_mat* A, const double* b, double* x, const Prec& P, int restart, double rtol,
                      int maxiters, double timeout_s, gnp_solve_info* info, void* stream) {
  gnp_model* M = P.kind == GNP_PRECOND_GNP ? P.M : nullptr;
  GNP_REQUIRE(A && b && x, "fgmres_solve: null argument");
  GNP_REQUIRE(timeout_s >= 0.0 && timeout_s < 1e9, "fgmres_solve: timeout %g out of [0, 1e9) s", timeout_s);
  GNP_REQUIRE(restart >= 1 && restart <= GNP_MAX_RESTART, "fgmres_solve: restart %d out of [1, %d]",
              restart, GNP_MAX_RESTART);
  GNP_REQUIRE(maxiters >= 0, "fgmres_solve: maxiters < 0");
  GNP_REQUIRE(rtol >= 0.0, "fgmres_solve: rtol < 0");
  GNP_REQUIRE(!M || M->A == A, "fgmres_solve: the preconditioner was built for another matrix");
  GNP_REQUIRE(P.kind != GNP_PRECOND_GNP || M, "fgmres_solve: GNP preconditioner without a model");
  cudaStream_t st = as_stream(stream);
  const auto t0 = std::chrono::steady_clock::now();
  GNP_TRY(solver_ensure(A, restart, maxiters));
  Solver* S = A->solver;
  if (P.kind == GNP_PRECOND_JACOBI || P.kind == GNP_PRECOND_GMRES) GNP_TRY(solver_ensure_zd(S, restart));
  if (st == nullptr || st == cudaStreamLegacy) {
    // graphs cannot be captured on the legacy default stream: order the caller's
    // earlier work, then run the (synchronous) solve on the solver's own stream
    GNP_TRY_CUDA(cudaStreamSynchronize(st));
    st = S->own;
  }
  if (M) GNP_TRY(apply_prepare(M));
  const int n = A->n;
  const int nt = (n + TILE - 1) / TILE;
  const int nb = red_blocks(n);
  GNP_TRY(solve_init_launch(A, S, b, x, rtol, maxiters, restart, timeout_s, st));
  GNP_TRY(check_launch("fgmres init"));
  GNP_TRY(read_state(S, st));
  int status = GNP_OK;
  CycleCtl ctl_c;
  const bool prof = g_profile_gconv && M != nullptr && M->cfg.L > 0;
  double gconv_ms = 0.0;
  long long gconv_launches = 0;
  DevState hs = *S->st_host;
  if (hs.bnorm == 0.0) {
    GNP_TRY_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, st));
    hs.beta = 0.0;
  } else if (!std::isfinite(hs.beta) || !std::isfinite(hs.bnorm)) {
    status = GNP_ERR_NAN;
  } else if (hs.beta > hs.tol) {
    if (maxiters == 0) status = GNP_ERR_NOT_CONVERGED;
    const bool use_graph = graphs_enabled();
    if (prof) GNP_TRY(ensure_events(S, restart, M->cfg.L));
    while (status == GNP_OK && hs.iters < maxiters) {
      const double beta_prev = hs.beta;
      if (use_graph) {
        const unsigned long long ver = M ? model_version(M) : 0ull;
        if (!S->gexec || S->g_model != P.key || S->g_kind != P.kind || S->g_version != ver || S->g_m != restart ||
            S->g_hprec != (M ? M->hprec : -1) || S->g_b != b || S->g_x != x || S->g_stream != st ||
            S->g_prof != prof || S->g_dcgs != dcgs_enabled()) {
          if (S->gexec) cudaGraphExecDestroy(S->gexec);
          S->gexec = nullptr;
          cudaGraph_t graph;
          GNP_TRY_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
          int ls = launch_cycle(A, S, P, restart, b, x, st, prof, nullptr);
          cudaError_t ce = cudaStreamEndCapture(st, &graph);
          if (ls != GNP_OK) return ls;
          if (ce != cudaSuccess) {
            set_error("fgmres: graph capture failed: %s", cudaGetErrorString(ce));
            return GNP_ERR_CUDA;
          }
          ce = cudaGraphInstantiate(&S->gexec, graph, 0);
          cudaGraphDestroy(graph);
          if (ce != cudaSuccess) {
            set_error("fgmres: graph instantiate failed: %s", cudaGetErrorString(ce));
            S->gexec = nullptr;
            return GNP_ERR_CUDA;
          }
          S->g_model = P.key;
          S->g_kind = P.kind;
          S->g_version = ver;
          S->g_m = restart;
          S->g_hprec = M ? M->hprec : -1;
          S->g_b = b;
          S->g_x = x;
          S->g_stream = st;
          S->g_prof = prof;
          S->g_dcgs = dcgs_enabled();
        }
        GNP_TRY_CUDA(cudaGraphLaunch(S->gexec, st));
      } else {
        GNP_TRY(launch_cycle(A, S, P, restart, b, x, st, prof, nullptr));
      }
      const int iters_before = hs.iters;
      ++ctl_c.cycles;
      GNP_TRY(read_state(S, st));
      hs = *S->st_host;
      if (prof) {
        const int steps = hs.iters - iters_before;  // Arnoldi steps this cycle ran
        for (int j = 0; j < steps; ++j)
          for (int l = 0; l < M->cfg.L; ++l) {
            float ms = 0.f;
            const size_t e = ((size_t)j * M->cfg.L + l) * 2;
            GNP_TRY_CUDA(cudaEventElapsedTime(&ms, S->events[e], S->events[e + 1]));
            gconv_ms += ms;
            ++gconv_launches;
          }
      }
      if (cycle_after(hs, beta_prev, maxiters, ctl_c, &status)) break;
    }
  }
  GNP_TRY_CUDA(cudaStreamSynchronize(st));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) {
    info->iters = hs.iters;
    info->restarts = ctl_c.restarts;
    info->status = status;
    info->seconds = secs;
    info->gconv_ms = gconv_ms;
    info->gconv_launches = (int)gconv_launches;
    info->cycles = ctl_c.cycles;
    const double bn = hs.bnorm > 0.0 ? hs.bnorm : 1.0;
    info->rel_res_true = hs.bnorm > 0.0 ? hs.beta / bn : 0.0;
    info->rel_res_est = hs.iters > 0 ? hs.res_est / bn : info->rel_res_true;
    if (info->res_history) {
      const int cnt = hs.bnorm > 0.0 ? hs.iters + 1 : 1;
      if (hs.bnorm > 0.0) {
        GNP_TRY_CUDA(cudaMemcpy(info->res_history, S->hist, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
      } else {
        info->res_history[0] = 0.0;
      }
      info->res_history_len = cnt;
    }
    if (info->time_history) {
      const int cnt = hs.bnorm > 0.0 ? hs.iters + 1 : 1;
      if (hs.bnorm > 0.0) {
        std::vector<unsigned long long> ns(cnt);
        GNP_TRY_CUDA(cudaMemcpy(ns.data(), S->thist, sizeof(unsigned long long) * cnt, cudaMemcpyDeviceToHost));
        for (int i = 0; i < cnt; ++i) info->time_history[i] = 1e-9 * (double)ns[i];
      } else {
        info->time_history[0] = 0.0;
      }
    }
    if (info->hessenberg) {
      const int cols = hs.iters > 0 ? hs.last_jj : 0;
      GNP_TRY_CUDA(cudaMemcpy(info->hessenberg, S->H, sizeof(double) * (size_t)(restart + 1) * restart,
                              cudaMemcpyDeviceToHost));
      info->hessenberg_cols = cols;
    }
  }
  return status;
}

}  // namespace gnp

static Prec model_prec(gnp_model* M) {
  Prec P;
  P.kind = M ? GNP_PRECOND_GNP : GNP_PRECOND_IDENTITY;
  P.M = M;
  P.key = M;
  return P;
}

extern "C" int fgmres_solve_timeout(gnp_mat* A, const double* b, double* x, gnp_model* M, int restart,
                                    double rtol, int maxiters, double timeout_s, gnp_solve_info* info,
                                    void* stream) {
  return solve_impl(A, b, x, model_prec(M), restart, rtol, maxiters, timeout_s, info, stream);
}

extern "C" int fgmres_solve(gnp_mat* A, const double* b, double* x, gnp_model* M, int restart,
                            double rtol, int maxiters, gnp_solve_info* info, void* stream) {
  return solve_impl(A, b, x, model_prec(M), restart, rtol, maxiters, 0.0, info, stream);
}

extern "C" int fgmres_solve_precond(gnp_mat* A, const double* b, double* x, gnp_precond* P, int restart,
                                    double rtol, int maxiters, double timeout_s, gnp_solve_info* info,
                                    void* stream) {
  if (!P) return solve_impl(A, b, x, model_prec(nullptr), restart, rtol, maxiters, timeout_s, info, stream);
  GNP_REQUIRE(precond_matrix(P) == A, "fgmres_solve_precond: the preconditioner was built for another matrix");
  return solve_impl(A, b, x, precond_view(P), restart, rtol, maxiters, timeout_s, info, stream);
}
