// Flexible GMRES for several right-hand sides at once: k systems A x_r = b_r with one
// matrix and one preconditioner M (Sec. 4: one trained GNP serves any number of
// right-hand sides), advanced in lockstep so that every sparse gather is shared.
//
// Layout: every n-vector of the k systems is stored node-major, element (i, r) at
// i*K + r (K = k rounded up to 2, 4 or 8; the padding systems have b = 0 and are done from
// the start).  Krylov column c of V (float64) and Z (float32) is the n x K block at c*n*K.
// The GNP hidden block is [n][K][16]: one gather of neighbour i moves K*64 bytes.
//
// One Arnoldi step j for all systems (each kernel reads j and an any-active flag from
// device memory, so one captured CUDA graph replays a whole restart cycle):
//   k_mencode, (L-1) x k_mgconv, k_mgconv_dec   z_r = M(v_r) for every active system
//   (M = I: k_mvscale only normalises v_r)
//   k_mspmv       w_r = A z_r (one tile gather for all systems) and CGS2 pass 1
//                 (h1 = V^T w_r, ||w_r||^2)
//   k_mcgs<2>     pass 2 (w1 = w - V h1, h2 = V^T w1, ||w1||^2); its last block forms
//                 h_{j+1,j} = sqrt(||w1||^2 - ||h2||^2) (reading c29) and runs the Givens
//                 update of every active system (one thread per system) and the cycle
//                 decision
//   k_mcgs<3>     column j+1 = w1 - V h2 (no reduction)
// Cycle end: k_mxupdate (y_r = R_r^{-1} g_r, x_r += Z y_r) and k_mresidual (r = b - A x,
// beta_r, restart).  A system whose cycle ended early waits, inactive, for the others;
// its iterates and counts are those of a solve on its own.
#include <chrono>
#include <cmath>
#include <cstring>

#include "gconv_common.cuh"
#include "solver.h"

namespace gnp {

constexpr int MROWS = 128;  // rows per tile of the float64 gathers

struct MultiSolver {
  int n = 0, K = 0, m_cap = 0, maxit_cap = 0, L = -1;
  double* V = nullptr;   // [(m+1) n K]
  float* Z = nullptr;    // [m n K]
  double* w = nullptr;   // [n K]
  double* b = nullptr;   // [n K] right-hand sides (padded)
  double* x = nullptr;   // [n K] iterates
  float* Hg[2] = {nullptr, nullptr};  // GNP hidden blocks [n K 16]
  DevState* st = nullptr;       // [K]
  DevState* st_host = nullptr;  // pinned [K]
  int* ctl = nullptr;           // {j, any system active, j of the column k_mcgs<K, 3> forms}
  double* one = nullptr;        // device 1.0: tau of the unit-norm basis vectors
  int* done = nullptr;          // [K] device flags: system finished
  int* done_host = nullptr;     // pinned [K]
  double* H = nullptr;   // [K][(m+1) m]
  double* R = nullptr;   // [K][(m+1) m]
  double* cs = nullptr;  // [K][m]
  double* sn = nullptr;  // [K][m]
  double* g = nullptr;   // [K][m+1]
  double* h1 = nullptr;  // [(m+2) K]
  double* h2 = nullptr;  // [(m+2) K]
  double* hist = nullptr;              // [K][maxiters+1]
  unsigned long long* thist = nullptr;  // [K][maxiters+1]
  RedScratch red;
  cudaGraphExec_t gexec = nullptr;
  const void* g_model = nullptr;
  unsigned long long g_version = 0;
  int g_m = 0;
  cudaStream_t g_stream = nullptr;
  bool g_ortho = false;
  cudaStream_t own = nullptr;
  // overlapped CGS2: the reorthogonalisation stream and its fork/join events
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

// Per-system strides of the small arrays (sized by the caps).
struct MStrides {
  int hs, ms, gs, hist;
};

__host__ __device__ inline MStrides mstrides(int m_cap, int maxit_cap) {
  return MStrides{(m_cap + 1) * m_cap, m_cap, m_cap + 1, maxit_cap + 1};
}

// ---------------------------------------------------------------- traits

// float64 CSR gather of K values per node (x float64 or float32): G lanes per slot,
// NV values per lane.
template <int K, class XT>
struct TrSpmvM {
  static constexpr int G = K >= 4 ? 2 : 1, NV = K / G, STRIDE = K;
  using acc = double;
  using val_t = double;
  using x_t = XT;
  __device__ __forceinline__ static void load(const XT* X, int c, int q, double (&h)[NV]) {
    const XT* p = X + (size_t)c * K + q * NV;
    if constexpr (sizeof(XT) == 8 && NV % 2 == 0) {
#pragma unroll
      for (int u = 0; u < NV / 2; ++u) {
        const double2 t = __ldg(reinterpret_cast<const double2*>(p) + u);
        h[2 * u] = t.x;
        h[2 * u + 1] = t.y;
      }
    } else if constexpr (sizeof(XT) == 4 && NV == 4) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(p));
      h[0] = t.x; h[1] = t.y; h[2] = t.z; h[3] = t.w;
    } else if constexpr (sizeof(XT) == 4 && NV == 2) {
      const float2 t = __ldg(reinterpret_cast<const float2*>(p));
      h[0] = t.x; h[1] = t.y;
    } else {
#pragma unroll
      for (int u = 0; u < NV; ++u) h[u] = (double)__ldg(p + u);
    }
  }
};

// float32 hidden block of K systems: 4K lanes x float4 per node (K*64 bytes).
template <int K>
struct TrHidM {
  static constexpr int G = 4 * K, NV = 4, STRIDE = 16 * K + 4;
  using acc = float;
  using val_t = float;
  using x_t = float;
  __device__ __forceinline__ static void load(const float* X, int c, int q, float (&h)[4]) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(X + (size_t)c * 16 * K) + q);
    h[0] = t.x; h[1] = t.y; h[2] = t.z; h[3] = t.w;
  }
};

__device__ __forceinline__ int mstep(const int* ctl) { return ctl[0]; }

// ---------------------------------------------------------------- norms, scaling

// ||b_r|| and tol_r = rtol ||b_r||; the clock of the solve starts here.
template <int K>
__global__ void __launch_bounds__(RED_THREADS)
k_mbnorm(const double* __restrict__ b, int n, DevState* st, double* __restrict__ partials, unsigned* counter) {
  __shared__ double sred[RED_SH];
  __shared__ double tot[K];
  if (blockIdx.x == 0 && threadIdx.x < K) st[threadIdx.x].t0 = global_ns();
  double a[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) a[k] = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int r = 0; r < K; ++r) {
      const double v = b[(size_t)i * K + r];
      a[r] += v * v;
    }
  }
  block_reduce_kc<false>(a, sred, partials + (size_t)blockIdx.x * K, K);
  if (!last_block_arrive(counter)) return;
  reduce_partials(partials, gridDim.x, K, tot);
  if (threadIdx.x < K) {
    DevState* s = st + threadIdx.x;
    s->bnorm = sqrt(tot[threadIdx.x]);
    s->tol = s->rtol * s->bnorm;
  }
  if (threadIdx.x == 0) *counter = 0;
}

// v_r <- v_r / vscale_r for the active systems (M = identity).
template <int K>
__global__ void __launch_bounds__(RED_THREADS)
k_mvscale(double* __restrict__ V, int n, const DevState* st, const int* ctl) {
  if (!ctl[1]) return;
  double* v = V + (size_t)mstep(ctl) * n * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * K;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % K);
    if (st[r].active) v[e] = v[e] / st[r].vscale;
  }
}

// ---------------------------------------------------------------- GNP for K systems

// v_r <- v_r / vscale_r (unit norm, so tau = 1), u = sqrt(n) v_r, then the encoder
// (1 -> 32 -> 16) into H0 [n][K][16].  One thread per (node, system).
template <int K>
__global__ void __launch_bounds__(RED_THREADS)
k_mencode(double* __restrict__ V, int n, const DevState* st, const int* ctl, double sqrt_n,
          float* __restrict__ H0, const __grid_constant__ EncW ew) {
  if (!ctl[1]) return;
  double* v = V + (size_t)mstep(ctl) * n * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * K;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % K);
    if (!st[r].active) continue;
    const double x = v[e] / st[r].vscale;
    v[e] = x;
    const float u = (float)(x * sqrt_n);
    float h[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) h[c] = ew.b2[c];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const float a = fmaxf(fmaf(u, ew.W1[k], ew.b1[k]), 0.0f);
#pragma unroll
      for (int c = 0; c < 16; ++c) h[c] = fmaf(a, ew.W2[k * 16 + c], h[c]);
    }
    float4* o = reinterpret_cast<float4*>(H0 + e * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = make_float4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
  }
}

// The encoder of overlapped-CGS2 step s >= 1 (s = ctl[0]; V_{s-1} final, h_{s-1} in h):
// v'_s = (w - V_{s-1} h_{s-1}) / rho_{s-1} per active system into column s, encoded as
// k_mencode encodes (unit norm, tau = 1).  One thread per (node, system).
template <int K>
__global__ void __launch_bounds__(RED_THREADS)
k_mencode_d(double* __restrict__ V, const double* __restrict__ w, int n, const DevState* st, const int* ctl,
            const double* __restrict__ h, double sqrt_n, float* __restrict__ H0, const __grid_constant__ EncW ew) {
  if (!ctl[1]) return;
  __shared__ double sh[(GNP_MAX_RESTART_MULTI + 2) * K];
  __shared__ double rinv[K];
  __shared__ int act[K];
  const int s = mstep(ctl);
  for (int k = threadIdx.x; k < s * K; k += blockDim.x) sh[k] = h[k];
  if (threadIdx.x < K) {
    rinv[threadIdx.x] = st[threadIdx.x].rho_inv;
    act[threadIdx.x] = st[threadIdx.x].active;
  }
  __syncthreads();
  double* vout = V + (size_t)s * n * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * K;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % K);
    if (!act[r]) continue;
    const long long i = e / K;
    double y = w[e];
    for (int c = 0; c < s; ++c) y -= V[((size_t)c * n + i) * K + r] * sh[c * K + r];
    y = y * rinv[r];
    vout[e] = y;
    const float u = (float)(y * sqrt_n);
    float hh[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) hh[c] = ew.b2[c];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const float a = fmaxf(fmaf(u, ew.W1[k], ew.b1[k]), 0.0f);
#pragma unroll
      for (int c = 0; c < 16; ++c) hh[c] = fmaf(a, ew.W2[k * 16 + c], hh[c]);
    }
    float4* o = reinterpret_cast<float4*>(H0 + e * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = make_float4(hh[4 * q], hh[4 * q + 1], hh[4 * q + 2], hh[4 * q + 3]);
  }
}

template <int K>
struct MGconvSmem {
  static constexpr int ROWS = TILE / K;  // one epilogue thread per (node, system)
  TileSmem<TrHidM<K>, ROWS> g;
  __align__(16) float stile[TILE * 20];  // the tile's own hidden rows, 16 floats + pad each
};

// Coalesced copy of `pairs` 16-float hidden rows between global memory and the tile.
template <bool TO_GLOBAL>
__device__ __forceinline__ void mtile_copy(float* stile, float* gbase, int pairs) {
  float4* gb = reinterpret_cast<float4*>(gbase);
  for (int i = threadIdx.x; i < pairs * 4; i += blockDim.x) {
    float4* s = reinterpret_cast<float4*>(stile + (i >> 2) * 20) + (i & 3);
    if (TO_GLOBAL) gb[i] = *s;
    else *s = __ldg(gb + i);
  }
}

// One Res-GCONV layer (Eq. 7, or the residual variant) for K systems; LAST also applies
// the decoder and tau/sqrt(n) = 1/sqrt(n) and writes z into column j of Z.
template <int K, int FORM, bool LAST>
__global__ void __launch_bounds__(TILE, 3)
k_mgconv(const int* __restrict__ rp, const int* __restrict__ col, const float* __restrict__ valhat,
         const float* __restrict__ Hin, float* __restrict__ Hout, float* __restrict__ Zbase, int n,
         const int* __restrict__ ctl, double inv_sqrt_n, const __grid_constant__ LayerW lw,
         const __grid_constant__ DecW dw) {
  using TR = TrHidM<K>;
  constexpr int ROWS = MGconvSmem<K>::ROWS;
  if (!ctl[1]) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  MGconvSmem<K>& sm = *reinterpret_cast<MGconvSmem<K>*>(smraw);
  const int r0 = blockIdx.x * ROWS;
  const int rows = min(ROWS, n - r0);
  tile_load_rp<TR>(sm.g, rp, r0, rows);
  mtile_copy<false>(sm.stile, const_cast<float*>(Hin) + (size_t)r0 * K * 16, rows * K);
  __syncthreads();
  tile_gather<TR, TileSmem<TrHidM<K>, ROWS>, 8>(sm.g, rows, col, valhat, Hin);  // 8 rows in flight per lane
  __syncthreads();
  const int t = threadIdx.x;  // pair (row t / K, system t % K)
  const int row = t / K, sys = t % K;
  float o[16];
  if (row < rows) {
    float h[16], agg[16];
    const float4* hs = reinterpret_cast<const float4*>(sm.stile + t * 20);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 v = hs[q];
      h[4 * q] = v.x; h[4 * q + 1] = v.y; h[4 * q + 2] = v.z; h[4 * q + 3] = v.w;
    }
    tile_row_sum<TR, 16>(sm.g, row, 16 * sys, agg);
    // two outputs per paired multiply-add (each lane an fmaf, inputs in order)
#pragma unroll
    for (int k = 0; k < 16; ++k) o[k] = 0.0f;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
#pragma unroll
      for (int k = 0; k < 16; k += 2) ffma2(o[k], o[k + 1], agg[c], agg[c], lw.W[c * 16 + k], lw.W[c * 16 + k + 1]);
    }
    if (FORM == GNP_LAYER_PAPER) {
#pragma unroll
      for (int c = 0; c < 16; ++c) {
#pragma unroll
        for (int k = 0; k < 16; k += 2) ffma2(o[k], o[k + 1], h[c], h[c], lw.U[c * 16 + k], lw.U[c * 16 + k + 1]);
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) o[k] = fmaxf(o[k], 0.0f);
    } else {
#pragma unroll
      for (int k = 0; k < 16; ++k) o[k] = h[k] + fmaxf(o[k], 0.0f);
    }
  }
  if constexpr (LAST) {
    if (row < rows) {
      float z = dw.b2;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        float a = dw.b1[k];
#pragma unroll
        for (int c = 0; c < 16; ++c) a = fmaf(o[c], dw.W1[c * 32 + k], a);
        z = fmaf(fmaxf(a, 0.0f), dw.W2[k], z);
      }
      float* zc = Zbase + (size_t)mstep(ctl) * n * K;
      zc[(size_t)r0 * K + t] = z * (float)inv_sqrt_n;
    }
  } else {
    // pair t's input was read by this thread only: overwrite in place
    if (row < rows) {
      float4* d = reinterpret_cast<float4*>(sm.stile + t * 20);
#pragma unroll
      for (int q = 0; q < 4; ++q) d[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    }
    __syncthreads();
    mtile_copy<true>(sm.stile, Hout + (size_t)r0 * K * 16, rows * K);
  }
}

// ---------------------------------------------------------------- SpMV, residual

// w = A z for the K systems; z is column j of Z (float32) or of V (float64).  With DOTS
// the kernel is also CGS2 pass 1: h1 = V_j^T w and ||w||^2 per system, each block adding
// its own rows' products (KC per register chunk, a fixed-order block reduction) and the
// last block the blocks' partials in order.
// RDOT (the overlapped schedule; j = s, V_s final): the last block keeps h_s = V_s^T w in h1
// and per active system rho_s by Pythagoras, normalised as in the one-system step
// (RHO_FLOOR), 1/rho, ||w||; a system whose step broke down (w = 0 or not finite) has
// its column s finished at once with the first-pass values, which ends its cycle.  It
// then advances the step (ctl[0] = s + 1) and the any-active flag.
template <int K>
__device__ __forceinline__ void mrdot_tail(int s, const double* shtot, DevState* st, int* ctl, double* h,
                                           double* H, double* R, double* cs, double* sn, double* g, double* hist,
                                           unsigned long long* thist, MStrides ms) {
  __shared__ double scol[K][GNP_MAX_RESTART_MULTI + 2];
  __shared__ int anyact;
  for (int k = threadIdx.x; k < (s + 1) * K; k += blockDim.x) h[k] = shtot[k];
  if (threadIdx.x == 0) anyact = 0;
  __syncthreads();
  if (threadIdx.x < K) {
    const int r = threadIdx.x;
    DevState* sr = st + r;
    if (sr->active) {
      double bb = 0.0;
      for (int c = 0; c <= s; ++c) bb = fma(shtot[c * K + r], shtot[c * K + r], bb);
      const double omega = shtot[(s + 1) * K + r];
      const double rho = sqrt(fmax(omega - bb, 0.0));
      const double wn = sqrt(omega);
      const double rho_n = fmax(rho, RHO_FLOOR * wn);
      const bool brk = !(rho_n > 0.0) || !isfinite(rho_n) || !isfinite(bb);
      sr->rho = rho_n;
      sr->rho_est = rho;
      sr->rho_inv = brk ? 0.0 : 1.0 / rho_n;
      sr->wnorm0 = wn;
      sr->jd = s;
      if (brk) {
        for (int c = 0; c <= s; ++c) scol[r][c] = shtot[c * K + r];
        double* csr = cs + (size_t)r * ms.ms;
        double* snr = sn + (size_t)r * ms.ms;
        arnoldi_step_finish(sr, s, scol[r], rho, csr, snr, H + (size_t)r * ms.hs, R + (size_t)r * ms.hs, csr, snr,
                            g + (size_t)r * ms.gs, hist + (size_t)r * ms.hist, thist + (size_t)r * ms.hist, true,
                            wn);
      }
      if (sr->active) atomicOr(&anyact, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl[0] = s + 1;
    ctl[1] = anyact;
  }
}

template <int K, class XT, bool DOTS, bool RDOT = false>
__global__ void __launch_bounds__(TILE)
k_mspmv(const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
        const XT* __restrict__ Xbase, double* __restrict__ w, int n, int* __restrict__ ctl,
        const double* __restrict__ V, DevState* st, double* __restrict__ h1, double* __restrict__ partials,
        unsigned* counter, double* __restrict__ H = nullptr, double* __restrict__ R = nullptr,
        double* __restrict__ cs = nullptr, double* __restrict__ sn = nullptr, double* __restrict__ g = nullptr,
        double* __restrict__ hist = nullptr, unsigned long long* __restrict__ thist = nullptr,
        MStrides ms = MStrides{0, 0, 0, 0}) {
  static_assert(!RDOT || DOTS, "the first-pass tail needs the dots");
  using TR = TrSpmvM<K, XT>;
  if (!ctl[1]) return;
  __shared__ TileSmem<TR, MROWS> sm;
  const int j = mstep(ctl);
  const XT* x = Xbase + (size_t)j * n * K;
  const int r0 = blockIdx.x * MROWS;
  const int rows = min(MROWS, n - r0);
  tile_load_rp<TR>(sm, rp, r0, rows);
  __syncthreads();
  tile_gather<TR>(sm, rows, col, val, x);
  __syncthreads();
  const int t = threadIdx.x;
  double s[K];
#pragma unroll
  for (int r = 0; r < K; ++r) s[r] = 0.0;
  if (t < rows) {
    tile_row_sum<TR, K>(sm, t, 0, s);
    double2* wo = reinterpret_cast<double2*>(w + (size_t)(r0 + t) * K);
#pragma unroll
    for (int u = 0; u < K / 2; ++u) wo[u] = make_double2(s[2 * u], s[2 * u + 1]);
  }
  if constexpr (DOTS) {
    constexpr int CC = KC / K;  // columns per reduction
    __shared__ double sred[RED_SH];
    __shared__ double shtot[(GNP_MAX_RESTART_MULTI + 2) * K];
    const int Kc = j + 2;  // V_j^T w and, as column j+1, ||w||^2
    for (int c0 = 0; c0 < Kc; c0 += CC) {
      double a[KC];
#pragma unroll
      for (int k = 0; k < KC; ++k) a[k] = 0.0;
      if (t < rows) {
        const size_t i = (size_t)(r0 + t);
#pragma unroll
        for (int cl = 0; cl < CC; ++cl) {
          const int c = c0 + cl;
          if (c == j + 1) {
#pragma unroll
            for (int r = 0; r < K; ++r) a[cl * K + r] = s[r] * s[r];
          } else if (c <= j) {
            const double2* vp = reinterpret_cast<const double2*>(V + ((size_t)c * n + i) * K);
#pragma unroll
            for (int u = 0; u < K / 2; ++u) {
              const double2 vv = vp[u];
              a[cl * K + 2 * u] = vv.x * s[2 * u];
              a[cl * K + 2 * u + 1] = vv.y * s[2 * u + 1];
            }
          }
        }
      }
      block_reduce_kc<false>(a, sred, partials + (size_t)blockIdx.x * Kc * K + c0 * K, min(KC, (Kc - c0) * K));
    }
    if (!last_block_arrive(counter)) return;
    reduce_partials(partials, gridDim.x, Kc * K, shtot);
    if (threadIdx.x == 0) *counter = 0;
    if constexpr (RDOT) {
      mrdot_tail<K>(j, shtot, st, ctl, h1, H, R, cs, sn, g, hist, thist, ms);
      return;
    }
    for (int k = threadIdx.x; k < (j + 1) * K; k += blockDim.x) h1[k] = shtot[k];
    if (threadIdx.x < K && st[threadIdx.x].active) st[threadIdx.x].wnorm0 = sqrt(shtot[(j + 1) * K + threadIdx.x]);
  }
}

// r = b - A x -> column 0 of V, beta_r = ||r_r||; the last block restarts every system's
// cycle (a finished system stays inactive).
template <int K>
__global__ void __launch_bounds__(TILE)
k_mresidual(const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
            const double* __restrict__ x, const double* __restrict__ b, double* __restrict__ V0, int n,
            DevState* st, int* ctl, const int* __restrict__ done, double* __restrict__ g,
            double* __restrict__ hist, unsigned long long* __restrict__ thist, MStrides ms,
            double* __restrict__ partials, unsigned* counter) {
  using TR = TrSpmvM<K, double>;
  __shared__ TileSmem<TR, MROWS> sm;
  __shared__ double sred[RED_SH];
  __shared__ double tot[K];
  __shared__ int anyact;
  const int r0 = blockIdx.x * MROWS;
  const int rows = min(MROWS, n - r0);
  tile_load_rp<TR>(sm, rp, r0, rows);
  __syncthreads();
  tile_gather<TR>(sm, rows, col, val, x);
  __syncthreads();
  double a[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) a[k] = 0.0;
  const int t = threadIdx.x;
  if (t < rows) {
    double s[K];
    tile_row_sum<TR, K>(sm, t, 0, s);
    const size_t base = (size_t)(r0 + t) * K;
#pragma unroll
    for (int r = 0; r < K; ++r) {
      const double res = b[base + r] - s[r];
      V0[base + r] = res;
      a[r] = res * res;
    }
  }
  block_reduce_kc<false>(a, sred, partials + (size_t)blockIdx.x * K, K);
  if (!last_block_arrive(counter)) return;
  reduce_partials(partials, gridDim.x, K, tot);
  if (t == 0) anyact = 0;
  __syncthreads();
  if (t < K) {
    DevState* s = st + t;
    const double beta = sqrt(tot[t]);
    s->beta = beta;
    if (s->iters == 0) {
      hist[(size_t)t * ms.hist] = beta / s->bnorm;
      thist[(size_t)t * ms.hist] = global_ns() - s->t0;
    }
    s->last_flags = s->flags;
    s->last_jj = s->jj;
    s->j = 0;
    s->jj = 0;
    s->flags = 0;
    s->vscale = beta;
    g[(size_t)t * ms.gs] = beta;
    s->active = (!done[t] && isfinite(beta) && beta > s->tol && s->iters < s->maxiters) ? 1 : 0;
    if (s->active) atomicOr(&anyact, 1);
  }
  __syncthreads();
  if (t == 0) {
    ctl[0] = 0;
    ctl[1] = anyact;
    *counter = 0;
  }
}

// ---------------------------------------------------------------- CGS2 for K systems

// Dot products of the rows this thread visits: for columns c0..c0+CC-1 of V (column
// j+1 stands for w itself, giving ||w_r||^2), a[cl*K + r] += V[c][i][r] y[i][r].
template <int K, int CC>
__device__ __forceinline__ void mdots(const double* __restrict__ V, const double* __restrict__ y, int n, int j,
                                      int c0, int Kc, double (&a)[KC]) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double yv[K];
#pragma unroll
    for (int u = 0; u < K / 2; ++u) {
      const double2 t = reinterpret_cast<const double2*>(y + (size_t)i * K)[u];
      yv[2 * u] = t.x;
      yv[2 * u + 1] = t.y;
    }
#pragma unroll
    for (int cl = 0; cl < CC; ++cl) {
      const int c = c0 + cl;
      if (c < Kc) {
        if (c == j + 1) {
#pragma unroll
          for (int r = 0; r < K; ++r) a[cl * K + r] += yv[r] * yv[r];
        } else {
          const double2* vp = reinterpret_cast<const double2*>(V + ((size_t)c * n + i) * K);
#pragma unroll
          for (int u = 0; u < K / 2; ++u) {
            const double2 t = vp[u];
            a[cl * K + 2 * u] += t.x * yv[2 * u];
            a[cl * K + 2 * u + 1] += t.y * yv[2 * u + 1];
          }
        }
      }
    }
  }
}

// k_mspmv for matrices whose rows are short (at most ROW_DMAX_M nonzeros): one thread per
// row forms its K sums with eight nonzeros' loads in flight (four at K = 8; no tile),
// then the pass-1 dots run over the same grid-stride rows (mdots re-reads only the w this
// thread wrote).
constexpr int ROW_DMAX_M = 16;

template <int K, class XT>
__device__ __forceinline__ void mload_k(const XT* __restrict__ x, int c, double (&h)[K]) {
  const XT* p = x + (size_t)c * K;
  if constexpr (sizeof(XT) == 8) {
#pragma unroll
    for (int u = 0; u < K / 2; ++u) {
      const double2 t = __ldg(reinterpret_cast<const double2*>(p) + u);
      h[2 * u] = t.x;
      h[2 * u + 1] = t.y;
    }
  } else if constexpr (K == 2) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    h[0] = t.x;
    h[1] = t.y;
  } else {
#pragma unroll
    for (int u = 0; u < K / 4; ++u) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(p) + u);
      h[4 * u] = t.x; h[4 * u + 1] = t.y; h[4 * u + 2] = t.z; h[4 * u + 3] = t.w;
    }
  }
}

template <int K, class XT, bool RDOT = false>
__global__ void __launch_bounds__(RED_THREADS)
k_mspmv_row(const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
            const XT* __restrict__ Xbase, double* __restrict__ w, int n, int* __restrict__ ctl,
            const double* __restrict__ V, DevState* st, double* __restrict__ h1, double* __restrict__ partials,
            unsigned* counter, double* __restrict__ H = nullptr, double* __restrict__ R = nullptr,
            double* __restrict__ cs = nullptr, double* __restrict__ sn = nullptr, double* __restrict__ g = nullptr,
            double* __restrict__ hist = nullptr, unsigned long long* __restrict__ thist = nullptr,
            MStrides ms = MStrides{0, 0, 0, 0}) {
  if (!ctl[1]) return;
  constexpr int CC = KC / K;
  constexpr int NF = K >= 8 ? 4 : 8;  // nonzeros in flight (registers: NF x K doubles)
  __shared__ double sred[RED_SH];
  __shared__ double shtot[(GNP_MAX_RESTART_MULTI + 2) * K];
  const int j = mstep(ctl);
  const XT* x = Xbase + (size_t)j * n * K;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gstride = gridDim.x * blockDim.x;
  for (int i = gtid; i < n; i += gstride) {
    const int rs = __ldg(rp + i), re = __ldg(rp + i + 1);
    double s[K];
#pragma unroll
    for (int r = 0; r < K; ++r) s[r] = 0.0;
    for (int e0 = rs; e0 < re; e0 += NF) {  // NF nonzeros' loads in flight, added in order
      int c[NF];
      double v[NF];
#pragma unroll
      for (int u = 0; u < NF; ++u) {
        const bool ok = e0 + u < re;
        c[u] = ok ? __ldg(col + e0 + u) : 0;
        v[u] = ok ? __ldg(val + e0 + u) : 0.0;
      }
      double xv[NF][K];
#pragma unroll
      for (int u = 0; u < NF; ++u)
        if (e0 + u < re) mload_k<K, XT>(x, c[u], xv[u]);
#pragma unroll
      for (int u = 0; u < NF; ++u)
        if (e0 + u < re) {
#pragma unroll
          for (int r = 0; r < K; ++r) s[r] = fma(v[u], xv[u][r], s[r]);
        }
    }
    double2* wo = reinterpret_cast<double2*>(w + (size_t)i * K);
#pragma unroll
    for (int u = 0; u < K / 2; ++u) wo[u] = make_double2(s[2 * u], s[2 * u + 1]);
  }
  const int Kc = j + 2;  // V_j^T w and, as column j+1, ||w||^2
  for (int c0 = 0; c0 < Kc; c0 += CC) {
    double a[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) a[k] = 0.0;
    mdots<K, CC>(V, w, n, j, c0, Kc, a);
    block_reduce_kc<false>(a, sred, partials + (size_t)blockIdx.x * Kc * K + c0 * K, min(KC, (Kc - c0) * K));
  }
  if (!last_block_arrive(counter)) return;
  reduce_partials(partials, gridDim.x, Kc * K, shtot);
  if (threadIdx.x == 0) *counter = 0;
  if constexpr (RDOT) {
    mrdot_tail<K>(j, shtot, st, ctl, h1, H, R, cs, sn, g, hist, thist, ms);
    return;
  }
  for (int k = threadIdx.x; k < (j + 1) * K; k += blockDim.x) h1[k] = shtot[k];
  if (threadIdx.x < K && st[threadIdx.x].active) st[threadIdx.x].wnorm0 = sqrt(shtot[(j + 1) * K + threadIdx.x]);
}

// The reorthogonalisation branch of overlapped step s = ctl[0] >= 1, beside the layers:
// a_s = V_{s-1}^T v'_s and ||v'_s||^2 per system (mdots with column s standing for v'_s
// itself); the last block forms nu_s, keeps a_s in ha, and for every active system
// finishes column s-1 of H_bar, [h_{s-1} + rho_{s-1} a_s; rho_{s-1} nu_s] (lagged:
// arnoldi_step_finish leaves the step counter to the first pass), then the any-active flag.
template <int K>
__global__ void __launch_bounds__(RED_THREADS)
k_mreorth_dots(const double* __restrict__ V, int n, DevState* st, int* ctl, double* __restrict__ ha,
               const double* __restrict__ h, double* __restrict__ H, double* __restrict__ R,
               double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g,
               double* __restrict__ hist, unsigned long long* __restrict__ thist, MStrides ms,
               double* __restrict__ partials, unsigned* counter) {
  if (!ctl[1]) return;
  constexpr int CC = KC / K;
  __shared__ double sred[RED_SH];
  __shared__ double shtot[(GNP_MAX_RESTART_MULTI + 2) * K];
  __shared__ double scol[K][GNP_MAX_RESTART_MULTI + 2];
  __shared__ int anyact;
  const int s = mstep(ctl);
  const double* y = V + (size_t)s * n * K;
  const int Kc = s + 1;  // a_s and, as column s, ||v'_s||^2
  for (int c0 = 0; c0 < Kc; c0 += CC) {
    double a[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) a[k] = 0.0;
    mdots<K, CC>(V, y, n, s - 1, c0, Kc, a);
    block_reduce_kc<false>(a, sred, partials + (size_t)blockIdx.x * Kc * K + c0 * K, min(KC, (Kc - c0) * K));
  }
  if (!last_block_arrive(counter)) return;
  reduce_partials(partials, gridDim.x, Kc * K, shtot);
  for (int k = threadIdx.x; k < s * K; k += blockDim.x) ha[k] = shtot[k];
  if (threadIdx.x == 0) anyact = 0;
  __syncthreads();
  if (threadIdx.x < K) {
    const int r = threadIdx.x;
    DevState* sr = st + r;
    if (sr->active) {
      double aa = 0.0;
      for (int c = 0; c < s; ++c) aa = fma(shtot[c * K + r], shtot[c * K + r], aa);
      const double nu = sqrt(fmax(shtot[s * K + r] - aa, 0.0));
      sr->nu_inv = 1.0 / nu;
      const double rp = sr->rho;  // rho_{s-1}, the normalisation of v'_s
      for (int c = 0; c < s; ++c) scol[r][c] = fma(rp, shtot[c * K + r], h[c * K + r]);
      double* csr = cs + (size_t)r * ms.ms;
      double* snr = sn + (size_t)r * ms.ms;
      arnoldi_step_finish(sr, s - 1, scol[r], rp * nu, csr, snr, H + (size_t)r * ms.hs, R + (size_t)r * ms.hs, csr,
                          snr, g + (size_t)r * ms.gs, hist + (size_t)r * ms.hist, thist + (size_t)r * ms.hist, true,
                          sr->wnorm0);
      if (sr->active) atomicOr(&anyact, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl[1] = anyact;
    *counter = 0;
  }
}

// v_s = (v'_s - V_{s-1} a_s) / nu_s in place for the active systems (after k_mreorth_dots).
template <int K>
__global__ void __launch_bounds__(RED_THREADS)
k_mreorth_update(double* __restrict__ V, int n, const DevState* st, const int* ctl, const double* __restrict__ ha) {
  if (!ctl[1]) return;
  __shared__ double sa[(GNP_MAX_RESTART_MULTI + 2) * K];
  __shared__ double ninv[K];
  __shared__ int act[K];
  const int s = mstep(ctl);
  for (int k = threadIdx.x; k < s * K; k += blockDim.x) sa[k] = ha[k];
  if (threadIdx.x < K) {
    ninv[threadIdx.x] = st[threadIdx.x].nu_inv;
    act[threadIdx.x] = st[threadIdx.x].active;
  }
  __syncthreads();
  double* vs = V + (size_t)s * n * K;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * K;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % K);
    if (!act[r]) continue;
    const long long i = e / K;
    double x = vs[e];
    for (int c = 0; c < s; ++c) x -= V[((size_t)c * n + i) * K + r] * sa[c * K + r];
    vs[e] = x * ninv[r];
  }
}

// End of an overlapped cycle: the last column of every active system, [h_{m-1}; rho_{m-1}].
template <int K>
__global__ void k_mdfinish(DevState* st, const int* ctl, const double* __restrict__ h, double* __restrict__ H,
                           double* __restrict__ R, double* __restrict__ cs, double* __restrict__ sn,
                           double* __restrict__ g, double* __restrict__ hist, unsigned long long* __restrict__ thist,
                           MStrides ms) {
  __shared__ double scol[K][GNP_MAX_RESTART_MULTI + 2];
  if (!ctl[1] || threadIdx.x >= K) return;
  const int r = threadIdx.x;
  DevState* sr = st + r;
  if (!sr->active) return;
  const int s = sr->jd;
  for (int c = 0; c <= s; ++c) scol[r][c] = h[c * K + r];
  double* csr = cs + (size_t)r * ms.ms;
  double* snr = sn + (size_t)r * ms.ms;
  arnoldi_step_finish(sr, s, scol[r], sr->rho_est, csr, snr, H + (size_t)r * ms.hs, R + (size_t)r * ms.hs, csr, snr,
                      g + (size_t)r * ms.gs, hist + (size_t)r * ms.hist, thist + (size_t)r * ms.hist, true,
                      sr->wnorm0);
}

// (Pass 1, h1 = V_j^T w and ||w||^2, runs inside k_mspmv.)
// PASS 2: w1 = w - V_j h1 (in place), h2 = V_j^T w1
// and ||w1||^2; its last block finishes the step of every active system
// (arnoldi_step_finish, one thread per system) with column j = h1 + h2 and
// h_{j+1,j} = sqrt(||w1||^2 - ||h2||^2) (reading c29, as in the one-system solver: V has
// orthonormal columns and h2 = V^T w1, so this equals ||w1 - V h2|| to rounding), and
// advances the step.  PASS 3: column j+1 = w1 - V_j h2 (normalised by the next step's
// first kernel, which divides by the system's vscale = h_{j+1,j}); no reduction.
template <int K, int PASS>
__global__ void __launch_bounds__(RED_THREADS)
k_mcgs(double* __restrict__ V, int n, double* __restrict__ w, DevState* st, int* ctl, double* __restrict__ h1,
       double* __restrict__ h2, double* __restrict__ H, double* __restrict__ R, double* __restrict__ cs,
       double* __restrict__ sn, double* __restrict__ g, double* __restrict__ hist,
       unsigned long long* __restrict__ thist, MStrides ms, double* __restrict__ partials, unsigned* counter) {
  static_assert(PASS == 2 || PASS == 3, "pass 1 is fused into k_mspmv");
  constexpr int CC = KC / K;  // columns per reduction
  if (!ctl[1]) return;
  __shared__ double sred[RED_SH];
  __shared__ double shh[(GNP_MAX_RESTART_MULTI + 2) * K];
  __shared__ double shtot[(GNP_MAX_RESTART_MULTI + 2) * K];
  __shared__ int anyact;
  const int j = (PASS == 3) ? ctl[2] : mstep(ctl);  // pass 2 has advanced ctl[0] already
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gstride = gridDim.x * blockDim.x;
  if (PASS >= 2) {
    const double* hp = (PASS == 2) ? h1 : h2;
    for (int k = threadIdx.x; k < (j + 1) * K; k += blockDim.x) shh[k] = hp[k];
    __syncthreads();
    // w <- w - V_j h (PASS 2 in place; PASS 3 into column j+1)
    double* out = (PASS == 2) ? w : V + (size_t)(j + 1) * n * K;
    for (int i = gtid; i < n; i += gstride) {
      double xv[K];
#pragma unroll
      for (int r = 0; r < K; ++r) xv[r] = w[(size_t)i * K + r];
      for (int c = 0; c <= j; ++c) {
        const double* vp = V + ((size_t)c * n + i) * K;
#pragma unroll
        for (int r = 0; r < K; ++r) xv[r] -= vp[r] * shh[c * K + r];
      }
#pragma unroll
      for (int r = 0; r < K; ++r) out[(size_t)i * K + r] = xv[r];
    }
  }
  if (PASS == 3) return;  // the new column is formed; pass 2 finished the step
  // dot products over j+2 "columns": V_j^T y and, as column j+1, ||y_r||^2
  const double* y = w;
  const int Kc = j + 2;
  for (int c0 = 0; c0 < Kc; c0 += CC) {
    double a[KC];
#pragma unroll
    for (int k = 0; k < KC; ++k) a[k] = 0.0;
    mdots<K, CC>(V, y, n, j, c0, Kc, a);
    block_reduce_kc<false>(a, sred, partials + (size_t)blockIdx.x * Kc * K + c0 * K, min(KC, (Kc - c0) * K));
  }
  if (!last_block_arrive(counter)) return;
  reduce_partials(partials, gridDim.x, Kc * K, shtot);
  // PASS 2: h2 for pass 3; stage column j of every system (h1 + h2) in shared memory
  // (reuse shh) and finish the step
  for (int k = threadIdx.x; k < (j + 1) * K; k += blockDim.x) h2[k] = shtot[k];
  __syncthreads();
  for (int k = threadIdx.x; k < (j + 1) * K; k += blockDim.x) {
    const int c = k / K, r = k % K;
    shh[r * (GNP_MAX_RESTART_MULTI + 2) + c] = h1[k] + shtot[k];
  }
  if (threadIdx.x == 0) anyact = 0;
  __syncthreads();
  if (threadIdx.x < K) {
    const int r = threadIdx.x;
    DevState* s = st + r;
    if (s->active) {
      double h2sq = 0.0;
      for (int c = 0; c <= j; ++c) h2sq += shtot[c * K + r] * shtot[c * K + r];
      const double hn = sqrt(fmax(shtot[(j + 1) * K + r] - h2sq, 0.0));
      double* csr = cs + (size_t)r * ms.ms;
      double* snr = sn + (size_t)r * ms.ms;
      arnoldi_step_finish(s, j, shh + r * (GNP_MAX_RESTART_MULTI + 2), hn, csr, snr,
                          H + (size_t)r * ms.hs, R + (size_t)r * ms.hs, csr, snr, g + (size_t)r * ms.gs,
                          hist + (size_t)r * ms.hist, thist + (size_t)r * ms.hist);
      if (s->active) atomicOr(&anyact, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl[2] = j;
    ctl[0] = j + 1;
    ctl[1] = anyact;
    *counter = 0;
  }
}

// y_r = R_r^{-1} g_r (one warp per system, redundantly in every block), then
// x_r += Z[:, :jj_r] y_r with Z float32 (GNP) or float64 (V, M = identity).
template <int K, class ZT>
__global__ void __launch_bounds__(RED_THREADS)
k_mxupdate(const ZT* __restrict__ Z, double* __restrict__ x, int n, const DevState* st,
           const double* __restrict__ R, const double* __restrict__ g, MStrides ms, int m) {
  __shared__ double y[K][GNP_MAX_RESTART_MULTI];
  __shared__ int jjs[K];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int ldh = m + 1;
  if (threadIdx.x < K) jjs[threadIdx.x] = st[threadIdx.x].jj;
  __syncthreads();
  for (int r = w; r < K; r += blockDim.x >> 5) {
    const int jj = jjs[r];
    const double* Rr = R + (size_t)r * ms.hs;
    const double* gr = g + (size_t)r * ms.gs;
    for (int i = jj - 1; i >= 0; --i) {
      double part = 0.0;
      for (int k = i + 1 + lane; k < jj; k += 32) part += Rr[(size_t)k * ldh + i] * y[r][k];
      part = warp_sum(part);
      if (lane == 0) y[r][i] = (gr[i] - part) / Rr[(size_t)i * ldh + i];
      __syncwarp();
    }
  }
  __syncthreads();
  int jmax = 0;
#pragma unroll
  for (int r = 0; r < K; ++r) jmax = max(jmax, jjs[r]);
  if (jmax == 0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int r = 0; r < K; ++r) {
      const int jj = jjs[r];
      if (jj == 0) continue;
      double acc = x[(size_t)i * K + r];
      for (int c = 0; c < jj; ++c) acc += (double)Z[((size_t)c * n + i) * K + r] * y[r][c];
      x[(size_t)i * K + r] = acc;
    }
  }
}

// Standalone multi-vector apply: per-system vscale = ||v_r|| (tau_r), active = tau_r > 0.
template <int K>
__global__ void k_mapply_setup(DevState* st, int* ctl, const double* __restrict__ tau) {
  if (threadIdx.x < K) {
    DevState* s = st + threadIdx.x;
    s->vscale = tau[threadIdx.x];
    s->active = tau[threadIdx.x] > 0.0 ? 1 : 0;
  }
  if (threadIdx.x == 0) {
    ctl[0] = 0;
    ctl[1] = 1;
  }
}

// z[i][r] (caller layout [n][k]) = tau_r * zn[i][r]: M(v) = tau M(v / tau) (Eq. 8).
template <int K>
__global__ void k_mapply_out(const float* __restrict__ zn, const double* __restrict__ tau, int k, int n,
                             float* __restrict__ z) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * k;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / k;
    const int r = (int)(e % k);
    z[e] = tau[r] > 0.0 ? (float)((double)zn[i * K + r] * tau[r]) : 0.0f;
  }
}

template <int K>
__global__ void k_mtau(const DevState* st, double* __restrict__ tau) {
  if (threadIdx.x < K) tau[threadIdx.x] = st[threadIdx.x].bnorm;
}

// Gather / scatter between the caller's [n][k] layout and the padded [n][K] one.
template <int K>
__global__ void k_mpack(const double* __restrict__ src, int k, int n, double* __restrict__ dst) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * K;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / K;
    const int r = (int)(e % K);
    dst[e] = r < k ? src[i * k + r] : 0.0;
  }
}

template <int K>
__global__ void k_munpack(const double* __restrict__ src, int k, int n, double* __restrict__ dst) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * k;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / k;
    const int r = (int)(e % k);
    dst[e] = src[i * K + r];
  }
}

// x_r = 0 for one system (zero right-hand side).
template <int K>
__global__ void k_mzero(double* __restrict__ x, int n, int r) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[(size_t)i * K + r] = 0.0;
}

// ---------------------------------------------------------------- host side

void multi_solver_free(MultiSolver* s) {
  if (!s) return;
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  if (s->own) cudaStreamDestroy(s->own);
  if (s->side) cudaStreamDestroy(s->side);
  if (s->fork) cudaEventDestroy(s->fork);
  if (s->join) cudaEventDestroy(s->join);
  dev_free(s->V);
  dev_free(s->Z);
  dev_free(s->w);
  dev_free(s->b);
  dev_free(s->x);
  dev_free(s->Hg[0]);
  dev_free(s->Hg[1]);
  dev_free(s->st);
  if (s->st_host) cudaFreeHost(s->st_host);
  dev_free(s->ctl);
  dev_free(s->one);
  dev_free(s->done);
  if (s->done_host) cudaFreeHost(s->done_host);
  dev_free(s->H);
  dev_free(s->R);
  dev_free(s->cs);
  dev_free(s->sn);
  dev_free(s->g);
  dev_free(s->h1);
  dev_free(s->h2);
  dev_free(s->hist);
  dev_free(s->thist);
  red_free(s->red);
  delete s;
}

static int multi_create(int n, int K, int m, int maxiters, MultiSolver** out) {
  *out = nullptr;
  MultiSolver* s = new MultiSolver();
  s->n = n;
  s->K = K;
  const size_t nK = (size_t)n * K;
  int e = GNP_OK;
  do {
    if ((e = dev_alloc(&s->V, nK * (m + 1))) != GNP_OK) break;
    if ((e = dev_alloc(&s->Z, nK * m)) != GNP_OK) break;
    if ((e = dev_alloc(&s->w, nK)) != GNP_OK) break;
    if ((e = dev_alloc(&s->b, nK)) != GNP_OK) break;
    if ((e = dev_alloc(&s->x, nK)) != GNP_OK) break;
    if ((e = dev_alloc(&s->Hg[0], nK * 16)) != GNP_OK) break;
    if ((e = dev_alloc(&s->Hg[1], nK * 16)) != GNP_OK) break;
    if ((e = dev_alloc(&s->st, (size_t)K)) != GNP_OK) break;
    if ((e = dev_alloc(&s->ctl, 3)) != GNP_OK) break;
    if ((e = dev_alloc(&s->one, 1)) != GNP_OK) break;
    {
      const double one = 1.0;
      if (cudaMemcpy(s->one, &one, sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("multi_create: cudaMemcpy failed");
        e = GNP_ERR_CUDA;
        break;
      }
    }
    if ((e = dev_alloc(&s->done, (size_t)K)) != GNP_OK) break;
    if ((e = dev_alloc(&s->H, (size_t)K * (m + 1) * m)) != GNP_OK) break;
    if ((e = dev_alloc(&s->R, (size_t)K * (m + 1) * m)) != GNP_OK) break;
    if ((e = dev_alloc(&s->cs, (size_t)K * m)) != GNP_OK) break;
    if ((e = dev_alloc(&s->sn, (size_t)K * m)) != GNP_OK) break;
    if ((e = dev_alloc(&s->g, (size_t)K * (m + 1))) != GNP_OK) break;
    if ((e = dev_alloc(&s->h1, (size_t)K * (m + 2))) != GNP_OK) break;
    if ((e = dev_alloc(&s->h2, (size_t)K * (m + 2))) != GNP_OK) break;
    if ((e = dev_alloc(&s->hist, (size_t)K * (maxiters + 1))) != GNP_OK) break;
    if ((e = dev_alloc(&s->thist, (size_t)K * (maxiters + 1))) != GNP_OK) break;
    const int maxb = std::max(4 * NUM_SMS_GB300, (n + MROWS - 1) / MROWS);  // >= dot_blocks(n)
    if ((e = red_alloc(s->red, maxb, (m + 2) * K)) != GNP_OK) break;
    if (cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&s->st_host), sizeof(DevState) * K) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&s->done_host), sizeof(int) * K) != cudaSuccess) {
      set_error("multi solver: stream or pinned allocation failed");
      e = GNP_ERR_OOM;
      break;
    }
  } while (0);
  if (e != GNP_OK) {
    multi_solver_free(s);
    return e;
  }
  s->m_cap = m;
  s->maxit_cap = maxiters;
  *out = s;
  return GNP_OK;
}

template <int K>
static int mgconv_attrs() {
  static bool done = false;
  if (done) return GNP_OK;
  const int bytes = (int)sizeof(MGconvSmem<K>);
  const void* fs[] = {(const void*)k_mgconv<K, GNP_LAYER_PAPER, false>, (const void*)k_mgconv<K, GNP_LAYER_PAPER, true>,
                      (const void*)k_mgconv<K, GNP_LAYER_RESID, false>, (const void*)k_mgconv<K, GNP_LAYER_RESID, true>};
  for (const void* f : fs) {
    GNP_TRY_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    GNP_TRY_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      std::min(100, (3 * (bytes + 1024) * 100 + 228 * 1024 - 1) / (228 * 1024))));
  }
  done = true;
  return GNP_OK;
}

// The L Res-GCONV layers of the K systems from S->Hg[0] (the last one fused with the
// decoder, z into column j of Z): the short-row kernels over the n K (node, system) pairs
// when every row has at most 16 nonzeros, else the K-node tile gather.
template <int K, int FORM>
static void mgnp_layers(gnp_model* M, MultiSolver* S, cudaStream_t st) {
  const gnp_mat* A = M->A;
  const int n = A->n, L = M->cfg.L;
  const double sqrt_n = std::sqrt((double)n);
  if (multi_row_ok(M)) {
    const ColPtr zp{S->Z, sizeof(float) * (size_t)n * K, S->ctl, 0};
    multi_row_layers(M, K, S->Hg[0], S->Hg[1], zp, S->one, S->ctl, st);  // launch errors: check_launch
    return;
  }
  EncW ew;
  DecW dw;
  fill_enc_dec(M->w_host, L, ew, dw);
  const int smem = (int)sizeof(MGconvSmem<K>);
  const int nt = (n + MGconvSmem<K>::ROWS - 1) / MGconvSmem<K>::ROWS;
  float* H0 = S->Hg[0];
  float* H1 = S->Hg[1];
  for (int l = 0; l < L; ++l) {
    LayerW lw;
    fill_layer_w(M->w_host, l, lw);
    if (l + 1 < L)
      k_mgconv<K, FORM, false><<<nt, TILE, smem, st>>>(A->rp, A->col, M->valhat, H0, H1, S->Z, n, S->ctl,
                                                      1.0 / sqrt_n, lw, dw);
    else
      k_mgconv<K, FORM, true><<<nt, TILE, smem, st>>>(A->rp, A->col, M->valhat, H0, H1, S->Z, n, S->ctl,
                                                     1.0 / sqrt_n, lw, dw);
    std::swap(H0, H1);
  }
}

// z_r = M(v_r) for every active system: the encoder (v_r normalised by vscale_r), then the
// layers.
template <int K, int FORM>
static void launch_mgnp(gnp_model* M, MultiSolver* S, cudaStream_t st) {
  const int n = M->A->n;
  EncW ew;
  DecW dw;
  fill_enc_dec(M->w_host, M->cfg.L, ew, dw);
  const int ne = (int)std::min<long long>(((long long)n * K + RED_THREADS - 1) / RED_THREADS, 8LL * NUM_SMS_GB300);
  k_mencode<K><<<ne, RED_THREADS, 0, st>>>(S->V, n, S->st, S->ctl, std::sqrt((double)n), S->Hg[0], ew);
  mgnp_layers<K, FORM>(M, S, st);
}

// The reorthogonalisation stream of the overlapped schedule (highest priority) and its
// fork/join events, made on first use.
static int multi_side(MultiSolver* S) {
  if (S->side) return GNP_OK;
  int lo = 0, hi = 0;
  GNP_TRY_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  GNP_TRY_CUDA(cudaStreamCreateWithPriority(&S->side, cudaStreamNonBlocking, hi));
  GNP_TRY_CUDA(cudaEventCreateWithFlags(&S->fork, cudaEventDisableTiming));
  GNP_TRY_CUDA(cudaEventCreateWithFlags(&S->join, cudaEventDisableTiming));
  return GNP_OK;
}

// The overlapped schedule applies to the GNP (M = I keeps the two-reduction passes).
static bool multi_overlapped(const gnp_model* M) { return M && ortho_overlapped(); }

// One overlapped restart cycle (the one-system schedule of krylov.cu for K systems): per
// step the encoder forms v'_j, the second pass of v'_j runs on S->side beside the layers,
// and k_mspmv_row<RDOT> makes the first pass against the final V_j.
template <int K>
static int launch_mcycle_ovl(gnp_mat* A, MultiSolver* S, gnp_model* M, int m, cudaStream_t st) {
  const int n = A->n;
  const int ntr = (n + MROWS - 1) / MROWS;
  const int nb = red_blocks(n);
  const int ncg = dot_blocks(n);
  const MStrides ms = mstrides(S->m_cap, S->maxit_cap);
  const double sqrt_n = std::sqrt((double)n);
  const bool short_rows = A->max_deg <= ROW_DMAX_M;
  GNP_TRY(multi_side(S));
  EncW ew;
  DecW dw;
  fill_enc_dec(M->w_host, M->cfg.L, ew, dw);
  const int ne = (int)std::min<long long>(((long long)n * K + RED_THREADS - 1) / RED_THREADS, 8LL * NUM_SMS_GB300);
  for (int j = 0; j < m; ++j) {
    if (j == 0) {
      k_mencode<K><<<ne, RED_THREADS, 0, st>>>(S->V, n, S->st, S->ctl, sqrt_n, S->Hg[0], ew);
    } else {
      k_mencode_d<K><<<ne, RED_THREADS, 0, st>>>(S->V, S->w, n, S->st, S->ctl, S->h2, sqrt_n, S->Hg[0], ew);
      GNP_TRY_CUDA(cudaEventRecord(S->fork, st));
      GNP_TRY_CUDA(cudaStreamWaitEvent(S->side, S->fork, 0));
      k_mreorth_dots<K><<<ncg, RED_THREADS, 0, S->side>>>(S->V, n, S->st, S->ctl, S->h1, S->h2, S->H, S->R, S->cs,
                                                          S->sn, S->g, S->hist, S->thist, ms, S->red.partials,
                                                          S->red.counter);
      k_mreorth_update<K><<<nb, RED_THREADS, 0, S->side>>>(S->V, n, S->st, S->ctl, S->h1);
      GNP_TRY_CUDA(cudaEventRecord(S->join, S->side));
    }
    if (M->cfg.form == GNP_LAYER_PAPER) mgnp_layers<K, GNP_LAYER_PAPER>(M, S, st);
    else mgnp_layers<K, GNP_LAYER_RESID>(M, S, st);
    if (j > 0) GNP_TRY_CUDA(cudaStreamWaitEvent(st, S->join, 0));
    if (short_rows)
      k_mspmv_row<K, float, true><<<ncg, RED_THREADS, 0, st>>>(A->rp, A->col, A->val, S->Z, S->w, n, S->ctl, S->V,
                                                               S->st, S->h2, S->red.partials, S->red.counter, S->H,
                                                               S->R, S->cs, S->sn, S->g, S->hist, S->thist, ms);
    else
      k_mspmv<K, float, true, true><<<ntr, TILE, 0, st>>>(A->rp, A->col, A->val, S->Z, S->w, n, S->ctl, S->V, S->st,
                                                          S->h2, S->red.partials, S->red.counter, S->H, S->R, S->cs,
                                                          S->sn, S->g, S->hist, S->thist, ms);
  }
  k_mdfinish<K><<<1, 32, 0, st>>>(S->st, S->ctl, S->h2, S->H, S->R, S->cs, S->sn, S->g, S->hist, S->thist, ms);
  k_mxupdate<K, float><<<nb, RED_THREADS, 0, st>>>(S->Z, S->x, n, S->st, S->R, S->g, ms, m);
  k_mresidual<K><<<ntr, TILE, 0, st>>>(A->rp, A->col, A->val, S->x, S->b, S->V, n, S->st, S->ctl, S->done, S->g,
                                       S->hist, S->thist, ms, S->red.partials, S->red.counter);
  return check_launch("multi cycle (overlapped CGS2)");
}

// One restart cycle for all systems: m Arnoldi steps, x update, residual.
template <int K>
static int launch_mcycle(gnp_mat* A, MultiSolver* S, gnp_model* M, int m, cudaStream_t st) {
  if (multi_overlapped(M)) return launch_mcycle_ovl<K>(A, S, M, m, st);
  const int n = A->n;
  const int ntr = (n + MROWS - 1) / MROWS;
  const int nb = red_blocks(n);
  const int ncg = dot_blocks(n);
  const MStrides ms = mstrides(S->m_cap, S->maxit_cap);
  const bool short_rows = A->max_deg <= ROW_DMAX_M;
  for (int j = 0; j < m; ++j) {
    // w = A z with CGS2 pass 1 (h1, ||w||^2) in the same kernel
    if (M) {
      if (M->cfg.form == GNP_LAYER_PAPER) launch_mgnp<K, GNP_LAYER_PAPER>(M, S, st);
      else launch_mgnp<K, GNP_LAYER_RESID>(M, S, st);
      if (short_rows)
        k_mspmv_row<K, float><<<ncg, RED_THREADS, 0, st>>>(A->rp, A->col, A->val, S->Z, S->w, n, S->ctl, S->V,
                                                           S->st, S->h1, S->red.partials, S->red.counter);
      else
        k_mspmv<K, float, true><<<ntr, TILE, 0, st>>>(A->rp, A->col, A->val, S->Z, S->w, n, S->ctl, S->V, S->st,
                                                      S->h1, S->red.partials, S->red.counter);
    } else {
      k_mvscale<K><<<nb, RED_THREADS, 0, st>>>(S->V, n, S->st, S->ctl);
      if (short_rows)
        k_mspmv_row<K, double><<<ncg, RED_THREADS, 0, st>>>(A->rp, A->col, A->val, S->V, S->w, n, S->ctl, S->V,
                                                            S->st, S->h1, S->red.partials, S->red.counter);
      else
        k_mspmv<K, double, true><<<ntr, TILE, 0, st>>>(A->rp, A->col, A->val, S->V, S->w, n, S->ctl, S->V,
                                                       S->st, S->h1, S->red.partials, S->red.counter);
    }
    k_mcgs<K, 2><<<ncg, RED_THREADS, 0, st>>>(S->V, n, S->w, S->st, S->ctl, S->h1, S->h2, S->H, S->R, S->cs,
                                              S->sn, S->g, S->hist, S->thist, ms, S->red.partials, S->red.counter);
    k_mcgs<K, 3><<<ncg, RED_THREADS, 0, st>>>(S->V, n, S->w, S->st, S->ctl, S->h1, S->h2, S->H, S->R, S->cs,
                                              S->sn, S->g, S->hist, S->thist, ms, S->red.partials, S->red.counter);
  }
  if (M)
    k_mxupdate<K, float><<<nb, RED_THREADS, 0, st>>>(S->Z, S->x, n, S->st, S->R, S->g, ms, m);
  else
    k_mxupdate<K, double><<<nb, RED_THREADS, 0, st>>>(S->V, S->x, n, S->st, S->R, S->g, ms, m);
  k_mresidual<K><<<ntr, TILE, 0, st>>>(A->rp, A->col, A->val, S->x, S->b, S->V, n, S->st, S->ctl, S->done, S->g,
                                       S->hist, S->thist, ms, S->red.partials, S->red.counter);
  return check_launch("multi cycle");
}

static int mread(MultiSolver* S, cudaStream_t st) {
  GNP_TRY_CUDA(cudaMemcpyAsync(S->st_host, S->st, sizeof(DevState) * S->K, cudaMemcpyDeviceToHost, st));
  GNP_TRY_CUDA(cudaStreamSynchronize(st));
  return GNP_OK;
}

static int mdone_upload(MultiSolver* S, cudaStream_t st) {
  GNP_TRY_CUDA(cudaMemcpyAsync(S->done, S->done_host, sizeof(int) * S->K, cudaMemcpyHostToDevice, st));
  return GNP_OK;
}

template <int K>
static int solve_multi(gnp_mat* A, const double* B, double* X, int k, gnp_model* M, int restart, double rtol,
                       int maxiters, gnp_solve_info* infos, cudaStream_t st_in) {
  const auto t0 = std::chrono::steady_clock::now();
  MultiSolver*& S = A->msolver;
  if (!S || S->K != K || S->m_cap < restart || S->maxit_cap < maxiters) {
    const int m_new = S && S->K == K ? std::max(restart, S->m_cap) : restart;
    const int it_new = S && S->K == K ? std::max(maxiters, S->maxit_cap) : maxiters;
    multi_solver_free(S);
    S = nullptr;
    GNP_TRY(multi_create(A->n, K, m_new, it_new, &S));
  }
  cudaStream_t st = st_in;
  if (st == nullptr || st == cudaStreamLegacy) {
    GNP_TRY_CUDA(cudaStreamSynchronize(st));
    st = S->own;
  }
  if (M) {
    GNP_TRY(apply_prepare(M));
    GNP_TRY(mgconv_attrs<K>());
  }
  const int n = A->n;
  const int nb = red_blocks(n);
  const int ntr = (n + MROWS - 1) / MROWS;
  const MStrides ms = mstrides(S->m_cap, S->maxit_cap);
  const int ge = (int)std::min<long long>(((long long)n * K + 255) / 256, 8LL * NUM_SMS_GB300);
  k_mpack<K><<<ge, 256, 0, st>>>(B, k, n, S->b);
  k_mpack<K><<<ge, 256, 0, st>>>(X, k, n, S->x);
  for (int r = 0; r < K; ++r) {
    DevState init{};
    init.maxiters = maxiters;
    init.m = restart;
    init.rtol = rtol;
    S->st_host[r] = init;
    S->done_host[r] = r < k ? 0 : 1;
  }
  GNP_TRY_CUDA(cudaMemcpyAsync(S->st, S->st_host, sizeof(DevState) * K, cudaMemcpyHostToDevice, st));
  GNP_TRY(mdone_upload(S, st));
  GNP_TRY_CUDA(cudaMemsetAsync(S->H, 0, sizeof(double) * (size_t)K * ms.hs, st));
  k_mbnorm<K><<<nb, RED_THREADS, 0, st>>>(S->b, n, S->st, S->red.partials, S->red.counter);
  k_mresidual<K><<<ntr, TILE, 0, st>>>(A->rp, A->col, A->val, S->x, S->b, S->V, n, S->st, S->ctl, S->done, S->g,
                                       S->hist, S->thist, ms, S->red.partials, S->red.counter);
  GNP_TRY(check_launch("multi init"));
  GNP_TRY(mread(S, st));
  std::vector<int> status(K, GNP_OK);
  std::vector<CycleCtl> cc(K);
  std::vector<DevState> fin(K);
  std::vector<double> beta_prev(K);
  int remaining = 0;
  for (int r = 0; r < K; ++r) {
    const DevState& hs = S->st_host[r];
    fin[r] = hs;
    if (r >= k) continue;
    bool end = true;
    if (hs.bnorm == 0.0) {
      k_mzero<K><<<nb, RED_THREADS, 0, st>>>(S->x, n, r);
      fin[r].beta = 0.0;
    } else if (!std::isfinite(hs.beta) || !std::isfinite(hs.bnorm)) {
      status[r] = GNP_ERR_NAN;
    } else if (hs.beta <= hs.tol) {
      status[r] = GNP_OK;
    } else if (maxiters == 0) {
      status[r] = GNP_ERR_NOT_CONVERGED;
    } else {
      end = false;
    }
    if (end) S->done_host[r] = 1;
    else ++remaining;
  }
  GNP_TRY(mdone_upload(S, st));
  int cycles = 0;
  if (remaining > 0) {
    // the first cycle must see the systems that ended at the start as inactive
    k_mresidual<K><<<ntr, TILE, 0, st>>>(A->rp, A->col, A->val, S->x, S->b, S->V, n, S->st, S->ctl, S->done,
                                         S->g, S->hist, S->thist, ms, S->red.partials, S->red.counter);
    GNP_TRY(check_launch("multi restart"));
  }
  const unsigned long long ver = M ? model_version(M) : 0ull;
  while (remaining > 0) {
    if (!S->gexec || S->g_model != M || S->g_version != ver || S->g_m != restart || S->g_stream != st ||
        S->g_ortho != ortho_overlapped()) {
      if (S->gexec) cudaGraphExecDestroy(S->gexec);
      S->gexec = nullptr;
      cudaGraph_t graph;
      GNP_TRY_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      int ls = launch_mcycle<K>(A, S, M, restart, st);
      cudaError_t ce = cudaStreamEndCapture(st, &graph);
      if (ls != GNP_OK) return ls;
      if (ce != cudaSuccess) {
        set_error("multi: graph capture failed: %s", cudaGetErrorString(ce));
        return GNP_ERR_CUDA;
      }
      ce = cudaGraphInstantiate(&S->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) {
        S->gexec = nullptr;
        set_error("multi: graph instantiate failed: %s", cudaGetErrorString(ce));
        return GNP_ERR_CUDA;
      }
      S->g_model = M;
      S->g_version = ver;
      S->g_m = restart;
      S->g_stream = st;
      S->g_ortho = ortho_overlapped();
    }
    for (int r = 0; r < K; ++r) beta_prev[r] = S->st_host[r].beta;
    GNP_TRY_CUDA(cudaGraphLaunch(S->gexec, st));
    ++cycles;
    GNP_TRY(mread(S, st));
    for (int r = 0; r < k; ++r) {
      if (S->done_host[r]) continue;
      const DevState& hs = S->st_host[r];
      int s = GNP_OK;
      if (cycle_after(hs, beta_prev[r], maxiters, cc[r], &s)) {
        status[r] = s;
        fin[r] = hs;
        S->done_host[r] = 1;
        --remaining;
      }
    }
    GNP_TRY(mdone_upload(S, st));
  }
  k_munpack<K><<<ge, 256, 0, st>>>(S->x, k, n, X);
  GNP_TRY(check_launch("multi unpack"));
  GNP_TRY_CUDA(cudaStreamSynchronize(st));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  int worst = GNP_OK;
  for (int r = 0; r < k; ++r) {
    if (status[r] != GNP_OK && worst == GNP_OK) worst = status[r];
    if (!infos) continue;
    gnp_solve_info* info = infos + r;
    const DevState& hs = fin[r];
    info->iters = hs.iters;
    info->restarts = cc[r].restarts;
    info->status = status[r];
    info->seconds = secs;
    info->cycles = cycles;
    info->gconv_launches = 0;
    info->gconv_ms = 0.0;
    const double bn = hs.bnorm > 0.0 ? hs.bnorm : 1.0;
    info->rel_res_true = hs.bnorm > 0.0 ? hs.beta / bn : 0.0;
    info->rel_res_est = hs.iters > 0 ? hs.res_est / bn : info->rel_res_true;
    const int cnt = hs.bnorm > 0.0 ? hs.iters + 1 : 1;
    if (info->res_history) {
      if (hs.bnorm > 0.0) {
        GNP_TRY_CUDA(cudaMemcpy(info->res_history, S->hist + (size_t)r * ms.hist, sizeof(double) * cnt,
                                cudaMemcpyDeviceToHost));
      } else {
        info->res_history[0] = 0.0;
      }
      info->res_history_len = cnt;
    }
    if (info->time_history) {
      if (hs.bnorm > 0.0) {
        std::vector<unsigned long long> ns(cnt);
        GNP_TRY_CUDA(cudaMemcpy(ns.data(), S->thist + (size_t)r * ms.hist, sizeof(unsigned long long) * cnt,
                                cudaMemcpyDeviceToHost));
        for (int i = 0; i < cnt; ++i) info->time_history[i] = 1e-9 * (double)ns[i];
      } else {
        info->time_history[0] = 0.0;
      }
    }
    if (info->hessenberg) info->hessenberg_cols = 0;
  }
  return worst;
}

template <int K>
static int apply_multi(gnp_model* M, const double* v, int k, float* z, cudaStream_t st) {
  gnp_mat* A = M->A;
  MultiSolver*& S = A->msolver;
  if (!S || S->K != K) {
    multi_solver_free(S);
    S = nullptr;
    GNP_TRY(multi_create(A->n, K, 1, 1, &S));
  }
  GNP_TRY(apply_prepare(M));
  GNP_TRY(mgconv_attrs<K>());
  const int n = A->n;
  const int nb = red_blocks(n);
  const int ge = (int)std::min<long long>(((long long)n * K + 255) / 256, 8LL * NUM_SMS_GB300);
  k_mpack<K><<<ge, 256, 0, st>>>(v, k, n, S->V);
  k_mbnorm<K><<<nb, RED_THREADS, 0, st>>>(S->V, n, S->st, S->red.partials, S->red.counter);
  // tau_r = the bnorm the kernel just stored; copy it out of the states into h1
  k_mtau<K><<<1, 32, 0, st>>>(S->st, S->h1);
  k_mapply_setup<K><<<1, 32, 0, st>>>(S->st, S->ctl, S->h1);
  if (M->cfg.form == GNP_LAYER_PAPER) launch_mgnp<K, GNP_LAYER_PAPER>(M, S, st);
  else launch_mgnp<K, GNP_LAYER_RESID>(M, S, st);
  k_mapply_out<K><<<ge, 256, 0, st>>>(S->Z, S->h1, k, n, z);
  return check_launch("gnp_apply_multi");
}

}  // namespace gnp

using namespace gnp;

extern "C" int gnp_apply_multi(gnp_model* M, const double* v, int k, float* z, void* stream) {
  GNP_REQUIRE(M && v && z, "gnp_apply_multi: null argument");
  GNP_REQUIRE(k >= 1 && k <= GNP_MAX_RHS, "gnp_apply_multi: k = %d out of [1, %d]", k, GNP_MAX_RHS);
  GNP_REQUIRE(M->hprec == GNP_H_FP32 && M->cfg.L >= 1, "gnp_apply_multi: float32 hidden blocks, L >= 1");
  GNP_REQUIRE(!M->cfg.no_scale, "gnp_apply_multi: the scaling s is required");
  cudaStream_t st = as_stream(stream);
  if (k <= 2) return apply_multi<2>(M, v, k, z, st);
  if (k <= 4) return apply_multi<4>(M, v, k, z, st);
  return apply_multi<8>(M, v, k, z, st);
}

extern "C" int fgmres_solve_multi(gnp_mat* A, const double* B, double* X, int k, gnp_model* M, int restart,
                                  double rtol, int maxiters, gnp_solve_info* infos, void* stream) {
  GNP_REQUIRE(A && B && X, "fgmres_solve_multi: null argument");
  GNP_REQUIRE(k >= 1 && k <= GNP_MAX_RHS, "fgmres_solve_multi: k = %d out of [1, %d]", k, GNP_MAX_RHS);
  GNP_REQUIRE(restart >= 1 && restart <= GNP_MAX_RESTART_MULTI, "fgmres_solve_multi: restart %d out of [1, %d]",
              restart, GNP_MAX_RESTART_MULTI);
  GNP_REQUIRE(maxiters >= 0 && rtol >= 0.0, "fgmres_solve_multi: bad maxiters/rtol");
  GNP_REQUIRE(!M || M->A == A, "fgmres_solve_multi: the preconditioner was built for another matrix");
  GNP_REQUIRE(!M || M->hprec == GNP_H_FP32, "fgmres_solve_multi: float32 hidden blocks only");
  GNP_REQUIRE(!M || M->cfg.L >= 1, "fgmres_solve_multi: the GNP needs at least one layer");
  GNP_REQUIRE(!M || !M->cfg.no_scale, "fgmres_solve_multi: the scaling s is required");
  cudaStream_t st = as_stream(stream);
  if (k <= 2) return solve_multi<2>(A, B, X, k, M, restart, rtol, maxiters, infos, st);
  if (k <= 4) return solve_multi<4>(A, B, X, k, M, restart, rtol, maxiters, infos, st);
  return solve_multi<8>(A, B, X, k, M, restart, rtol, maxiters, infos, st);
}
