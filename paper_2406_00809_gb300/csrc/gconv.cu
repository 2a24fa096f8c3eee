// The GNP operator z = M(v) (Sec. 2.3, Fig. 1): scaling s (Eq. 8), MLP encoder,
// L Res-GCONV layers over A_hat = A/gamma (Eqs. 6-7), MLP decoder, back-scaling.
//
// Kernels (one launch each):
//   k_vnorm      tau = ||v||_2 (deterministic two-level reduction; standalone apply).
//   k_encode     u_i = (sqrt(n)/tau) v_i; h_i = W2^T ReLU(W1^T u_i + b1) + b2 (1->32->16);
//                inside FGMRES it first scales the stored vector to v_j = w / h_{j,j-1}.
//   k_encode_vn  the encoder of FGMRES steps >= 1: forms v_j = (w1 - V h2) / h_{j,j-1}
//                itself while one extra block finishes the previous step.
//   k_gconv_row  one Res-GCONV layer for matrices whose rows have at most 16 nonzeros:
//                four lanes per row gather every neighbour at once, then per row four
//                threads compute ReLU(h_i U + (A_hat H)_i W) or h_i + ReLU((A_hat H)_i W)
//                on paired float32 multiply-adds.
//   k_gconv      one Res-GCONV layer for any row lengths: nnz-balanced CSR tile gather
//                over the n x 16 hidden block with 16-byte loads, thread-per-row epilogue
//                with U and W as uniform kernel-parameter operands.
//   k_gconv_row_dec, k_gconv_dec  the last layer with the decoder (16->32->1) and the
//                back-scaling tau/sqrt(n) fused into the epilogue: writes z_i, never H^L.
// Hidden blocks are node-major (16 contiguous values per node), float32 or bfloat16.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstring>

#include "gconv_common.cuh"
#include "gconv_rows.cuh"
#include "solver.h"

namespace gnp {


// A_hat values = A / gamma in float32 (Eq. 6), in the CSR order.
__global__ void k_scale_values(const double* __restrict__ val, long long nnz, double gamma,
                               float* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = (float)(val[e] / gamma);
}

__device__ __forceinline__ void* colptr(const ColPtr& p) {
  int j = p.jptr ? *p.jptr : 0;
  return static_cast<char*>(p.base) + (size_t)(j + p.off) * p.stride;
}

// ---------------------------------------------------------------- k_vnorm

__global__ void __launch_bounds__(RED_THREADS)
k_vnorm(ColPtr vp, const int* __restrict__ ctl, int n, double* __restrict__ partials,
        unsigned* __restrict__ counter, double* __restrict__ tau) {
  if (ctl && !ctl[1]) return;
  __shared__ double sh[32];
  const double* v = static_cast<const double*>(colptr(vp));
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double x = v[i];
    acc += x * x;
  }
  double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
  if (last_block_arrive(counter)) {
    __shared__ double tot[1];
    reduce_partials(partials, gridDim.x, 1, tot);
    if (threadIdx.x == 0) {
      *tau = sqrt(tot[0]);
      *counter = 0;
    }
  }
}


// ---------------------------------------------------------------- tile staging


// Coalesced copy between a global tile of `rows` hidden rows and the smem staging tile.
template <class HT, bool TO_GLOBAL>
__device__ __forceinline__ void tile_copy(uint32_t* stile, HT* g, int r0, int rows) {
  constexpr int V16 = HTraits<HT>::ROW_BYTES / 16;  // 16-byte chunks per row
  uint4* gb = reinterpret_cast<uint4*>(g + (size_t)r0 * 16);
  for (int i = threadIdx.x; i < rows * V16; i += blockDim.x) {
    int r = i / V16, k = i % V16;
    uint4* s = reinterpret_cast<uint4*>(stile + r * HTraits<HT>::SROW) + k;
    if (TO_GLOBAL) gb[i] = *s;
    else *s = __ldg(gb + i);
  }
}

// ---------------------------------------------------------------- k_encode

// Standalone apply: u = (sqrt(n)/tau) v with tau from k_vnorm.  Inside FGMRES
// (vscale != null): v_j = w / h is unit-norm by construction, so the encoder scales the
// stored w by 1/h (h the device scalar), writes v_j back in place and uses tau = 1 (it stores
// tau = 1 for the decoder's back-scaling).  noscale (the ablation without s): u = v, and
// tau = sqrt(n) is stored so that the decoder's factor tau/sqrt(n) is 1.
template <class HT>
__device__ __forceinline__ void encode_body(VGrid gr, ColPtr vp, const double* __restrict__ vscale,
                                            double* __restrict__ tau, const int* __restrict__ ctl, int n,
                                            double sqrt_n, int noscale, HT* __restrict__ H, const EncW& ew) {
  if (ctl && !ctl[1]) return;
  __shared__ __align__(16) uint32_t stile[TILE * HTraits<HT>::SROW];
  double* v = static_cast<double*>(colptr(vp));
  const int r0 = gr.bid * TILE;
  const int rows = min(TILE, n - r0);
  const int t = threadIdx.x;
  // the block's scalars once (a float64 division is slow on GB300): u = f * v, and the
  // FGMRES step's v_j = w * (1 / h_{j,j-1})
  __shared__ double s_f, s_inv;
  if (t == 0) {
    s_inv = vscale ? 1.0 / *vscale : 1.0;  // v_j = w / h whether or not s is applied
    if (noscale) {
      s_f = 1.0;
      if (gr.bid == 0) *tau = sqrt_n;
    } else if (vscale) {
      s_f = sqrt_n;
      if (gr.bid == 0) *tau = 1.0;
    } else {
      const double tv = *tau;
      s_f = tv > 0.0 ? sqrt_n / tv : 0.0;
    }
  }
  __syncthreads();
  const double f = s_f;
  if (t < rows) {
    double x = v[r0 + t];
    if (vscale) {
      x = x * s_inv;
      v[r0 + t] = x;
    }
    float u = (float)(x * f);
    float h[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) h[c] = ew.b2[c];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const float a = fmaxf(fmaf(u, ew.W1[k], ew.b1[k]), 0.0f);
#pragma unroll
      for (int c = 0; c < 16; c += 2)  // two outputs per paired multiply-add, each an fmaf
        ffma2(h[c], h[c + 1], a, a, ew.W2[k * 16 + c], ew.W2[k * 16 + c + 1]);
    }
    stage_row<HT>(stile, t, h);
  }
  __syncthreads();
  tile_copy<HT, true>(stile, H, r0, rows);
}

template <class HT>
__global__ void __launch_bounds__(TILE)
k_encode(ColPtr vp, const double* __restrict__ vscale, double* __restrict__ tau, const int* __restrict__ ctl,
         int n, double sqrt_n, int noscale, HT* __restrict__ H, const __grid_constant__ EncW ew) {
  encode_body<HT>(hw_grid(), vp, vscale, tau, ctl, n, sqrt_n, noscale, H, ew);
}

// The encoder inside FGMRES from step 1 on (vn: the pending step j = st->jv): the last
// block finishes step j (vnext_finish: Givens update, continue decision) while the others
// form v_{j+1} = (w1 - V_j h2) / h_{j+1,j} for their rows in float64, store it as
// V[:, j+1] and encode it as k_encode does with u = sqrt(n) v (unit-norm v, tau = 1;
// noscale: u = v, tau = sqrt(n)).  The rows are formed even if the finish ends the cycle;
// every later kernel of the step then sees active = 0 and returns.
template <class HT>
__device__ __forceinline__ void encode_vn_body(VGrid gr, const VNext& vn, int n, double sqrt_n, int noscale,
                                               double* __restrict__ tau, HT* __restrict__ H, const EncW& ew) {
  if (gr.bid == gr.nblk - 1) {
    vnext_finish(vn);
    return;
  }
  const DevState* st = vn.st;
  if (!st->active) return;
  __shared__ __align__(16) uint32_t stile[TILE * HTraits<HT>::SROW];
  __shared__ double shh[GNP_MAX_RESTART + 4];
  __shared__ double shn, sinv;
  const int j = st->jv;
  const int t = threadIdx.x;
  for (int k = t; k <= j; k += blockDim.x) shh[k] = vn.h2[k];
  vnext_hnorm(vn.h2, j, st->w1sq, &shn);
  if (t == 0) {
    sinv = 1.0 / shn;  // once per block (thread 0 wrote shn): float64 division is slow
    if (gr.bid == 0) *tau = noscale ? sqrt_n : 1.0;
  }
  __syncthreads();
  const double inv = sinv;
  const double f = noscale ? 1.0 : sqrt_n;
  const int r0 = gr.bid * TILE;
  const int rows = min(TILE, n - r0);
  if (t < rows) {
    const size_t ld = (size_t)n;
    const int i = r0 + t;
    double x = vn.w[i];
#pragma unroll 8
    for (int k = 0; k <= j; ++k) x -= vn.V[k * ld + i] * shh[k];
    x = x * inv;
    vn.V[(size_t)(j + 1) * ld + i] = x;
    const float u = (float)(x * f);
    float h[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) h[c] = ew.b2[c];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const float a = fmaxf(fmaf(u, ew.W1[k], ew.b1[k]), 0.0f);
#pragma unroll
      for (int c = 0; c < 16; c += 2) ffma2(h[c], h[c + 1], a, a, ew.W2[k * 16 + c], ew.W2[k * 16 + c + 1]);
    }
    stage_row<HT>(stile, t, h);
  }
  __syncthreads();
  tile_copy<HT, true>(stile, H, r0, rows);
}

template <class HT>
__global__ void __launch_bounds__(TILE)
k_encode_vn(const VNext vn, int n, double sqrt_n, int noscale, double* __restrict__ tau, HT* __restrict__ H,
            const __grid_constant__ EncW ew) {
  encode_vn_body<HT>(hw_grid(), vn, n, sqrt_n, noscale, tau, H, ew);
}

// The encoder of the overlapped-CGS2 step s + 1 >= 1 (vn.dcgs; s = st->jd, whose first
// pass just finished; V_s is final): for its rows,
//   v'_{s+1} = (w_s - V_s h_s) / rho_s   (-> V[:, s+1], rho_s as normalised by the pass),
// encoded as k_encode_vn encodes its vector (unit norm: u = sqrt(n) v', tau = 1;
// noscale: u = v', tau = sqrt(n)).  After a breakdown 1/rho_s is 0 and v'_{s+1} = 0; the
// cycle has ended by then, and every later kernel returns.
template <class HT>
__global__ void __launch_bounds__(TILE)
k_encode_dv(const VNext vn, int n, double sqrt_n, int noscale, double* __restrict__ tau, HT* __restrict__ H,
            const __grid_constant__ EncW ew) {
  const DevState* st = vn.st;
  if (!st->active) return;
  __shared__ __align__(16) uint32_t stile[TILE * HTraits<HT>::SROW];
  __shared__ double sh[GNP_MAX_RESTART + 4];
  __shared__ double s_rho;
  const int s = st->jd;
  const int t = threadIdx.x;
  for (int k = t; k <= s; k += blockDim.x) sh[k] = vn.h2[k];
  if (t == 0) {
    s_rho = st->rho_inv;
    if (blockIdx.x == 0) *tau = noscale ? sqrt_n : 1.0;
  }
  __syncthreads();
  const double rho_inv = s_rho;
  const double f = noscale ? 1.0 : sqrt_n;
  const int r0 = blockIdx.x * TILE;
  const int rows = min(TILE, n - r0);
  if (t < rows) {
    const size_t ld = (size_t)n;
    const int i = r0 + t;
    double y = vn.w[i];
#pragma unroll 8
    for (int k = 0; k <= s; ++k) y -= vn.V[k * ld + i] * sh[k];
    y = y * rho_inv;
    vn.V[(size_t)(s + 1) * ld + i] = y;
    const float u = (float)(y * f);
    float h[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) h[c] = ew.b2[c];
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const float a = fmaxf(fmaf(u, ew.W1[k], ew.b1[k]), 0.0f);
#pragma unroll
      for (int c = 0; c < 16; c += 2) ffma2(h[c], h[c + 1], a, a, ew.W2[k * 16 + c], ew.W2[k * 16 + c + 1]);
    }
    stage_row<HT>(stile, t, h);
  }
  __syncthreads();
  tile_copy<HT, true>(stile, H, r0, rows);
}

// ---------------------------------------------------------------- k_gconv
//
// One block of TILE threads per ROWS consecutive rows (ROWS = 256: one epilogue thread per
// row; ROWS = 128: two, each computing 8 of the 16 outputs, which halves every thread's
// share of the gather and of the epilogue for matrices too small to fill the GPU with
// 256-row tiles).  The tile's nonzeros are split evenly over slots of G lanes (4 for
// float32 rows of 64 bytes, 2 for bfloat16 rows of 32 bytes); a slot walks its nonzero
// range loading each neighbour's row with one 16-byte load per lane, four nonzeros in
// flight; rows split between slots leave partial sums that the epilogue adds in slot
// order (common.cuh, tile_gather).  The block's own hidden rows come in with one
// coalesced tile copy.  Epilogue: U and W as uniform constant-bank operands; the output
// rows are staged in shared memory and the tile written back with coalesced stores, or
// (last layer) the decoder and tau/sqrt(n) produce z directly.

template <class HT, int ROWS>
struct GconvSmem {
  TileSmem<typename HTraits<HT>::TR, ROWS> g;
  __align__(16) uint32_t stile[ROWS * HTraits<HT>::SROW];
  float zpart[ROWS];  // second half of the decoder sum (two threads per row)
};


// Store outputs [K0, K0+OPT) of row t into the staging tile (the row's own slot).
template <class HT, int K0, int OPT>
__device__ __forceinline__ void stage_part(uint32_t* stile, int t, const float (&o)[OPT]) {
  if constexpr (OPT == 16) {
    stage_row<HT>(stile, t, o);
  } else if constexpr (sizeof(HT) == 4) {
    float4* d = reinterpret_cast<float4*>(stile + t * HTraits<HT>::SROW + K0);
#pragma unroll
    for (int q = 0; q < OPT / 4; ++q) d[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
  } else {
    static_assert(OPT == 8, "bfloat16 halves are 8 values (16 bytes)");
    uint4* d = reinterpret_cast<uint4*>(stile + t * HTraits<HT>::SROW + K0 / 2);
    d[0] = make_uint4(pack_bf16x2(o[0], o[1]), pack_bf16x2(o[2], o[3]), pack_bf16x2(o[4], o[5]),
                      pack_bf16x2(o[6], o[7]));
  }
}

// Gather + this thread's share of the layer for row t = threadIdx.x % ROWS; `part`
// (threadIdx.x / ROWS, warp-uniform) selects the outputs.  Leaves the outputs in `o`.
template <class HT, int FORM, int ROWS, int K0, int OPT>
__device__ __forceinline__ void gconv_part(GconvSmem<HT, ROWS>& sm, int t, int rows, const LayerW& lw,
                                           float (&o)[OPT]) {
  using TR = typename HTraits<HT>::TR;
  if (t < rows) {
    float h[16], agg[16];
    unstage_row<HT>(sm.stile, t, h);
    tile_row_sum<TR, 16>(sm.g, t, 0, agg);
    layer_part<FORM, K0, OPT>(h, agg, lw, o);
  }
}


// The tile's hidden rows and its gather; the row pointers are already in sm.g.rp.
template <class HT, int ROWS, int GROUP>
__device__ __forceinline__ void gconv_load_gather(GconvSmem<HT, ROWS>& sm, const int* __restrict__ col,
                                                  const float* __restrict__ valhat, const HT* __restrict__ Hin,
                                                  int r0, int rows) {
  using TR = typename HTraits<HT>::TR;
  tile_copy<HT, false>(sm.stile, const_cast<HT*>(Hin), r0, rows);
  __syncthreads();
  tile_gather<TR, TileSmem<TR, ROWS>, GROUP>(sm.g, rows, col, valhat, Hin);
  __syncthreads();
}

template <int ROWS> struct GconvBounds { static constexpr int MIN_BLOCKS = 3; };
template <> struct GconvBounds<128> { static constexpr int MIN_BLOCKS = 4; };

template <class HT, int FORM, int ROWS, int GROUP>
__global__ void __launch_bounds__(TILE, GconvBounds<ROWS>::MIN_BLOCKS)
k_gconv(const int* __restrict__ rp, const int* __restrict__ col, const float* __restrict__ valhat,
        const HT* __restrict__ Hin, HT* __restrict__ Hout, int n, int trows, const int* __restrict__ ctl,
        const __grid_constant__ LayerW lw) {
  static_assert(ROWS == TILE || 2 * ROWS == TILE, "one or two epilogue threads per row");
  extern __shared__ __align__(16) unsigned char smraw[];
  GconvSmem<HT, ROWS>& sm = *reinterpret_cast<GconvSmem<HT, ROWS>*>(smraw);
  const int r0 = blockIdx.x * trows;  // trows <= ROWS rows per tile
  const int rows = min(trows, n - r0);
  tile_load_rp<typename HTraits<HT>::TR>(sm.g, rp, r0, rows);
  pdl_wait();
  if (ctl && !ctl[1]) return;
  gconv_load_gather<HT, ROWS, GROUP>(sm, col, valhat, Hin, r0, rows);
  const int t = threadIdx.x % ROWS;
  if constexpr (ROWS == TILE) {
    float o[16];
    gconv_part<HT, FORM, ROWS, 0, 16>(sm, t, rows, lw, o);
    // own row was read from stile by this thread only: safe to overwrite in place
    if (t < rows) stage_part<HT, 0, 16>(sm.stile, t, o);
  } else {
    float o[8];
    const bool hi = threadIdx.x >= ROWS;
    if (hi) gconv_part<HT, FORM, ROWS, 8, 8>(sm, t, rows, lw, o);
    else gconv_part<HT, FORM, ROWS, 0, 8>(sm, t, rows, lw, o);
    __syncthreads();  // both threads of a row have read its input from stile
    if (t < rows) {
      if (hi) stage_part<HT, 8, 8>(sm.stile, t, o);
      else stage_part<HT, 0, 8>(sm.stile, t, o);
    }
  }
  pdl_release();
  __syncthreads();
  tile_copy<HT, true>(sm.stile, Hout, r0, rows);
}


template <class HT, int FORM, int ROWS, int GROUP>
__global__ void __launch_bounds__(TILE, GconvBounds<ROWS>::MIN_BLOCKS)
k_gconv_dec(const int* __restrict__ rp, const int* __restrict__ col, const float* __restrict__ valhat,
            const HT* __restrict__ Hin, ColPtr zp, const double* __restrict__ tau, double sqrt_n,
            int n, int trows, const int* __restrict__ ctl, const __grid_constant__ LayerW lw,
            const __grid_constant__ DecW dw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  GconvSmem<HT, ROWS>& sm = *reinterpret_cast<GconvSmem<HT, ROWS>*>(smraw);
  const int r0 = blockIdx.x * trows;  // trows <= ROWS rows per tile
  const int rows = min(trows, n - r0);
  tile_load_rp<typename HTraits<HT>::TR>(sm.g, rp, r0, rows);
  pdl_wait();
  if (ctl && !ctl[1]) return;
  __shared__ float s_back;
  if (threadIdx.x == 0) {  // once per block: a float64 division is slow on GB300
    const double tv = *tau;
    s_back = (float)(tv > 0.0 ? tv / sqrt_n : 0.0);
  }
  gconv_load_gather<HT, ROWS, GROUP>(sm, col, valhat, Hin, r0, rows);  // ends with a barrier
  const int t = threadIdx.x % ROWS;
  const float back = s_back;
  float* z = static_cast<float*>(colptr(zp));
  if constexpr (ROWS == TILE) {
    float o[16];
    gconv_part<HT, FORM, ROWS, 0, 16>(sm, t, rows, lw, o);
    if (t < rows) z[r0 + t] = decode_row(o, dw) * back;
  } else {
    // the two halves of each output row meet in float32 in the (no longer needed)
    // aggregate area; each thread then evaluates half of the decoder's hidden units
    float o[8];
    const bool hi = threadIdx.x >= ROWS;
    if (hi) gconv_part<HT, FORM, ROWS, 8, 8>(sm, t, rows, lw, o);
    else gconv_part<HT, FORM, ROWS, 0, 8>(sm, t, rows, lw, o);
    using TR = typename HTraits<HT>::TR;
    constexpr int ST = TR::STRIDE;
    static_assert(ST >= 16, "aggregate rows hold 16 floats");
    __syncthreads();  // every thread is done with the aggregates
    if (t < rows) {
#pragma unroll
      for (int k = 0; k < 8; ++k) sm.g.agg[t * ST + (hi ? 8 : 0) + k] = o[k];
    }
    __syncthreads();
    float zp_part = 0.0f;
    if (t < rows) {
      float full[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) full[k] = sm.g.agg[t * ST + k];
      zp_part = hi ? decode_part<16, 16>(full, dw) : decode_part<0, 16>(full, dw);
      if (hi) sm.zpart[t] = zp_part;
    }
    __syncthreads();
    if (!hi && t < rows) z[r0 + t] = ((dw.b2 + zp_part) + sm.zpart[t]) * back;
  }
}

// Standalone decoder (L = 0, or the trace path that keeps H^L).
template <class HT>
__global__ void __launch_bounds__(TILE)
k_decode(const HT* __restrict__ H, ColPtr zp, const double* __restrict__ tau, double sqrt_n, int n,
         const int* __restrict__ ctl, const __grid_constant__ DecW dw) {
  if (ctl && !ctl[1]) return;
  __shared__ __align__(16) uint32_t stile[TILE * HTraits<HT>::SROW];
  const int r0 = blockIdx.x * TILE;
  const int rows = min(TILE, n - r0);
  __shared__ float s_back;
  if (threadIdx.x == 0) {  // once per block: a float64 division is slow on GB300
    const double tv = *tau;
    s_back = (float)(tv > 0.0 ? tv / sqrt_n : 0.0);
  }
  tile_copy<HT, false>(stile, const_cast<HT*>(H), r0, rows);
  __syncthreads();
  if (threadIdx.x < rows) {
    float o[16];
    unstage_row<HT>(stile, threadIdx.x, o);
    float* z = static_cast<float*>(colptr(zp));
    z[r0 + threadIdx.x] = decode_row(o, dw) * s_back;
  }
}

// ---------------------------------------------------------------- k_gconv_row
//
// Res-GCONV for matrices whose rows are all short (at most ROW_DMAX nonzeros: stencils,
// meshes).  A block of TILE threads owns RB = TILE / LPR consecutive rows.
//   gather: LPR lanes per row, lane p holding the row-vector quarter/half [p*PW, p*PW+PW)
//     (PW = 16 / LPR values).  Row pointers, column indices and values are loaded before
//     the programmatic-launch wait (the matrix is never written), so they overlap the
//     previous layer's tail; after the wait a lane loads its part of the block's own row
//     and of every neighbour row, DB neighbours in flight, and sums a_ij h_j in column
//     order.  No slot bookkeeping, no carries: each row is one lane group's.
//   epilogue: the parts of h_i and (A_hat H)_i meet in shared memory; thread t computes
//     outputs [q*PW, q*PW+PW) of row t % RB with q = t / RB, which is the same for a whole
//     warp, so the weights are uniform kernel-parameter loads; it writes them straight
//     out.  Each output's 16- or 32-term sum runs on paired float32 multiply-adds
//     (fma.rn.f32x2), the even inputs in one lane and the odd ones in the other, over a
//     transposed copy of U and W (LayerWT): half the multiply-add instructions.
//   decoder (last layer): the output parts meet in shared memory again and part q
//     evaluates decoder units [q*32/LPR, (q+1)*32/LPR); the parts add in order.
constexpr int ROW_DMAX = 16;

template <class HT, int LPR>
struct RowTraits;
template <>
struct RowTraits<float, 2> {  // 8 floats: two 16-byte loads
  static constexpr int PW = 8;
  __device__ __forceinline__ static void load(const float* X, int c, int p, float (&x)[8]) {
    const float4* s = reinterpret_cast<const float4*>(X + (size_t)c * 16 + 8 * p);
    const float4 a = __ldg(s), b = __ldg(s + 1);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
  }
  __device__ __forceinline__ static void store(float* Y, int r, int p, const float (&o)[8]) {
    float4* d = reinterpret_cast<float4*>(Y + (size_t)r * 16 + 8 * p);
    d[0] = make_float4(o[0], o[1], o[2], o[3]);
    d[1] = make_float4(o[4], o[5], o[6], o[7]);
  }
};
template <>
struct RowTraits<float, 4> {  // 4 floats: one 16-byte load
  static constexpr int PW = 4;
  __device__ __forceinline__ static void load(const float* X, int c, int p, float (&x)[4]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(X + (size_t)c * 16 + 4 * p));
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
  }
  __device__ __forceinline__ static void store(float* Y, int r, int p, const float (&o)[4]) {
    *reinterpret_cast<float4*>(Y + (size_t)r * 16 + 4 * p) = make_float4(o[0], o[1], o[2], o[3]);
  }
};
template <>
struct RowTraits<uint16_t, 2> {  // 8 bfloat16: one 16-byte load
  static constexpr int PW = 8;
  __device__ __forceinline__ static void load(const uint16_t* X, int c, int p, float (&x)[8]) {
    const uint4 t = __ldg(reinterpret_cast<const uint4*>(X + (size_t)c * 16 + 8 * p));
    x[0] = bf16lo(t.x); x[1] = bf16hi(t.x); x[2] = bf16lo(t.y); x[3] = bf16hi(t.y);
    x[4] = bf16lo(t.z); x[5] = bf16hi(t.z); x[6] = bf16lo(t.w); x[7] = bf16hi(t.w);
  }
  __device__ __forceinline__ static void store(uint16_t* Y, int r, int p, const float (&o)[8]) {
    *reinterpret_cast<uint4*>(Y + (size_t)r * 16 + 8 * p) =
        make_uint4(pack_bf16x2(o[0], o[1]), pack_bf16x2(o[2], o[3]), pack_bf16x2(o[4], o[5]),
                   pack_bf16x2(o[6], o[7]));
  }
};
template <>
struct RowTraits<uint16_t, 4> {  // 4 bfloat16: one 8-byte load
  static constexpr int PW = 4;
  __device__ __forceinline__ static void load(const uint16_t* X, int c, int p, float (&x)[4]) {
    const uint2 t = __ldg(reinterpret_cast<const uint2*>(X + (size_t)c * 16 + 4 * p));
    x[0] = bf16lo(t.x); x[1] = bf16hi(t.x); x[2] = bf16lo(t.y); x[3] = bf16hi(t.y);
  }
  __device__ __forceinline__ static void store(uint16_t* Y, int r, int p, const float (&o)[4]) {
    *reinterpret_cast<uint2*>(Y + (size_t)r * 16 + 4 * p) =
        make_uint2(pack_bf16x2(o[0], o[1]), pack_bf16x2(o[2], o[3]));
  }
};

constexpr int RSTR = 20;  // shared row stride in floats (conflict-free 16-byte accesses)

template <int LPR>
struct RowSmem {
  static constexpr int RB = TILE / LPR;
  __align__(16) float h[RB * RSTR];
  __align__(16) float agg[RB * RSTR];
  float zpart[LPR][RB];
};

// Gather into shared memory: part p of h_i and of (A_hat H)_i for the block's rows.
// Before the call the caller has loaded rs / deg / c / v (first DB entries) of its row.
//
// K systems at once (K > 1): r is the pair (node r / K, system r % K) of an [n K, 16]
// hidden block, the CSR row is the node's and neighbour c of the pair is row c K + s.
template <class HT, int LPR, int DB, int K = 1>
__device__ __forceinline__ void row_gather(RowSmem<LPR>& sm, const int* __restrict__ col,
                                           const float* __restrict__ valhat, const HT* __restrict__ Hin,
                                           int r, int gr, int p, int rs, int deg, const int (&c0)[DB],
                                           const float (&v0)[DB]) {
  const int sys = K > 1 ? r % K : 0;
  using RT = RowTraits<HT, LPR>;
  constexpr int PW = RT::PW;
  float acc[PW], hv[PW];
#pragma unroll
  for (int k = 0; k < PW; ++k) acc[k] = 0.0f;
  if (deg >= 0) {
    RT::load(Hin, r, p, hv);
    float x[DB][PW];
#pragma unroll
    for (int k = 0; k < DB; ++k)
      if (k < deg) RT::load(Hin, c0[k] * K + sys, p, x[k]);
#pragma unroll
    for (int k = 0; k < DB; ++k)
      if (k < deg) {
#pragma unroll
        for (int i = 0; i < PW; ++i) acc[i] = fmaf(v0[k], x[k][i], acc[i]);
      }
    for (int e0 = DB; e0 < deg; e0 += DB) {  // rows longer than DB: further batches
      int c[DB];
      float v[DB];
#pragma unroll
      for (int k = 0; k < DB; ++k) {
        c[k] = (e0 + k < deg) ? __ldg(col + rs + e0 + k) : 0;
        v[k] = (e0 + k < deg) ? __ldg(valhat + rs + e0 + k) : 0.0f;
      }
#pragma unroll
      for (int k = 0; k < DB; ++k)
        if (e0 + k < deg) RT::load(Hin, c[k] * K + sys, p, x[k]);
#pragma unroll
      for (int k = 0; k < DB; ++k)
        if (e0 + k < deg) {
#pragma unroll
          for (int i = 0; i < PW; ++i) acc[i] = fmaf(v[k], x[k][i], acc[i]);
        }
    }
#pragma unroll
    for (int q = 0; q < PW / 4; ++q) {
      reinterpret_cast<float4*>(sm.h + gr * RSTR + p * PW)[q] =
          make_float4(hv[4 * q], hv[4 * q + 1], hv[4 * q + 2], hv[4 * q + 3]);
      reinterpret_cast<float4*>(sm.agg + gr * RSTR + p * PW)[q] =
          make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
  }
}

// Row pointers and the first DB column indices / values of this lane's row.
// (K > 1: r is a pair of the K-system block and n the number of pairs; the row is node r / K.)
template <int DB, int K = 1>
__device__ __forceinline__ void row_prefetch(const int* __restrict__ rp, const int* __restrict__ col,
                                             const float* __restrict__ valhat, int r, int n, int& rs,
                                             int& deg, int (&c)[DB], float (&v)[DB]) {
  rs = 0;
  deg = -1;  // no row
  if (r < n) {
    const int node = K > 1 ? r / K : r;
    rs = __ldg(rp + node);
    deg = __ldg(rp + node + 1) - rs;
  }
#pragma unroll
  for (int k = 0; k < DB; ++k) {
    c[k] = (k < deg) ? __ldg(col + rs + k) : 0;
    v[k] = (k < deg) ? __ldg(valhat + rs + k) : 0.0f;
  }
}

// sum_c x_c M[c][k] for one output k, x from 16 shared floats, MT the transposed weights
// (MT[k*16 + c]): the even and the odd inputs accumulate in the two lanes of a paired
// multiply-add and meet at the end.
__device__ __forceinline__ void dot16_pairs(const float* __restrict__ xrow, const float* mt, float& se, float& so) {
  const float4* xp = reinterpret_cast<const float4*>(xrow);
#pragma unroll
  for (int c4 = 0; c4 < 4; ++c4) {
    const float4 x = xp[c4];
    ffma2(se, so, x.x, x.y, mt[4 * c4], mt[4 * c4 + 1]);
    ffma2(se, so, x.z, x.w, mt[4 * c4 + 2], mt[4 * c4 + 3]);
  }
}

// Outputs [Q*PW, Q*PW+PW) of epilogue row er (h and agg from shared memory):
// ReLU(h U + agg W) or h + ReLU(agg W), each output's sum split over even and odd inputs.
template <int FORM, int LPR, int Q>
__device__ __forceinline__ void row_layer(const RowSmem<LPR>& sm, int er, const LayerWT& lw,
                                          float (&o)[16 / LPR]) {
  constexpr int PW = 16 / LPR, K0 = Q * PW;
  const float* ar = sm.agg + er * RSTR;
  const float* hr = sm.h + er * RSTR;
#pragma unroll
  for (int k = 0; k < PW; ++k) {
    float se = 0.0f, so = 0.0f;
    dot16_pairs(ar, lw.WT + (K0 + k) * 16, se, so);
    if (FORM == GNP_LAYER_PAPER) {
      dot16_pairs(hr, lw.UT + (K0 + k) * 16, se, so);
      o[k] = fmaxf(se + so, 0.0f);
    } else {
      o[k] = hr[K0 + k] + fmaxf(se + so, 0.0f);
    }
  }
}

// Decoder units [K0, K0+KU) of one row (o in shared memory): sum_k w2_k ReLU(b1_k + o D1[:, k]).
template <int K0, int KU>
__device__ __forceinline__ float decode_part_pairs(const float* orow, const DecWT& dw) {
  float ze = 0.0f, zo = 0.0f;
#pragma unroll
  for (int k = K0; k < K0 + KU; k += 2) {
    float ae = 0.0f, ao = 0.0f, be = 0.0f, bo = 0.0f;
    dot16_pairs(orow, dw.DT1 + k * 16, ae, ao);
    dot16_pairs(orow, dw.DT1 + (k + 1) * 16, be, bo);
    const float a0 = fmaxf(dw.b1[k] + (ae + ao), 0.0f);
    const float a1 = fmaxf(dw.b1[k + 1] + (be + bo), 0.0f);
    ffma2(ze, zo, a0, a1, dw.W2[k], dw.W2[k + 1]);
  }
  return ze + zo;
}

template <int FORM, int LPR>
__device__ __forceinline__ void row_layer_q(const RowSmem<LPR>& sm, int er, int q, const LayerWT& lw,
                                            float (&o)[16 / LPR]) {
  if constexpr (LPR == 2) {
    if (q == 0) row_layer<FORM, 2, 0>(sm, er, lw, o);
    else row_layer<FORM, 2, 1>(sm, er, lw, o);
  } else {
    if (q == 0) row_layer<FORM, 4, 0>(sm, er, lw, o);
    else if (q == 1) row_layer<FORM, 4, 1>(sm, er, lw, o);
    else if (q == 2) row_layer<FORM, 4, 2>(sm, er, lw, o);
    else row_layer<FORM, 4, 3>(sm, er, lw, o);
  }
}

// Resident blocks per SM the short-row kernels are compiled for.  Capping the registers
// for more resident blocks (six per SM at four lanes per row: 40 registers instead of 48)
// measured slower.
template <int LPR> struct RowBounds { static constexpr int MIN_BLOCKS = 1; };

template <class HT, int FORM, int LPR, int DB, int K = 1>
__device__ __forceinline__ void gconv_row_body(VGrid gb, const int* __restrict__ rp, const int* __restrict__ col,
                                               const float* __restrict__ valhat, const HT* __restrict__ Hin,
                                               HT* __restrict__ Hout, int n, const int* __restrict__ ctl,
                                               const LayerWT& lw) {
  constexpr int RB = TILE / LPR;
  __shared__ RowSmem<LPR> sm;
  const int t = threadIdx.x;
  const int r0 = gb.bid * RB;
  const int gr = t / LPR, p = t % LPR;
  int rs, deg, c[DB];
  float v[DB];
  row_prefetch<DB, K>(rp, col, valhat, r0 + gr, n, rs, deg, c, v);
  pdl_wait();
  if (ctl && !ctl[1]) return;
  row_gather<HT, LPR, DB, K>(sm, col, valhat, Hin, r0 + gr, gr, p, rs, deg, c, v);
  __syncthreads();
  const int er = t % RB, q = t / RB;
  float o[16 / LPR];
  if (r0 + er < n) row_layer_q<FORM, LPR>(sm, er, q, lw, o);
  pdl_release();
  if (r0 + er < n) RowTraits<HT, LPR>::store(Hout, r0 + er, q, o);
}

template <class HT, int FORM, int LPR, int DB, int K = 1>
__global__ void __launch_bounds__(TILE, RowBounds<LPR>::MIN_BLOCKS)
k_gconv_row(const int* __restrict__ rp, const int* __restrict__ col, const float* __restrict__ valhat,
            const HT* __restrict__ Hin, HT* __restrict__ Hout, int n, const int* __restrict__ ctl,
            const __grid_constant__ LayerWT lw) {
  gconv_row_body<HT, FORM, LPR, DB, K>(hw_grid(), rp, col, valhat, Hin, Hout, n, ctl, lw);
}

template <class HT, int FORM, int LPR, int DB, int K = 1>
__device__ __forceinline__ void gconv_row_dec_body(VGrid gb, const int* __restrict__ rp, const int* __restrict__ col,
                                                   const float* __restrict__ valhat, const HT* __restrict__ Hin,
                                                   ColPtr zp, const double* __restrict__ tau, double sqrt_n, int n,
                                                   const int* __restrict__ ctl, const LayerWT& lw, const DecWT& dw) {
  constexpr int RB = TILE / LPR;
  constexpr int PW = 16 / LPR;
  __shared__ RowSmem<LPR> sm;
  const int t = threadIdx.x;
  const int r0 = gb.bid * RB;
  const int gr = t / LPR, p = t % LPR;
  int rs, deg, c[DB];
  float v[DB];
  row_prefetch<DB, K>(rp, col, valhat, r0 + gr, n, rs, deg, c, v);
  pdl_wait();
  if (ctl && !ctl[1]) return;
  __shared__ float s_back;
  if (t == 0) {  // once per block: a float64 division is slow on GB300
    const double tv = *tau;
    s_back = (float)(tv > 0.0 ? tv / sqrt_n : 0.0);
  }
  row_gather<HT, LPR, DB, K>(sm, col, valhat, Hin, r0 + gr, gr, p, rs, deg, c, v);
  __syncthreads();
  const int er = t % RB, q = t / RB;
  const bool valid = r0 + er < n;
  float o[PW];
  if (valid) row_layer_q<FORM, LPR>(sm, er, q, lw, o);
  __syncthreads();  // every thread is done with h and agg
  if (valid) {
#pragma unroll
    for (int k = 0; k < PW / 4; ++k)
      reinterpret_cast<float4*>(sm.agg + er * RSTR + q * PW)[k] =
          make_float4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
  }
  __syncthreads();
  if (valid) {
    const float* orow = sm.agg + er * RSTR;
    float part;
    if constexpr (LPR == 2) {
      part = q == 0 ? decode_part_pairs<0, 16>(orow, dw) : decode_part_pairs<16, 16>(orow, dw);
    } else {
      part = q == 0 ? decode_part_pairs<0, 8>(orow, dw)
                    : q == 1 ? decode_part_pairs<8, 8>(orow, dw)
                             : q == 2 ? decode_part_pairs<16, 8>(orow, dw) : decode_part_pairs<24, 8>(orow, dw);
    }
    sm.zpart[q][er] = part;
  }
  __syncthreads();
  if (q == 0 && valid) {
    float zz = dw.b2;
#pragma unroll
    for (int k = 0; k < LPR; ++k) zz += sm.zpart[k][er];
    static_cast<float*>(colptr(zp))[r0 + er] = zz * s_back;
  }
}

template <class HT, int FORM, int LPR, int DB, int K = 1>
__global__ void __launch_bounds__(TILE, RowBounds<LPR>::MIN_BLOCKS)
k_gconv_row_dec(const int* __restrict__ rp, const int* __restrict__ col, const float* __restrict__ valhat,
                const HT* __restrict__ Hin, ColPtr zp, const double* __restrict__ tau, double sqrt_n, int n,
                const int* __restrict__ ctl, const __grid_constant__ LayerWT lw, const __grid_constant__ DecWT dw) {
  gconv_row_dec_body<HT, FORM, LPR, DB, K>(hw_grid(), rp, col, valhat, Hin, zp, tau, sqrt_n, n, ctl, lw, dw);
}

template <class HT>
__global__ void k_hidden_to_f32(const HT* __restrict__ H, float* __restrict__ out, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    if constexpr (sizeof(HT) == 4) out[i] = H[i];
    else out[i] = __uint_as_float(((uint32_t)H[i]) << 16);
  }
}

// ---------------------------------------------------------------- grouped GNP (serving)
//
// The encoder, layer and decoder-fused layer bodies for up to GW requests in one launch
// (work table: each request's stand-alone grid).  Each request's weights travel in the
// kernel parameters; a switch on the entry index hands the body that request's copy at a
// constant offset, so the epilogues read constant-bank operands as the stand-alone
// kernels do (six inlined copies of each body).
static_assert(GW == 6, "GNP_GW_SWITCH has six cases");
#define GNP_GW_SWITCH(i, CALL) \
  switch (i) {                 \
    case 0: CALL(0); break;    \
    case 1: CALL(1); break;    \
    case 2: CALL(2); break;    \
    case 3: CALL(3); break;    \
    case 4: CALL(4); break;    \
    default: CALL(5); break;   \
  }

struct GEncP {
  GTable t;
  const GSlot* sl;
  EncW w[GW];
};
struct GLayerP {
  GTable t;
  const GSlot* sl;
  int l;
  LayerWT w[GW];
};
struct GDecP {
  GTable t;
  const GSlot* sl;
  LayerWT lw[GW];
  DecWT dw[GW];
};

// A request's grid here is its stand-alone encoder grid plus one block (k_encode_vn's); its
// block 0 also advances the request's phase (GCtl), which no other kernel of the round
// writes and which the cycle-end kernels read later in the round.  At a
// cycle's first step (st->fresh: k_residual just restarted it) the request runs k_encode's
// body, v_0 = r / beta, on the first nt blocks and the extra block returns; later steps
// run k_encode_vn's body (v_j formed from step j-1's passes, whose Givens update the extra
// block does; after step m-1 that update ends the cycle).
template <class HT>
__global__ void __launch_bounds__(TILE) kg_encode(const __grid_constant__ GEncP P) {
  VGrid g;
  const int i = gt_entry(P.t, g);
  const GSlot& d = P.sl[P.t.slot[i]];
  HT* H0 = static_cast<HT*>(d.Hh[0]);
  const int* ctl = reinterpret_cast<const int*>(d.st);
  if (g.bid == 0 && threadIdx.x == 0) d.gc->phase = d.gc->phase >= d.m ? 0 : d.gc->phase + 1;  // the round
  if (d.st->fresh) {
    if (g.bid == g.nblk - 1) return;
    const VGrid ge{g.bid, g.nblk - 1};
    const ColPtr v{d.V, sizeof(double) * (size_t)d.n, ctl, 0};
#define GNP_ENC0(k) encode_body<HT>(ge, v, &d.st->vscale, d.tau, ctl, d.n, d.sqrt_n, d.noscale, H0, P.w[k])
    GNP_GW_SWITCH(i, GNP_ENC0)
#undef GNP_ENC0
  } else {
    const VNext vn{d.V, d.w, d.h1, d.h2, d.st, d.Hb, d.R, d.cs, d.sn, d.g, d.hist, d.thist, d.hf, 0};
#define GNP_ENC1(k) encode_vn_body<HT>(g, vn, d.n, d.sqrt_n, d.noscale, d.tau, H0, P.w[k])
    GNP_GW_SWITCH(i, GNP_ENC1)
#undef GNP_ENC1
  }
}

// Layer P.l (< L - 1) of each request: Hh[l % 2] -> Hh[(l + 1) % 2].
template <class HT, int FORM>
__global__ void __launch_bounds__(TILE, RowBounds<4>::MIN_BLOCKS) kg_gconv_row(const __grid_constant__ GLayerP P) {
  VGrid g;
  const int i = gt_entry(P.t, g);
  const GSlot& d = P.sl[P.t.slot[i]];
  const HT* Hin = static_cast<const HT*>(d.Hh[P.l & 1]);
  HT* Hout = static_cast<HT*>(d.Hh[(P.l + 1) & 1]);
  const int* ctl = reinterpret_cast<const int*>(d.st);
#define GNP_LAY(k) gconv_row_body<HT, FORM, 4, 5>(g, d.rp, d.col, d.valhat, Hin, Hout, d.n, ctl, P.w[k])
  GNP_GW_SWITCH(i, GNP_LAY)
#undef GNP_LAY
}

// The decoder-fused last layer of each request: Hh[(L - 1) % 2] -> z_j.
template <class HT, int FORM>
__global__ void __launch_bounds__(TILE, RowBounds<4>::MIN_BLOCKS) kg_gconv_row_dec(const __grid_constant__ GDecP P) {
  VGrid g;
  const int i = gt_entry(P.t, g);
  const GSlot& d = P.sl[P.t.slot[i]];
  const HT* Hin = static_cast<const HT*>(d.Hh[(d.L - 1) & 1]);
  const int* ctl = reinterpret_cast<const int*>(d.st);
  const ColPtr z{d.Z, sizeof(float) * (size_t)d.n, ctl, 0};
#define GNP_DEC(k) \
  gconv_row_dec_body<HT, FORM, 4, 5>(g, d.rp, d.col, d.valhat, Hin, z, d.tau, d.sqrt_n, d.n, ctl, P.lw[k], P.dw[k])
  GNP_GW_SWITCH(i, GNP_DEC)
#undef GNP_DEC
}

// ---------------------------------------------------------------- host side

void fill_enc_dec(const std::vector<float>& w, int L, EncW& ew, DecW& dw) {
  memcpy(ew.W1, w.data() + ENC_W1, sizeof(ew.W1));
  memcpy(ew.b1, w.data() + ENC_B1, sizeof(ew.b1));
  memcpy(ew.W2, w.data() + ENC_W2, sizeof(ew.W2));
  memcpy(ew.b2, w.data() + ENC_B2, sizeof(ew.b2));
  const float* d = w.data() + dec_off(L);
  memcpy(dw.W1, d, sizeof(dw.W1));
  memcpy(dw.b1, d + 512, sizeof(dw.b1));
  memcpy(dw.W2, d + 544, sizeof(dw.W2));
  dw.b2 = d[576];
}

void fill_layer_wt(const std::vector<float>& w, int l, LayerWT& lw) {
  const float* p = w.data() + layer_off(l);
  for (int c = 0; c < 16; ++c)
    for (int k = 0; k < 16; ++k) {
      lw.UT[k * 16 + c] = p[c * 16 + k];
      lw.WT[k * 16 + c] = p[256 + c * 16 + k];
    }
}

void fill_dec_wt(const std::vector<float>& w, int L, DecWT& dw) {
  const float* d = w.data() + dec_off(L);
  for (int c = 0; c < 16; ++c)
    for (int k = 0; k < 32; ++k) dw.DT1[k * 16 + c] = d[c * 32 + k];
  memcpy(dw.b1, d + 512, sizeof(dw.b1));
  memcpy(dw.W2, d + 544, sizeof(dw.W2));
  dw.b2 = d[576];
}

void fill_layer_w(const std::vector<float>& w, int l, LayerW& lw) {
  const float* p = w.data() + layer_off(l);
  memcpy(lw.U, p, sizeof(lw.U));
  memcpy(lw.W, p + 256, sizeof(lw.W));
}

// Neighbour rows in flight per lane in the tile kernels' gather: 8 for float32 hidden
// rows, 4 for bfloat16 (8 rows of 8 values would spill); GNP_GCONV_GROUP=4|8 in the
// environment forces one (for tuning).
static int env_int(const char* name, int dflt) {
  const char* e = getenv(name);
  return e ? atoi(e) : dflt;
}

template <class HT>
static int gconv_group() {
  const int g = env_int("GNP_GCONV_GROUP", sizeof(HT) == 4 ? 8 : 4);
  return g == 4 ? 4 : 8;
}

template <class HT, int FORM, int ROWS>
static int set_attr_all(cudaFuncAttribute attr, int value) {
  GNP_TRY_CUDA(cudaFuncSetAttribute(k_gconv<HT, FORM, ROWS, 4>, attr, value));
  GNP_TRY_CUDA(cudaFuncSetAttribute(k_gconv_dec<HT, FORM, ROWS, 4>, attr, value));
  GNP_TRY_CUDA(cudaFuncSetAttribute(k_gconv<HT, FORM, ROWS, 8>, attr, value));
  GNP_TRY_CUDA(cudaFuncSetAttribute(k_gconv_dec<HT, FORM, ROWS, 8>, attr, value));
  return GNP_OK;
}

template <class HT, int FORM, int ROWS>
static int set_smem_attrs() {
  static bool done = false;
  if (done) return GNP_OK;
  const int bytes = (int)sizeof(GconvSmem<HT, ROWS>);
  GNP_TRY((set_attr_all<HT, FORM, ROWS>(cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)));
  done = true;
  return GNP_OK;
}

// Rows per Res-GCONV tile: 256-row tiles (one epilogue thread per row) at three
// resident blocks per SM were the fastest shape for both hidden-block precisions on both
// the 65,536-row and the 2^20-row workloads; 128-row tiles (two threads per row) are kept
// for tuning.  GNP_GCONV_ROWS=128|256 in the environment forces one.
template <class HT>
static int gconv_rows() {
  const int forced = env_int("GNP_GCONV_ROWS", 0);
  if (forced == 128 || forced == 256) return forced;
  return 256;
}

// Resident Res-GCONV blocks per SM.  The shared memory the blocks take comes out of the
// same 256 KB per SM as the L1 cache that serves the neighbour-row gathers, so the
// carveout is set to fit exactly this many blocks (more blocks, less L1).
// GNP_GCONV_BLOCKS=1..8 in the environment overrides it (for tuning).
template <class HT, int ROWS>
static int gconv_blocks() {
  const int forced = env_int("GNP_GCONV_BLOCKS", 0);
  if (forced >= 1 && forced <= 8) return forced;
  return ROWS == 256 ? 3 : 4;
}

// Rows per tile (at most ROWS): for float32 hidden blocks, n spread evenly over every
// resident block slot (152 SMs x gconv_blocks), so that no SM holds more rows than another
// and small systems still fill every slot (65,536 rows: 144-row tiles, 456 blocks, instead
// of 256 tiles of 256 rows on 1-2 blocks per SM); large systems use full ROWS-row tiles.
// GNP_GCONV_TILE=32..ROWS in the environment forces the tile height (for tuning).
template <class HT, int ROWS>
static int gconv_tile_rows(int n) {
  const int forced = env_int("GNP_GCONV_TILE", 0);
  if (forced >= 32 && forced <= ROWS) return forced;
  // bfloat16 rows are 32 bytes: a 256-row tile's nonzeros already give its 128 slots short
  // chains, and shorter tiles measured slower (65,536 rows: 0.080 ms apply at 256 rows,
  // 0.088 ms at 144); float32 gains from the even spread (0.097 -> 0.092 ms)
  if (sizeof(HT) == 2) return ROWS;
  const long long slots = (long long)NUM_SMS_GB300 * gconv_blocks<HT, ROWS>();
  int t = (int)((n + slots - 1) / slots);
  t = (t + 7) & ~7;
  return std::max(32, std::min(ROWS, t));
}

template <class HT, int FORM, int ROWS>
static int set_carveout() {
  static int applied = -1;
  const int blocks = gconv_blocks<HT, ROWS>();
  const int per_block = (int)sizeof(GconvSmem<HT, ROWS>) + 1024;  // + the runtime's reserved 1 KB
  const int pct = std::min(100, (blocks * per_block * 100 + 228 * 1024 - 1) / (228 * 1024));
  if (pct == applied) return GNP_OK;
  GNP_TRY((set_attr_all<HT, FORM, ROWS>(cudaFuncAttributePreferredSharedMemoryCarveout, pct)));
  applied = pct;
  return GNP_OK;
}

template <class HT, int FORM>
static int set_smem_attrs_all() {
  GNP_TRY((set_smem_attrs<HT, FORM, 128>()));
  GNP_TRY((set_smem_attrs<HT, FORM, 256>()));
  GNP_TRY((set_carveout<HT, FORM, 128>()));
  GNP_TRY((set_carveout<HT, FORM, 256>()));
  return GNP_OK;
}


// Layers 0..L-1 (the last one fused with the decoder unless tracing), ROWS-row tiles,
// GROUP neighbour rows in flight per lane.
template <class HT, int FORM, int ROWS, int GROUP>
static int launch_layers_g(gnp_model* M, HT* H0, HT* H1, ColPtr z, float* trace, const int* ctl,
                         cudaStream_t st, cudaEvent_t* ev, const ApplyWs& W, const DecW& dw, double sqrt_n) {
  const gnp_mat* A = M->A;
  const int n = A->n, L = M->cfg.L;
  const int smem = (int)sizeof(GconvSmem<HT, ROWS>);
  const int trows = gconv_tile_rows<HT, ROWS>(n);
  const int ntg = (n + trows - 1) / trows;
  const long long hcount = (long long)n * 16;
  const int fused_last = (L > 0 && !trace) ? 1 : 0;
  const bool tma = tma_active(A);
  for (int l = 0; l < L - fused_last; ++l) {
    LayerW lw;
    fill_layer_w(M->w_host, l, lw);
    if (ev) GNP_TRY_CUDA(cudaEventRecordWithFlags(ev[2 * l], st, cudaEventRecordExternal));
    if (tma)
      GNP_TRY(tma_layer_launch<HT>(A, FORM, false, M->valhat, H0, H1, ColPtr{}, nullptr, sqrt_n, ctl, lw, dw, st));
    else
    GNP_TRY_CUDA(launch_pdl(k_gconv<HT, FORM, ROWS, GROUP>, ntg, smem, st, A->rp, A->col, (const float*)M->valhat,
                            (const HT*)H0, H1, n, trows, ctl, lw));
    if (ev) GNP_TRY_CUDA(cudaEventRecordWithFlags(ev[2 * l + 1], st, cudaEventRecordExternal));
    if (trace)
      k_hidden_to_f32<HT><<<4 * NUM_SMS_GB300, 256, 0, st>>>(H1, trace + (size_t)(l + 1) * hcount, hcount);
    std::swap(H0, H1);
  }
  if (fused_last) {
    LayerW lw;
    fill_layer_w(M->w_host, L - 1, lw);
    if (ev) GNP_TRY_CUDA(cudaEventRecordWithFlags(ev[2 * (L - 1)], st, cudaEventRecordExternal));
    if (tma)
      GNP_TRY(tma_layer_launch<HT>(A, FORM, true, M->valhat, H0, nullptr, z, W.tau, sqrt_n, ctl, lw, dw, st));
    else
    GNP_TRY_CUDA(launch_pdl(k_gconv_dec<HT, FORM, ROWS, GROUP>, ntg, smem, st, A->rp, A->col, (const float*)M->valhat,
                            (const HT*)H0, z, (const double*)W.tau, sqrt_n, n, trows, ctl, lw, dw));
    if (ev) GNP_TRY_CUDA(cudaEventRecordWithFlags(ev[2 * (L - 1) + 1], st, cudaEventRecordExternal));
  } else {
    k_decode<HT><<<(n + TILE - 1) / TILE, TILE, 0, st>>>(H0, z, W.tau, sqrt_n, n, ctl, dw);
  }
  return GNP_OK;
}

template <class HT, int FORM, int ROWS>
static int launch_layers(gnp_model* M, HT* H0, HT* H1, ColPtr z, float* trace, const int* ctl,
                         cudaStream_t st, cudaEvent_t* ev, const ApplyWs& W, const DecW& dw, double sqrt_n) {
  if (gconv_group<HT>() == 4)
    return launch_layers_g<HT, FORM, ROWS, 4>(M, H0, H1, z, trace, ctl, st, ev, W, dw, sqrt_n);
  return launch_layers_g<HT, FORM, ROWS, 8>(M, H0, H1, z, trace, ctl, st, ev, W, dw, sqrt_n);
}

// Layers 0..L-1 with the short-row kernels (RB = TILE / LPR rows per block).
template <class HT, int FORM, int LPR, int DB>
static int launch_layers_row(gnp_model* M, HT* H0, HT* H1, ColPtr z, float* trace, const int* ctl,
                             cudaStream_t st, cudaEvent_t* ev, const ApplyWs& W, const DecW& dw, double sqrt_n) {
  const gnp_mat* A = M->A;
  const int n = A->n, L = M->cfg.L;
  constexpr int RB = TILE / LPR;
  const int nb = (n + RB - 1) / RB;
  const long long hcount = (long long)n * 16;
  const int fused_last = (L > 0 && !trace) ? 1 : 0;
  for (int l = 0; l < L - fused_last; ++l) {
    LayerWT lw;
    fill_layer_wt(M->w_host, l, lw);
    if (ev) GNP_TRY_CUDA(cudaEventRecordWithFlags(ev[2 * l], st, cudaEventRecordExternal));
    GNP_TRY_CUDA(launch_pdl(k_gconv_row<HT, FORM, LPR, DB>, nb, 0, st, A->rp, A->col, (const float*)M->valhat,
                            (const HT*)H0, H1, n, ctl, lw));
    if (ev) GNP_TRY_CUDA(cudaEventRecordWithFlags(ev[2 * l + 1], st, cudaEventRecordExternal));
    if (trace)
      k_hidden_to_f32<HT><<<4 * NUM_SMS_GB300, 256, 0, st>>>(H1, trace + (size_t)(l + 1) * hcount, hcount);
    std::swap(H0, H1);
  }
  if (fused_last) {
    LayerWT lw;
    fill_layer_wt(M->w_host, L - 1, lw);
    DecWT dwt;
    fill_dec_wt(M->w_host, L, dwt);
    if (ev) GNP_TRY_CUDA(cudaEventRecordWithFlags(ev[2 * (L - 1)], st, cudaEventRecordExternal));
    GNP_TRY_CUDA(launch_pdl(k_gconv_row_dec<HT, FORM, LPR, DB>, nb, 0, st, A->rp, A->col,
                            (const float*)M->valhat, (const HT*)H0, z, (const double*)W.tau, sqrt_n, n, ctl, lw,
                            dwt));
    if (ev) GNP_TRY_CUDA(cudaEventRecordWithFlags(ev[2 * (L - 1) + 1], st, cudaEventRecordExternal));
  } else {
    k_decode<HT><<<(n + TILE - 1) / TILE, TILE, 0, st>>>(H0, z, W.tau, sqrt_n, n, ctl, dw);
  }
  return GNP_OK;
}

// Short-row kernels when every row has at most ROW_DMAX nonzeros (GNP_GCONV_ROWK=0 in the
// environment forces the tile kernels; GNP_ROW_LPR=2|4 sets the lanes per row and
// GNP_ROW_DB=4|5 the neighbour loads in flight, for tuning).  Five loads in flight cover a
// 5-point stencil row in one round trip (56 registers, four blocks per SM): 93.2 -> 89.7 us
// per FGMRES step at 65,536 rows against four (48 registers, five blocks); eight measured
// slower (more registers, fewer resident blocks).  Rows of at most four take four.
static int row_kernel_mode(const gnp_mat* A) {
  if (!env_int("GNP_GCONV_ROWK", 1) || A->max_deg > ROW_DMAX) return 0;
  const int forced = env_int("GNP_ROW_DB", 0);
  const int db = forced == 4 || forced == 5 ? forced : (A->max_deg <= 4 ? 4 : 5);
  return (env_int("GNP_ROW_LPR", 4) == 2 ? 20 : 40) + db;
}

// The L layers of the K-system GNP (multi-right-hand-side FGMRES) on the short-row
// kernels: the [n K, 16] float32 hidden block is a one-system block over n K pairs whose
// pair (i, s) gathers pairs (c, s); the last layer applies the decoder and writes
// z = column zp (pairs in node-major order), scaled by *tau_one / sqrt(n) = 1 / sqrt(n).
template <int FORM, int K>
static int multi_row_layers_k(gnp_model* M, float* H0, float* H1, ColPtr zp, const double* tau_one,
                              const int* ctl, cudaStream_t st) {
  const gnp_mat* A = M->A;
  const int L = M->cfg.L;
  const int np = A->n * K;
  constexpr int LPR = 4, DB = 5;
  constexpr int RB = TILE / LPR;
  const int nb = (np + RB - 1) / RB;
  const double sqrt_n = std::sqrt((double)A->n);
  for (int l = 0; l < L - 1; ++l) {
    LayerWT lw;
    fill_layer_wt(M->w_host, l, lw);
    GNP_TRY_CUDA(launch_pdl(k_gconv_row<float, FORM, LPR, DB, K>, nb, 0, st, A->rp, A->col,
                            (const float*)M->valhat, (const float*)H0, H1, np, ctl, lw));
    std::swap(H0, H1);
  }
  LayerWT lw;
  fill_layer_wt(M->w_host, L - 1, lw);
  DecWT dwt;
  fill_dec_wt(M->w_host, L, dwt);
  GNP_TRY_CUDA(launch_pdl(k_gconv_row_dec<float, FORM, LPR, DB, K>, nb, 0, st, A->rp, A->col,
                          (const float*)M->valhat, (const float*)H0, zp, tau_one, sqrt_n, np, ctl, lw, dwt));
  return GNP_OK;
}

bool multi_row_ok(const gnp_model* M) { return M->cfg.L >= 1 && row_kernel_mode(M->A) != 0; }

// ---------------------------------------------------------------- grouped GNP launches

bool grouped_ok(const gnp_model* M) { return M && M->cfg.L >= 1 && row_kernel_mode(M->A) / 10 == 4; }

std::vector<GTable> gt_build(const std::vector<std::pair<int, int>>& entries, int cap) {
  std::vector<GTable> out;
  for (size_t e0 = 0; e0 < entries.size(); e0 += (size_t)cap) {
    GTable t{};
    t.count = (int)std::min(entries.size() - e0, (size_t)cap);
    int b = 0;
    for (int k = 0; k < t.count; ++k) {
      t.slot[k] = entries[e0 + k].first;
      t.start[k] = b;
      b += entries[e0 + k].second;
    }
    t.start[t.count] = b;
    out.push_back(t);
  }
  return out;
}

template <class HT, int FORM>
static int grouped_apply_t(const std::vector<GHost>& reqs, const GSlot* d_slots, cudaStream_t st) {
  constexpr int RB = TILE / 4;
  const int R = (int)reqs.size();
  int Lmax = 0;
  for (const GHost& q : reqs) Lmax = std::max(Lmax, q.M->cfg.L);
  for (int c0 = 0; c0 < R; c0 += GW) {  // encoder
    const int c1 = std::min(R, c0 + GW);
    std::vector<std::pair<int, int>> e;
    for (int k = c0; k < c1; ++k) e.push_back({reqs[k].slot, (reqs[k].n + TILE - 1) / TILE + 1});
    GEncP P{};
    P.t = gt_build(e, GW)[0];
    P.sl = d_slots;
    for (int k = c0; k < c1; ++k) {
      DecW dw;
      fill_enc_dec(reqs[k].M->w_host, reqs[k].M->cfg.L, P.w[k - c0], dw);
    }
    kg_encode<HT><<<P.t.start[P.t.count], TILE, 0, st>>>(P);
  }
  for (int l = 0; l + 1 < Lmax; ++l) {  // layers before the last
    std::vector<const GHost*> sub;
    for (const GHost& q : reqs)
      if (l + 1 < q.M->cfg.L) sub.push_back(&q);
    for (size_t c0 = 0; c0 < sub.size(); c0 += GW) {
      const size_t c1 = std::min(sub.size(), c0 + GW);
      std::vector<std::pair<int, int>> e;
      for (size_t k = c0; k < c1; ++k) e.push_back({sub[k]->slot, (sub[k]->n + RB - 1) / RB});
      GLayerP P{};
      P.t = gt_build(e, GW)[0];
      P.sl = d_slots;
      P.l = l;
      for (size_t k = c0; k < c1; ++k) fill_layer_wt(sub[k]->M->w_host, l, P.w[k - c0]);
      GNP_TRY_CUDA(launch_pdl(kg_gconv_row<HT, FORM>, P.t.start[P.t.count], 0, st, P));
    }
  }
  for (int c0 = 0; c0 < R; c0 += GW) {  // decoder-fused last layer
    const int c1 = std::min(R, c0 + GW);
    std::vector<std::pair<int, int>> e;
    for (int k = c0; k < c1; ++k) e.push_back({reqs[k].slot, (reqs[k].n + RB - 1) / RB});
    GDecP P{};
    P.t = gt_build(e, GW)[0];
    P.sl = d_slots;
    for (int k = c0; k < c1; ++k) {
      const gnp_model* M = reqs[k].M;
      fill_layer_wt(M->w_host, M->cfg.L - 1, P.lw[k - c0]);
      fill_dec_wt(M->w_host, M->cfg.L, P.dw[k - c0]);
    }
    GNP_TRY_CUDA(launch_pdl(kg_gconv_row_dec<HT, FORM>, P.t.start[P.t.count], 0, st, P));
  }
  return check_launch("grouped GNP apply");
}

int grouped_apply_launch(const std::vector<GHost>& reqs, const GSlot* d_slots, cudaStream_t st) {
  if (reqs.empty()) return GNP_OK;
  const gnp_model* M = reqs[0].M;
  for (const GHost& q : reqs)
    GNP_REQUIRE(grouped_ok(q.M) && q.M->hprec == M->hprec && q.M->cfg.form == M->cfg.form,
                "grouped_apply_launch: requests of one launch need the short-row kernels and one hidden "
                "precision and layer form");
  const bool paper = M->cfg.form == GNP_LAYER_PAPER;
  if (M->hprec == GNP_H_BF16)
    return paper ? grouped_apply_t<uint16_t, GNP_LAYER_PAPER>(reqs, d_slots, st)
                 : grouped_apply_t<uint16_t, GNP_LAYER_RESID>(reqs, d_slots, st);
  return paper ? grouped_apply_t<float, GNP_LAYER_PAPER>(reqs, d_slots, st)
               : grouped_apply_t<float, GNP_LAYER_RESID>(reqs, d_slots, st);
}

int multi_row_layers(gnp_model* M, int K, float* H0, float* H1, ColPtr zp, const double* tau_one, const int* ctl,
                     cudaStream_t st) {
  const bool paper = M->cfg.form == GNP_LAYER_PAPER;
  switch (K) {
    case 2: return paper ? multi_row_layers_k<GNP_LAYER_PAPER, 2>(M, H0, H1, zp, tau_one, ctl, st)
                         : multi_row_layers_k<GNP_LAYER_RESID, 2>(M, H0, H1, zp, tau_one, ctl, st);
    case 4: return paper ? multi_row_layers_k<GNP_LAYER_PAPER, 4>(M, H0, H1, zp, tau_one, ctl, st)
                         : multi_row_layers_k<GNP_LAYER_RESID, 4>(M, H0, H1, zp, tau_one, ctl, st);
    case 8: return paper ? multi_row_layers_k<GNP_LAYER_PAPER, 8>(M, H0, H1, zp, tau_one, ctl, st)
                         : multi_row_layers_k<GNP_LAYER_RESID, 8>(M, H0, H1, zp, tau_one, ctl, st);
    default:
      set_error("multi_row_layers: K = %d", K);
      return GNP_ERR_INVALID_ARG;
  }
}

// One Res-GCONV layer l on caller buffers, with the kernel the apply runs for its
// layers before the last (gnp_layer_apply).
template <class HT, int FORM, int LPR, int DB>
static int layer_row_one(gnp_model* M, int l, const HT* Hin, HT* Hout, cudaStream_t st) {
  constexpr int RB = TILE / LPR;
  const gnp_mat* A = M->A;
  LayerWT lw;
  fill_layer_wt(M->w_host, l, lw);
  GNP_TRY_CUDA(launch_pdl(k_gconv_row<HT, FORM, LPR, DB>, (A->n + RB - 1) / RB, 0, st, A->rp, A->col,
                          (const float*)M->valhat, Hin, Hout, A->n, (const int*)nullptr, lw));
  return GNP_OK;
}

template <class HT, int FORM, int ROWS, int GROUP>
static int layer_tile_one(gnp_model* M, int l, const HT* Hin, HT* Hout, cudaStream_t st) {
  const gnp_mat* A = M->A;
  const int n = A->n;
  const int trows = gconv_tile_rows<HT, ROWS>(n);
  LayerW lw;
  fill_layer_w(M->w_host, l, lw);
  if (tma_active(A)) {
    DecW dw;
    return tma_layer_launch<HT>(A, FORM, false, M->valhat, Hin, Hout, ColPtr{}, nullptr, 0.0, nullptr, lw, dw, st);
  }
  GNP_TRY_CUDA(launch_pdl(k_gconv<HT, FORM, ROWS, GROUP>, (n + trows - 1) / trows, (int)sizeof(GconvSmem<HT, ROWS>),
                          st, A->rp, A->col, (const float*)M->valhat, Hin, Hout, n, trows, (const int*)nullptr, lw));
  return GNP_OK;
}

template <class HT, int FORM>
static int layer_impl(gnp_model* M, int l, const HT* Hin, HT* Hout, cudaStream_t st) {
  GNP_TRY((set_smem_attrs_all<HT, FORM>()));
  switch (row_kernel_mode(M->A)) {
    case 24: GNP_TRY((layer_row_one<HT, FORM, 2, 4>(M, l, Hin, Hout, st))); break;
    case 25: GNP_TRY((layer_row_one<HT, FORM, 2, 5>(M, l, Hin, Hout, st))); break;
    case 44: GNP_TRY((layer_row_one<HT, FORM, 4, 4>(M, l, Hin, Hout, st))); break;
    case 45: GNP_TRY((layer_row_one<HT, FORM, 4, 5>(M, l, Hin, Hout, st))); break;
    default: {
      const bool g4 = gconv_group<HT>() == 4;
      if (gconv_rows<HT>() == 128) {
        GNP_TRY(g4 ? (layer_tile_one<HT, FORM, 128, 4>(M, l, Hin, Hout, st))
                   : (layer_tile_one<HT, FORM, 128, 8>(M, l, Hin, Hout, st)));
      } else {
        GNP_TRY(g4 ? (layer_tile_one<HT, FORM, 256, 4>(M, l, Hin, Hout, st))
                   : (layer_tile_one<HT, FORM, 256, 8>(M, l, Hin, Hout, st)));
      }
    }
  }
  return check_launch("gnp_layer_apply");
}

template <class HT, int FORM>
static int apply_impl(gnp_model* M, ColPtr v, const double* vscale, ColPtr z, float* trace,
                      const int* ctl, cudaStream_t st, cudaEvent_t* ev, const ApplyWs& W, const VNext* vn,
                      cudaEvent_t fork, cudaStream_t side) {
  const gnp_mat* A = M->A;
  const int n = A->n, L = M->cfg.L;
  const double sqrt_n = std::sqrt((double)n);
  GNP_TRY((set_smem_attrs_all<HT, FORM>()));
  const int nt = (n + TILE - 1) / TILE;
  const int nb = red_blocks(n);
  const int noscale = M->cfg.no_scale ? 1 : 0;
  if (!vscale && !noscale && !vn)
    k_vnorm<<<nb, RED_THREADS, 0, st>>>(v, ctl, n, W.red.partials, W.red.counter, W.tau);
  EncW ew;
  DecW dw;
  fill_enc_dec(M->w_host, L, ew, dw);
  HT* H0 = static_cast<HT*>(W.H[0]);
  HT* H1 = static_cast<HT*>(W.H[1]);
  if (vn && vn->dcgs) k_encode_dv<HT><<<nt, TILE, 0, st>>>(*vn, n, sqrt_n, noscale, W.tau, H0, ew);
  else if (vn) k_encode_vn<HT><<<nt + 1, TILE, 0, st>>>(*vn, n, sqrt_n, noscale, W.tau, H0, ew);
  else k_encode<HT><<<nt, TILE, 0, st>>>(v, vscale, W.tau, ctl, n, sqrt_n, noscale, H0, ew);
  if (fork) {
    GNP_TRY_CUDA(cudaEventRecord(fork, st));
    GNP_TRY_CUDA(cudaStreamWaitEvent(side, fork, 0));
  }
  if (trace) k_hidden_to_f32<HT><<<4 * NUM_SMS_GB300, 256, 0, st>>>(H0, trace, (long long)n * 16);
  switch (row_kernel_mode(A)) {
    case 24: GNP_TRY((launch_layers_row<HT, FORM, 2, 4>(M, H0, H1, z, trace, ctl, st, ev, W, dw, sqrt_n))); break;
    case 25: GNP_TRY((launch_layers_row<HT, FORM, 2, 5>(M, H0, H1, z, trace, ctl, st, ev, W, dw, sqrt_n))); break;
    case 44: GNP_TRY((launch_layers_row<HT, FORM, 4, 4>(M, H0, H1, z, trace, ctl, st, ev, W, dw, sqrt_n))); break;
    case 45: GNP_TRY((launch_layers_row<HT, FORM, 4, 5>(M, H0, H1, z, trace, ctl, st, ev, W, dw, sqrt_n))); break;
    default:
      if (gconv_rows<HT>() == 128)
        GNP_TRY((launch_layers<HT, FORM, 128>(M, H0, H1, z, trace, ctl, st, ev, W, dw, sqrt_n)));
      else
        GNP_TRY((launch_layers<HT, FORM, 256>(M, H0, H1, z, trace, ctl, st, ev, W, dw, sqrt_n)));
  }
  return check_launch("gnp apply");
}

int apply_launch(gnp_model* M, ColPtr v, const double* vscale, ColPtr z, float* trace,
                 const int* ctl, cudaStream_t st, cudaEvent_t* ev, const ApplyWs* ws, const VNext* vn,
                 cudaEvent_t fork, cudaStream_t side) {
  GNP_TRY(model_sync_host(M));
  const ApplyWs& W = ws ? *ws : M->ws;
  const int form = M->cfg.form;
  if (M->hprec == GNP_H_BF16) {
    return form == GNP_LAYER_PAPER
               ? apply_impl<uint16_t, GNP_LAYER_PAPER>(M, v, vscale, z, trace, ctl, st, ev, W, vn, fork, side)
               : apply_impl<uint16_t, GNP_LAYER_RESID>(M, v, vscale, z, trace, ctl, st, ev, W, vn, fork, side);
  }
  return form == GNP_LAYER_PAPER
             ? apply_impl<float, GNP_LAYER_PAPER>(M, v, vscale, z, trace, ctl, st, ev, W, vn, fork, side)
             : apply_impl<float, GNP_LAYER_RESID>(M, v, vscale, z, trace, ctl, st, ev, W, vn, fork, side);
}

int apply_ws_alloc(ApplyWs& ws, int n) {
  GNP_TRY(dev_alloc(reinterpret_cast<float**>(&ws.H[0]), (size_t)n * 16));
  GNP_TRY(dev_alloc(reinterpret_cast<float**>(&ws.H[1]), (size_t)n * 16));
  GNP_TRY(dev_alloc(&ws.tau, 2));
  GNP_TRY(red_alloc(ws.red, 4 * NUM_SMS_GB300, 1));
  return GNP_OK;
}

void apply_ws_free(ApplyWs& ws) {
  float* h0 = static_cast<float*>(ws.H[0]);
  float* h1 = static_cast<float*>(ws.H[1]);
  dev_free(h0);
  dev_free(h1);
  ws.H[0] = ws.H[1] = nullptr;
  dev_free(ws.tau);
  red_free(ws.red);
}

int apply_prepare(gnp_model* M) {
  GNP_TRY(model_sync_host(M));
  if (row_kernel_mode(M->A) == 0) GNP_TRY(tma_prepare(M->A));
  if (M->hprec == GNP_H_BF16) {
    if (M->cfg.form == GNP_LAYER_PAPER) GNP_TRY((set_smem_attrs_all<uint16_t, GNP_LAYER_PAPER>()));
    else GNP_TRY((set_smem_attrs_all<uint16_t, GNP_LAYER_RESID>()));
  } else {
    if (M->cfg.form == GNP_LAYER_PAPER) GNP_TRY((set_smem_attrs_all<float, GNP_LAYER_PAPER>()));
    else GNP_TRY((set_smem_attrs_all<float, GNP_LAYER_RESID>()));
  }
  return GNP_OK;
}

unsigned long long model_version(const gnp_model* M) { return M->version; }

int model_sync_host(gnp_model* M) {
  if (!M->host_stale) return GNP_OK;
  GNP_TRY_CUDA(cudaMemcpy(M->w_host.data(), M->w_best, sizeof(float) * M->w_host.size(),
                          cudaMemcpyDeviceToHost));
  M->host_stale = false;
  return GNP_OK;
}

}  // namespace gnp

using namespace gnp;

extern "C" {

int gnp_create(const gnp_mat* Ac, const gnp_config* cfg, const float* weights_host, gnp_model** out) {
  GNP_REQUIRE(out != nullptr, "gnp_create: out is null");
  *out = nullptr;
  GNP_REQUIRE(Ac && cfg && weights_host, "gnp_create: null argument");
  GNP_REQUIRE(cfg->L >= 0 && cfg->L <= GNP_MAX_LAYERS, "gnp_create: L = %d out of range", cfg->L);
  GNP_REQUIRE(cfg->form == GNP_LAYER_PAPER || cfg->form == GNP_LAYER_RESID, "gnp_create: bad form");
  GNP_REQUIRE(cfg->hprec == GNP_H_FP32 || cfg->hprec == GNP_H_BF16, "gnp_create: bad hprec");
  GNP_REQUIRE(cfg->sample_mode >= 0 && cfg->sample_mode <= 2, "gnp_create: sample_mode %d", cfg->sample_mode);
  GNP_REQUIRE(cfg->no_scale == 0 || cfg->no_scale == 1, "gnp_create: no_scale %d", cfg->no_scale);
  gnp_mat* A = const_cast<gnp_mat*>(Ac);
  gnp_model* M = new gnp_model();
  M->A = A;
  M->cfg = *cfg;
  M->hprec = cfg->hprec;
  const int cnt = weight_count(cfg->L);
  M->w_host.assign(weights_host, weights_host + cnt);
  int s = GNP_OK;
  const int n = A->n;
  const long long nnz = A->nnz;
  double* gdev = nullptr;
  do {
    if ((s = dev_alloc(&M->valhat, (size_t)nnz + NNZ_PAD)) != GNP_OK) break;
    if ((s = apply_ws_alloc(M->ws, n)) != GNP_OK) break;
    if ((s = dev_alloc(&M->w_dev, (size_t)cnt)) != GNP_OK) break;
    if ((s = dev_alloc(&M->w_best, (size_t)cnt)) != GNP_OK) break;
    if ((s = dev_alloc(&gdev, 1)) != GNP_OK) break;
    if ((s = gamma_launch(A, gdev, 0)) != GNP_OK) break;
    cudaError_t e = cudaMemcpy(&M->gamma, gdev, sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      set_error("gnp_create: %s", cudaGetErrorString(e));
      s = GNP_ERR_CUDA;
      break;
    }
    if (!(M->gamma > 0.0) || !std::isfinite(M->gamma)) {
      set_error("gnp_create: gamma = %g (matrix is zero or not finite)", M->gamma);
      s = GNP_ERR_INVALID_ARG;
      break;
    }
    if ((s = gnp_set_weights(M, weights_host, cnt)) != GNP_OK) break;
  } while (0);
  dev_free(gdev);
  if (s != GNP_OK) {
    gnp_destroy(M);
    return s;
  }
  // A_hat = A / gamma in float32 (Eq. 6)
  cudaMemset(M->valhat + nnz, 0, sizeof(float) * NNZ_PAD);
  if (nnz > 0) k_scale_values<<<4 * NUM_SMS_GB300, 256>>>(A->val, nnz, M->gamma, M->valhat);
  s = check_launch("k_scale_values");
  if (s == GNP_OK && cudaDeviceSynchronize() != cudaSuccess) {
    set_error("gnp_create: %s", cudaGetErrorString(cudaGetLastError()));
    s = GNP_ERR_CUDA;
  }
  // the TMA-gather layer's schedule, for matrices with rows too long for the short-row kernels
  if (s == GNP_OK && row_kernel_mode(A) == 0) s = tma_prepare(A);
  if (s != GNP_OK) {
    gnp_destroy(M);
    return s;
  }
  *out = M;
  return GNP_OK;
}

void gnp_destroy(gnp_model* M) {
  if (!M) return;
  train_free(M->train);
  M->train = nullptr;
  dev_free(M->valhat);
  dev_free(M->valhat_t);
  apply_ws_free(M->ws);
  dev_free(M->w_dev);
  dev_free(M->w_best);
  delete M;
}

int gnp_model_gamma(const gnp_model* M, double* gamma_out) {
  GNP_REQUIRE(M && gamma_out, "gnp_model_gamma: null argument");
  *gamma_out = M->gamma;
  return GNP_OK;
}

int gnp_set_hprec(gnp_model* M, int hprec) {
  GNP_REQUIRE(M, "gnp_set_hprec: null model");
  GNP_REQUIRE(hprec == GNP_H_FP32 || hprec == GNP_H_BF16, "gnp_set_hprec: bad hprec %d", hprec);
  if (M->hprec != hprec) ++M->version;
  M->hprec = hprec;
  return GNP_OK;
}

int gnp_apply(gnp_model* M, const double* v_dev, float* z_dev, void* stream) {
  return gnp_apply_trace(M, v_dev, z_dev, nullptr, stream);
}

int gnp_apply_trace(gnp_model* M, const double* v_dev, float* z_dev, float* hidden_dev, void* stream) {
  GNP_REQUIRE(M && v_dev && z_dev, "gnp_apply: null argument");
  ColPtr v{const_cast<double*>(v_dev), 0, nullptr, 0};
  ColPtr z{z_dev, 0, nullptr, 0};
  return apply_launch(M, v, nullptr, z, hidden_dev, nullptr, as_stream(stream));
}



int gnp_layer_apply(gnp_model* M, int layer, const void* h_in_dev, void* h_out_dev, void* stream) {
  GNP_REQUIRE(M && h_in_dev && h_out_dev, "gnp_layer_apply: null argument");
  GNP_REQUIRE(layer >= 0 && layer < M->cfg.L, "gnp_layer_apply: layer %d outside [0, %d)", layer, M->cfg.L);
  GNP_REQUIRE(h_in_dev != h_out_dev, "gnp_layer_apply: the input and output blocks must differ");
  GNP_TRY(model_sync_host(M));
  cudaStream_t st = as_stream(stream);
  const bool paper = M->cfg.form == GNP_LAYER_PAPER;
  if (M->hprec == GNP_H_BF16) {
    auto* hi = static_cast<const uint16_t*>(h_in_dev);
    auto* ho = static_cast<uint16_t*>(h_out_dev);
    return paper ? layer_impl<uint16_t, GNP_LAYER_PAPER>(M, layer, hi, ho, st)
                 : layer_impl<uint16_t, GNP_LAYER_RESID>(M, layer, hi, ho, st);
  }
  auto* hi = static_cast<const float*>(h_in_dev);
  auto* ho = static_cast<float*>(h_out_dev);
  return paper ? layer_impl<float, GNP_LAYER_PAPER>(M, layer, hi, ho, st)
               : layer_impl<float, GNP_LAYER_RESID>(M, layer, hi, ho, st);
}

int gnp_get_weights(gnp_model* M, float* host_blob, int* count) {
  GNP_REQUIRE(M && count, "gnp_get_weights: null argument");
  const int cnt = weight_count(M->cfg.L);
  if (!host_blob) {
    *count = cnt;
    return GNP_OK;
  }
  GNP_REQUIRE(*count >= cnt, "gnp_get_weights: buffer of %d < %d floats", *count, cnt);
  GNP_TRY(model_sync_host(M));
  memcpy(host_blob, M->w_host.data(), sizeof(float) * cnt);
  *count = cnt;
  return GNP_OK;
}

int gnp_set_weights(gnp_model* M, const float* host_blob, int count) {
  GNP_REQUIRE(M && host_blob, "gnp_set_weights: null argument");
  const int cnt = weight_count(M->cfg.L);
  GNP_REQUIRE(count == cnt, "gnp_set_weights: got %d floats, expected %d", count, cnt);
  M->w_host.assign(host_blob, host_blob + cnt);
  M->host_stale = false;
  ++M->version;
  GNP_TRY_CUDA(cudaMemcpy(M->w_dev, host_blob, sizeof(float) * cnt, cudaMemcpyHostToDevice));
  GNP_TRY_CUDA(cudaMemcpy(M->w_best, host_blob, sizeof(float) * cnt, cudaMemcpyHostToDevice));
  train_reset(M->train);
  return GNP_OK;
}

}  // extern "C"
