// Internal declarations shared by the translation units of libgnp.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/gnp.h"

namespace gnp {

// ------------------------------------------------------------------ errors

void set_error(const char* fmt, ...);

#define GNP_TRY_CUDA(call)                                                          \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      ::gnp::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                       __FILE__, __LINE__);                                         \
      return (e_ == cudaErrorMemoryAllocation) ? GNP_ERR_OOM : GNP_ERR_CUDA;        \
    }                                                                               \
  } while (0)

#define GNP_TRY(call)                 \
  do {                                \
    int s_ = (call);                  \
    if (s_ != GNP_OK) return s_;      \
  } while (0)

#define GNP_REQUIRE(cond, ...)                 \
  do {                                         \
    if (!(cond)) {                             \
      ::gnp::set_error(__VA_ARGS__);           \
      return GNP_ERR_INVALID_ARG;              \
    }                                          \
  } while (0)

// Check the launch of the kernel just enqueued.
int check_launch(const char* what);

template <class T>
int dev_alloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return GNP_OK;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    set_error("cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
    *p = nullptr;
    return GNP_ERR_OOM;
  }
  return GNP_OK;
}

template <class T>
void dev_free(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ------------------------------------------------------------ tiling constants

constexpr int TILE = 256;            // rows per tile = threads per tile-kernel block
constexpr int NNZ_PAD = 4;           // index/value arrays carry 4 spare (zero) entries
constexpr int RED_THREADS = 256;     // threads of the streaming reduction kernels
constexpr int NUM_SMS_GB300 = 152;

// A float64 reduction scratch: per-block partials plus an arrival counter that the
// last block resets.  One instance per concurrently running reduction chain.
struct RedScratch {
  double* partials = nullptr;   // [max_blocks * max_k]
  unsigned* counter = nullptr;  // one word, zero between launches
  int max_blocks = 0;
  int max_k = 0;
};
int red_alloc(RedScratch& r, int max_blocks, int max_k);
void red_free(RedScratch& r);

// Number of blocks of the grid-stride reduction kernels for a vector of length n: one
// row per thread up to four blocks per SM, so that small vectors still spread over
// every SM (latency, not bandwidth, bounds them).
inline int red_blocks(long long n) {
  long long per = (long long)RED_THREADS;
  long long b = (n + per - 1) / per;
  if (b < 1) b = 1;
  if (b > 4 * NUM_SMS_GB300) b = 4 * NUM_SMS_GB300;
  return (int)b;
}

// ------------------------------------------------------------------ objects

struct Solver;       // FGMRES workspace (krylov.cu)
struct MultiSolver;  // multi-right-hand-side FGMRES workspace (multi.cu)

// Work items of the TMA-gather Res-GCONV layer (gconv_tma.cu) for one matrix and one
// hidden-block precision: items[off[b] .. off[b+1]) = {tile, first nonzero, end, flags}
// for persistent block b (flags: 1 first chunk of the tile, 2 last chunk).
struct TmaSched {
  int4* items = nullptr;
  int* off = nullptr;
  int grid = 0;
  int cap = 0;
  long long nitems = 0;
};

struct CscView {
  int* ptr = nullptr;   // [n+1] column pointers of A (= row pointers of A^T)
  int* idx = nullptr;   // [nnz] row index of each entry
  int* perm = nullptr;  // [nnz] position of the entry in the CSR arrays
};

}  // namespace gnp

struct gnp_mat {
  int n = 0;
  long long nnz = 0;
  int device = 0;
  int max_deg = 0;           // most nonzeros in one row
  int* rp = nullptr;
  int* col = nullptr;
  double* val = nullptr;
  gnp::CscView csc;          // built lazily for training
  gnp::Solver* solver = nullptr;
  gnp::MultiSolver* msolver = nullptr;
  gnp::RedScratch red;       // for gnp_gamma / small reductions
  double* scratch_d = nullptr;   // [n] float64 scratch (column sums)
  gnp::TmaSched tma[2];      // TMA-gather layer schedule: [0] float32, [1] bfloat16 hidden block
  bool tma_built = false;
};

namespace gnp {

// ------------------------------------------------------------------ device helpers

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Deterministic block sum of one value per thread (fixed shuffle tree, then warp 0
// adds the warp totals in order).  Result valid in thread 0.  `sh` >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = lane < nw ? sh[lane] : 0.0;
    t = warp_sum(t);
  }
  return t;
}

// The block's place in the grid a kernel body works on: the hardware grid for a stand-alone
// launch, or one request's share of a grouped launch (several requests' grids laid end to
// end in one launch, see GTable).  A body reads bid / nblk where a kernel reads blockIdx.x
// / gridDim.x, so the same arithmetic runs in both.
struct VGrid {
  int bid;
  int nblk;
};
__device__ __forceinline__ VGrid hw_grid() { return VGrid{(int)blockIdx.x, (int)gridDim.x}; }

// Work table of a grouped launch (passed by value): entry i is request slot slot[i], whose
// blocks are start[i] .. start[i+1]-1 of the launch.  Block b finds its entry by a scan of
// at most GT_MAX entries; gt_entry returns the entry and sets the block's place in that
// request's grid.
constexpr int GT_MAX = 16;
struct GTable {
  int count;
  int slot[GT_MAX];
  int start[GT_MAX + 1];
};
__device__ __forceinline__ int gt_entry(const GTable& t, VGrid& g) {
  const int b = (int)blockIdx.x;
  int i = 0;
  while (i + 1 < t.count && b >= t.start[i + 1]) ++i;
  g.bid = b - t.start[i];
  g.nblk = t.start[i + 1] - t.start[i];
  return i;
}

// Last-block arrival: every block has written its partials; the block that arrives
// last (of nblk) sees true (after a fence) and may read all partials.  It must reset
// *counter.
__device__ __forceinline__ bool last_block_arrive(unsigned* counter, int nblk) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    s_last = (t == (unsigned)nblk - 1u);
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}
__device__ __forceinline__ bool last_block_arrive(unsigned* counter) { return last_block_arrive(counter, gridDim.x); }

// In the last block: out[k] = sum_b partials[b*K + k] for k < K, in a fixed order
// (lane-strided over blocks, then a fixed shuffle tree).  out is shared memory.
// This runs on one block while the rest of the GPU waits, so it is latency that counts:
// a warp takes RP_COLS columns at a time and issues the loads of up to RP_UNROLL blocks
// per lane (for every column) before it adds any, i.e. one L2 round trip per 256 blocks
// instead of one per 32.  The additions keep the order b = lane, lane + 32, ...
constexpr int RP_COLS = 4, RP_UNROLL = 8;
__device__ __forceinline__ void reduce_partials(const double* partials, int nblocks, int K,
                                                double* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k0 = w * RP_COLS; k0 < K; k0 += nw * RP_COLS) {
    double s[RP_COLS];
#pragma unroll
    for (int c = 0; c < RP_COLS; ++c) s[c] = 0.0;
    for (int b0 = lane; b0 < nblocks; b0 += 32 * RP_UNROLL) {
      double p[RP_UNROLL][RP_COLS];
#pragma unroll
      for (int u = 0; u < RP_UNROLL; ++u) {
        const int b = b0 + 32 * u;
#pragma unroll
        for (int c = 0; c < RP_COLS; ++c)
          p[u][c] = (b < nblocks && k0 + c < K) ? __ldcg(partials + (size_t)b * K + k0 + c) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < RP_UNROLL; ++u) {
        if (b0 + 32 * u < nblocks) {
#pragma unroll
          for (int c = 0; c < RP_COLS; ++c) s[c] += p[u][c];
        }
      }
    }
#pragma unroll
    for (int c = 0; c < RP_COLS; ++c) {
      const double t = warp_sum(s[c]);
      if (lane == 0 && k0 + c < K) out[k0 + c] = t;
    }
  }
  __syncthreads();
}

// --------------------------------------------------- nnz-balanced tile gather
//
// A block owns TILE consecutive rows [r0, r0+rows).  Its nnz range [E0, E0+E) is split
// evenly over S = TILE/G "slots" of G lanes; a slot walks its contiguous nnz range in
// order, accumulating sum_j a_ij x_j for the row it is in.  A row lying inside one
// slot's range is complete and written to s_agg; a row split over several slots leaves
// one partial sum per slot in cf (the slot's first row) or cl (its last row), and the
// epilogue adds them in slot order (deterministic).  Power-law rows of thousands of
// entries are thus shared by many slots instead of stalling one.
//
// Traits TR: G lanes per slot, NV accumulator scalars per lane (the row vector has
// W = G*NV entries), STRIDE = smem row stride of s_agg, scalar acc type `acc`,
// value type `val_t`, and a loader TR::load(X, c, q, out[NV]) of lane q's part of x_c.

// ROWS rows per tile (<= TILE, the block's thread count): fewer rows than threads give
// each slot fewer nonzeros, i.e. a shorter chain of dependent loads per block.
template <class TR, int ROWS = TILE>
struct TileSmem {
  static constexpr int G = TR::G;
  static constexpr int NV = TR::NV;
  static constexpr int S = TILE / G;
  static constexpr int W = G * NV;
  static constexpr int R = ROWS;
  using acc = typename TR::acc;
  int rp[ROWS + 1];
  int firstrow[S];
  acc cf[S][W];
  acc cl[S][W];
  acc agg[ROWS * TR::STRIDE];
};

// Slot of nonzero e: the largest s with floor(s E / S) <= e - E0 (32-bit arithmetic
// whenever E * S fits, which is every tile of fewer than 2^24 nonzeros).
__device__ __forceinline__ int slot_of(int e, int E0, int E, int S) {
  const unsigned ep = (unsigned)(e - E0) + 1u;
  if ((unsigned long long)E * (unsigned)S < (1ull << 32))
    return (int)((ep * (unsigned)S + (unsigned)E - 1u) / (unsigned)E) - 1;
  return (int)(((unsigned long long)ep * S + E - 1) / E) - 1;
}

template <class TR, class SM>
__device__ __forceinline__ void tile_flush(SM& sm, int s, int q, int fr, int r, int rstart,
                                           int rend, int a, int b,
                                           const typename TR::acc (&acc)[TR::NV]) {
  typename TR::acc* dst;
  if (rstart >= a && rend <= b)
    dst = &sm.agg[r * TR::STRIDE + q * TR::NV];
  else if (r == fr)
    dst = &sm.cf[s][q * TR::NV];
  else
    dst = &sm.cl[s][q * TR::NV];
#pragma unroll
  for (int k = 0; k < TR::NV; ++k) dst[k] = acc[k];
}

// Requires sm.rp[0..rows] loaded and a __syncthreads() before the call.  Ends with
// no barrier; the caller syncs before reading agg/cf/cl.
//
// GROUP neighbour rows are loaded at once per lane (4 or 8): the column indices and
// values of the next group are fetched while the current group's rows are in flight.
template <class TR, class SM, int GROUP = 4>
__device__ __forceinline__ void tile_gather(SM& sm, int rows, const int* __restrict__ col,
                                            const typename TR::val_t* __restrict__ val,
                                            const typename TR::x_t* __restrict__ X) {
  static_assert(GROUP == 4 || GROUP == 8, "4 or 8 rows in flight per lane");
  constexpr int G = TR::G, NV = TR::NV, S = TILE / G;
  using A = typename TR::acc;
  const int s = threadIdx.x / G, q = threadIdx.x % G;
  const int E0 = sm.rp[0];
  const int E = sm.rp[rows] - E0;
  const int a = E0 + (int)(((long long)s * E) / S);
  const int b = E0 + (int)(((long long)(s + 1) * E) / S);
  if (a >= b) {
    if (q == 0) sm.firstrow[s] = -1;
    return;
  }
  int lo = 0, hi = rows - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (sm.rp[mid] <= a) lo = mid; else hi = mid - 1;
  }
  int r = lo;
  const int fr = r;
  if (q == 0) sm.firstrow[s] = fr;
  int rstart = sm.rp[r];
  int rnext = sm.rp[r + 1];
  A acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = A(0);

  auto step = [&](int e, typename TR::val_t v, const A (&h)[NV]) {
    while (e >= rnext) {
      tile_flush<TR, SM>(sm, s, q, fr, r, rstart, rnext, a, b, acc);
#pragma unroll
      for (int k = 0; k < NV; ++k) acc[k] = A(0);
      ++r;
      rstart = rnext;
      rnext = sm.rp[r + 1];
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = fma(A(v), h[k], acc[k]);
  };

  // groups of GROUP nonzeros; the next group's column indices and values are loaded
  // while the current group's neighbour rows are in flight (one dependent round trip less)
  int e = a;
  int cn[GROUP];
  typename TR::val_t vn[GROUP];
  if (e + GROUP <= b) {
#pragma unroll
    for (int u = 0; u < GROUP; ++u) {
      cn[u] = __ldg(col + e + u);
      vn[u] = __ldg(val + e + u);
    }
  }
  for (; e + GROUP <= b; e += GROUP) {
    int c[GROUP];
    typename TR::val_t v[GROUP];
#pragma unroll
    for (int u = 0; u < GROUP; ++u) {
      c[u] = cn[u];
      v[u] = vn[u];
    }
    if (e + 2 * GROUP <= b) {
#pragma unroll
      for (int u = 0; u < GROUP; ++u) {
        cn[u] = __ldg(col + e + GROUP + u);
        vn[u] = __ldg(val + e + GROUP + u);
      }
    }
    A h[GROUP][NV];
#pragma unroll
    for (int u = 0; u < GROUP; ++u) TR::load(X, c[u], q, h[u]);
#pragma unroll
    for (int u = 0; u < GROUP; ++u) step(e + u, v[u], h[u]);
  }
  if (e < b) {  // the last b - e < GROUP nonzeros: one predicated group, one round trip
    int c[GROUP];
    typename TR::val_t v[GROUP];
    A h[GROUP][NV];
#pragma unroll
    for (int u = 0; u < GROUP; ++u) {
      if (e + u < b) {
        c[u] = __ldg(col + e + u);
        v[u] = __ldg(val + e + u);
      }
    }
#pragma unroll
    for (int u = 0; u < GROUP; ++u)
      if (e + u < b) TR::load(X, c[u], q, h[u]);
#pragma unroll
    for (int u = 0; u < GROUP; ++u)
      if (e + u < b) step(e + u, v[u], h[u]);
  }
  tile_flush<TR, SM>(sm, s, q, fr, r, rstart, rnext, a, b, acc);
}

// After the gather and a __syncthreads(): the complete sum of row t (W entries) for
// the epilogue thread t < rows.  Entries [k0, k0+cnt) are returned in out.
template <class TR, int CNT, class SM>
__device__ __forceinline__ void tile_row_sum(const SM& sm, int t, int k0,
                                             typename TR::acc (&out)[CNT]) {
  using A = typename TR::acc;
  constexpr int S = TILE / TR::G;
  const int rs = sm.rp[t], re = sm.rp[t + 1];
#pragma unroll
  for (int k = 0; k < CNT; ++k) out[k] = A(0);
  if (rs == re) return;
  const int E0 = sm.rp[0];
  // rows is implied by the caller; E from the last row pointer of the tile
  const int E = sm.rp[SM::R] - E0;  // caller pads rp beyond `rows` with the last value
  const int s_lo = slot_of(rs, E0, E, S);
  const int s_hi = slot_of(re - 1, E0, E, S);
  if (s_lo == s_hi) {
#pragma unroll
    for (int k = 0; k < CNT; ++k) out[k] = sm.agg[t * TR::STRIDE + k0 + k];
    return;
  }
  for (int s = s_lo; s <= s_hi; ++s) {
    const int fr = sm.firstrow[s];
    if (fr < 0) continue;  // empty slot (the tile has fewer nonzeros than slots)
    const A* src = (fr == t) ? sm.cf[s] : sm.cl[s];
#pragma unroll
    for (int k = 0; k < CNT; ++k) out[k] += src[k0 + k];
  }
}

// Load the row pointers of the tile into smem, padding entries past `rows` with the
// tile's last pointer so that sm.rp[TILE] is the end of the tile's nnz range.
template <class TR, class SM>
__device__ __forceinline__ void tile_load_rp(SM& sm, const int* __restrict__ rp, int r0,
                                             int rows) {
  for (int i = threadIdx.x; i <= SM::R; i += blockDim.x)
    sm.rp[i] = __ldg(rp + r0 + (i < rows ? i : rows));
}

// ------------------------------------------------------------------ bf16 helpers

__device__ __forceinline__ float bf16lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&p);
}

}  // namespace gnp
