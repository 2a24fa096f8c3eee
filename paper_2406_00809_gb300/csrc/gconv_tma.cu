// Res-GCONV layer (Eq. 7) for matrices with long rows, with the neighbour rows gathered by
// the Tensor Memory Accelerator into shared memory.
//
//   k_gconv_tma  one persistent block per SM walks its share of the matrix in items: an
//                item is a chunk of at most CAP consecutive nonzeros of one 64-row tile
//                (long tiles give several items).  For each item the block copies the
//                hidden rows H[col[e]] of its nonzeros into a shared-memory stage with
//                cp.async.bulk.tensor tile::gather4 (four rows per instruction, completion
//                counted in bytes on the stage's mbarrier); three stages, so that two
//                items are in flight while the third is consumed.  Consumption is the
//                nnz-balanced slot walk of the register-gather kernel, reading the rows
//                from shared memory: slots of G lanes split the item's nonzeros evenly, a
//                row inside one slot is written to the tile's aggregate at once, and
//                partial sums of rows split over slots (or items) are added to it in slot
//                order after the walk, so the result does not depend on timing.  After a
//                tile's last item, four threads per row form ReLU(h U + agg W) (or
//                h + ReLU(agg W)) and store the output rows, or (last layer) the decoder's
//                z = dec(.) tau / sqrt(n).
//
// The schedule (items per block, balanced by nonzeros over the SMs) depends only on the
// matrix and is built on the host once per matrix and hidden-block precision.  Every
// wait on an mbarrier is bounded (2 s of device time); a block that gives up, or meets a
// malformed item record, counts the event in a device flag (gnp_kernel_faults), waits
// (bounded) for its copies in flight and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstddef>
#include <cstdlib>
#include <numeric>
#include <queue>
#include <vector>

#include "gconv_rows.cuh"
#include "solver.h"

namespace gnp {

constexpr int TM_ROWS = 64;      // rows per tile
constexpr int TM_THREADS = 256;  // 8 warps; 4 threads per row in the epilogue
constexpr int TM_NST = 3;        // stages
static_assert(TM_ROWS * 4 == TM_THREADS, "four epilogue threads per row");

template <class HT> struct TmaCap;
template <> struct TmaCap<float> { static constexpr int CAP = 768; };      // 48 KB of rows per stage
template <> struct TmaCap<uint16_t> { static constexpr int CAP = 1024; };  // 32 KB of rows per stage

template <class HT>
struct TmaSmem {
  static constexpr int CAP = TmaCap<HT>::CAP;
  static constexpr int RB = HTraits<HT>::ROW_BYTES;
  static constexpr int G = HTraits<HT>::TR::G;
  static constexpr int NV = HTraits<HT>::TR::NV;
  static constexpr int S = TM_THREADS / G;
  static constexpr int SROW = HTraits<HT>::SROW;
  static_assert(CAP % 4 == 0 && CAP / 4 <= TM_THREADS, "one gather4 per thread per item");
  static_assert(4 * TM_THREADS >= CAP, "four values per thread per item");
  unsigned char g[TM_NST][CAP * RB];  // gathered rows (first member: 128-byte aligned base)
  float val[TM_NST][CAP];
  int rp[TM_NST][TM_ROWS + 1];
  int4 item[TM_NST];
  unsigned long long full[TM_NST];
  // read and written as 16-byte vectors: each starts on a 16-byte boundary
  __align__(16) float agg[TM_ROWS * 20];
  __align__(16) float cf[S][16];
  __align__(16) float cl[S][16];
  int firstrow[S];
  __align__(16) uint32_t stile[TM_ROWS * SROW];
  float zpart[TM_ROWS][4];
};
static_assert(offsetof(TmaSmem<float>, agg) % 16 == 0 && offsetof(TmaSmem<float>, cf) % 16 == 0 &&
                  offsetof(TmaSmem<float>, cl) % 16 == 0 && offsetof(TmaSmem<float>, stile) % 16 == 0 &&
                  offsetof(TmaSmem<float>, full) % 8 == 0 && offsetof(TmaSmem<float>, g) == 0,
              "vector-accessed members of the float32 layout are aligned");
static_assert(offsetof(TmaSmem<uint16_t>, agg) % 16 == 0 && offsetof(TmaSmem<uint16_t>, cf) % 16 == 0 &&
                  offsetof(TmaSmem<uint16_t>, cl) % 16 == 0 && offsetof(TmaSmem<uint16_t>, stile) % 16 == 0 &&
                  offsetof(TmaSmem<uint16_t>, full) % 8 == 0 && offsetof(TmaSmem<uint16_t>, g) == 0,
              "vector-accessed members of the bfloat16 layout are aligned");

__device__ int g_kernel_faults = 0;

__device__ __forceinline__ void* tma_colptr(const ColPtr& p) {
  const int j = p.jptr ? *p.jptr : 0;
  return static_cast<char*>(p.base) + (size_t)(j + p.off) * p.stride;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for phase `parity` of the mbarrier: false after 2 s of device time.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(1000000u)
        : "memory");
    if (ok) return true;
    if (global_ns() - t0 > 2000000000ull) return false;
  }
}

// Four hidden rows r0..r3 (box: one row of 16 values) into dst, counted on bar.
__device__ __forceinline__ void tma_gather4(uint32_t dst, const CUtensorMap* map, int r0, int r1, int r2, int r3,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Four bytes-per-lane row parts of a gathered row (lane q of a G-lane slot).
template <class HT>
__device__ __forceinline__ void smem_row_part(const unsigned char* row, int q, float (&h)[HTraits<HT>::TR::NV]) {
  const uint4 t = *reinterpret_cast<const uint4*>(row + 16 * q);
  if constexpr (sizeof(HT) == 4) {
    h[0] = __uint_as_float(t.x);
    h[1] = __uint_as_float(t.y);
    h[2] = __uint_as_float(t.z);
    h[3] = __uint_as_float(t.w);
  } else {
    h[0] = bf16lo(t.x); h[1] = bf16hi(t.x); h[2] = bf16lo(t.y); h[3] = bf16hi(t.y);
    h[4] = bf16lo(t.z); h[5] = bf16hi(t.z); h[6] = bf16lo(t.w); h[7] = bf16hi(t.w);
  }
}

// Per-thread registers that carry one item from its loads to its issue.
struct TmaFetch {
  int4 rec;     // {tile, e0, e1, flags}
  int c[4];     // column indices of nonzeros e0 + 4 t + u
  float v[4];   // their A_hat values
  int rpv;      // row pointer rp[r0 + min(t, rows)] (t <= TM_ROWS)
};

template <class HT>
__device__ __forceinline__ void tma_fetch(TmaFetch& f, const int4& rec, const int* __restrict__ rp,
                                          const int* __restrict__ col, const float* __restrict__ valhat, int n) {
  const int t = threadIdx.x;
  f.rec = rec;
  const int e0 = rec.y, e1 = rec.z;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = e0 + 4 * t + u;
    const bool ok = e < e1;
    f.c[u] = ok ? __ldg(col + e) : -1;
    f.v[u] = ok ? __ldg(valhat + e) : 0.0f;
  }
  f.rpv = 0;
  if (t <= TM_ROWS) {
    const int r0 = rec.x * TM_ROWS;
    const int rows = min(TM_ROWS, n - r0);
    f.rpv = __ldg(rp + r0 + min(t, rows));
  }
}

// Stage the item's values, row pointers and record, and start its row copies.
template <class HT>
__device__ __forceinline__ void tma_issue(TmaSmem<HT>& sm, int st, const TmaFetch& f, const CUtensorMap* map) {
  constexpr int CAP = TmaSmem<HT>::CAP;
  constexpr int RB = TmaSmem<HT>::RB;
  const int t = threadIdx.x;
#pragma unroll
  for (int u = 0; u < 4; ++u)
    if (4 * t + u < CAP) sm.val[st][4 * t + u] = f.v[u];
  if (t <= TM_ROWS) sm.rp[st][t] = f.rpv;
  if (t == 0) sm.item[st] = f.rec;
  const int nops = (f.rec.z - f.rec.y + 3) / 4;
  const uint32_t bar = smem_u32(&sm.full[st]);
  if (t == 0) mbar_arrive_expect_tx(bar, (uint32_t)(nops * 4 * RB));
  if (t < nops) {
    fence_proxy_async();
    const int c0 = f.c[0];  // valid: e0 + 4 t < e1
    tma_gather4(smem_u32(&sm.g[st][(size_t)4 * t * RB]), map, c0, f.c[1] >= 0 ? f.c[1] : c0,
                f.c[2] >= 0 ? f.c[2] : c0, f.c[3] >= 0 ? f.c[3] : c0, bar);
  }
}

template <class HT, int FORM>
__device__ __forceinline__ void tma_layer_q(const float (&h)[16], const float (&agg)[16], const LayerW& lw, int q,
                                            float (&o)[4]) {
  switch (q) {  // warp-uniform: the weights stay uniform operands
    case 0: layer_part<FORM, 0, 4>(h, agg, lw, o); break;
    case 1: layer_part<FORM, 4, 4>(h, agg, lw, o); break;
    case 2: layer_part<FORM, 8, 4>(h, agg, lw, o); break;
    default: layer_part<FORM, 12, 4>(h, agg, lw, o); break;
  }
}

__device__ __forceinline__ float tma_decode_q(const float (&o)[16], const DecW& dw, int q) {
  switch (q) {
    case 0: return decode_part<0, 8>(o, dw);
    case 1: return decode_part<8, 8>(o, dw);
    case 2: return decode_part<16, 8>(o, dw);
    default: return decode_part<24, 8>(o, dw);
  }
}

template <class HT, int FORM, bool DEC>
__global__ void __launch_bounds__(TM_THREADS, 1)
k_gconv_tma(const __grid_constant__ CUtensorMap hmap, const int4* __restrict__ items, const int* __restrict__ item_off,
            const int* __restrict__ rp, const int* __restrict__ col, const float* __restrict__ valhat,
            const HT* __restrict__ Hin, HT* __restrict__ Hout, ColPtr zp, const double* __restrict__ tau,
            double sqrt_n, int n, const int* __restrict__ ctl, const __grid_constant__ LayerW lw,
            const __grid_constant__ DecW dw) {
  using SM = TmaSmem<HT>;
  constexpr int CAP = SM::CAP, RB = SM::RB, G = SM::G, NV = SM::NV, S = SM::S, SROW = SM::SROW;
  extern __shared__ unsigned char smraw[];
  SM& sm = *reinterpret_cast<SM*>((reinterpret_cast<uintptr_t>(smraw) + 127) & ~uintptr_t(127));
  const int t = threadIdx.x;
  const int w = t >> 5, lane = t & 31;
  const int i0 = item_off[blockIdx.x];
  const int nit = item_off[blockIdx.x + 1] - i0;
  if (t == 0) {
    for (int s = 0; s < TM_NST; ++s) mbar_init(smem_u32(&sm.full[s]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = t; i < TM_ROWS * 20; i += TM_THREADS) sm.agg[i] = 0.0f;
  __syncthreads();
  pdl_wait();
  if ((ctl && !ctl[1]) || nit == 0) return;
  __shared__ float s_back;
  if (DEC && t == 0) {
    const double tv = *tau;
    s_back = (float)(tv > 0.0 ? tv / sqrt_n : 0.0);
  }
  // prologue: items 0 and 1 issued, item 2 fetched, record 3 loaded
  TmaFetch fa;
  int4 rec_next = make_int4(0, 0, 0, 0);
  for (int k = 0; k < 2 && k < nit; ++k) {
    tma_fetch<HT>(fa, items[i0 + k], rp, col, valhat, n);
    tma_issue<HT>(sm, k, fa, &hmap);
  }
  if (nit > 2) tma_fetch<HT>(fa, items[i0 + 2], rp, col, valhat, n);
  if (nit > 3) rec_next = items[i0 + 3];
  // every thread staged a part of items 0 and 1 (values, row pointers, the record); the
  // mbarrier releases only the arriving thread's writes, so the block syncs once here
  // (later items are staged two barriers before their use)
  __syncthreads();
  const int ntiles = (n + TM_ROWS - 1) / TM_ROWS;
  const int row = (w >> 2) * 32 + lane;  // epilogue / combine row (warp-uniform quarter)
  const int qq = w & 3;
  for (int i = 0; i < nit; ++i) {
    const int st = i % TM_NST;
    // 1. start item i+2 (its stage was released by the barrier that ended item i-1)
    if (i + 2 < nit) tma_issue<HT>(sm, (i + 2) % TM_NST, fa, &hmap);
    // 2. loads for item i+3 and the record of item i+4
    if (i + 3 < nit) tma_fetch<HT>(fa, rec_next, rp, col, valhat, n);
    if (i + 4 < nit) rec_next = items[i0 + i + 4];
    // 3. the item; the tile's own rows when it is the tile's last item
    const int4 rec = sm.item[st];
    const int tile = rec.x, e0 = rec.y, e1 = rec.z;
    const bool valid = tile >= 0 && tile < ntiles && e0 <= e1 && e1 - e0 <= CAP;  // a malformed record: skip
    const bool last = (rec.w & 2) != 0;
    const int r0 = valid ? tile * TM_ROWS : 0;
    const int rows = min(TM_ROWS, n - r0);
    uint4 own = make_uint4(0, 0, 0, 0);
    constexpr int OWN16 = TM_ROWS * RB / 16;  // 16-byte parts of the tile's own rows
    if (valid && last && t < rows * RB / 16) own = __ldg(reinterpret_cast<const uint4*>(Hin + (size_t)r0 * 16) + t);
    static_assert(OWN16 <= TM_THREADS, "one 16-byte part per thread");
    // 4. wait for the item's rows
    const bool ok = mbar_wait(smem_u32(&sm.full[st]), (uint32_t)((i / TM_NST) & 1));
    if (__syncthreads_or(!ok || !valid)) {
      if (t == 0) {
        atomicAdd(&g_kernel_faults, 1);
        for (int k = i + 1; k < nit && k < i + 3; ++k)
          mbar_wait(smem_u32(&sm.full[k % TM_NST]), (uint32_t)((k / TM_NST) & 1));
      }
      __syncthreads();
      return;
    }
    // 5. slot walk over [e0, e1) from shared memory
    const int* srp = sm.rp[st];
    const unsigned char* gst = sm.g[st];
    const float* sval = sm.val[st];
    {
      const int E = e1 - e0;
      const int s = t / G, q = t % G;
      const int a = e0 + (int)(((long long)s * E) / S);
      const int b = e0 + (int)(((long long)(s + 1) * E) / S);
      if (a >= b) {
        if (q == 0) sm.firstrow[s] = -1;
      } else {
        int lo = 0, hi = rows - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (srp[mid] <= a) lo = mid;
          else hi = mid - 1;
        }
        int r = lo;
        const int fr = r;
        if (q == 0) sm.firstrow[s] = fr;
        int rstart = srp[r], rnext = srp[r + 1];
        float acc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = 0.0f;
        auto flush = [&]() {
          float* dst;
          if (rstart >= a && rnext <= b) dst = &sm.agg[r * 20 + q * NV];
          else if (r == fr) dst = &sm.cf[s][q * NV];
          else dst = &sm.cl[s][q * NV];
#pragma unroll
          for (int k = 0; k < NV; ++k) dst[k] = acc[k];
        };
        for (int e = a; e < b; e += 4) {
          float h[4][NV];
          float v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (e + u < b) {
              smem_row_part<HT>(gst + (size_t)(e + u - e0) * RB, q, h[u]);
              v[u] = sval[e + u - e0];
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (e + u < b) {
              while (e + u >= rnext) {
                flush();
#pragma unroll
                for (int k = 0; k < NV; ++k) acc[k] = 0.0f;
                ++r;
                rstart = rnext;
                rnext = srp[r + 1];
              }
#pragma unroll
              for (int k = 0; k < NV; ++k) acc[k] = fmaf(v[u], h[u][k], acc[k]);
            }
          }
        }
        flush();
      }
    }
    __syncthreads();
    // 6. partial sums of rows split over slots or items, added in slot order
    if (row < rows) {
      const int rs = srp[row], re = srp[row + 1];
      const int lo = max(rs, e0), hi = min(re, e1);
      if (lo < hi) {
        const int E = e1 - e0;
        const int s_lo = slot_of(lo, e0, E, S), s_hi = slot_of(hi - 1, e0, E, S);
        const int a = e0 + (int)(((long long)s_lo * E) / S);
        const int b = e0 + (int)(((long long)(s_lo + 1) * E) / S);
        const bool complete = s_lo == s_hi && rs >= a && re <= b;
        if (!complete) {
          float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
          for (int s = s_lo; s <= s_hi; ++s) {
            const int fr = sm.firstrow[s];
            if (fr < 0) continue;
            const float4 p = *reinterpret_cast<const float4*>((fr == row ? sm.cf[s] : sm.cl[s]) + 4 * qq);
            sum.x += p.x;
            sum.y += p.y;
            sum.z += p.z;
            sum.w += p.w;
          }
          float4* d = reinterpret_cast<float4*>(&sm.agg[row * 20 + 4 * qq]);
          float4 cur = *d;
          cur.x += sum.x;
          cur.y += sum.y;
          cur.z += sum.z;
          cur.w += sum.w;
          *d = cur;
        }
      }
    }
    if (last) {
      // 7. epilogue of the tile: own rows to smem, then four threads per row
      if (t < rows * RB / 16) {
        const int rr = (t * 16) / RB, part = ((t * 16) % RB) / 16;
        reinterpret_cast<uint4*>(sm.stile + rr * SROW)[part] = own;
      }
      __syncthreads();
      float o[4];
      if (row < rows) {
        float h[16], ag[16];
        unstage_row<HT>(sm.stile, row, h);
#pragma unroll
        for (int k = 0; k < 16; ++k) ag[k] = sm.agg[row * 20 + k];
        tma_layer_q<HT, FORM>(h, ag, lw, qq, o);
      }
      __syncthreads();  // every thread has read its h and aggregate
      if constexpr (!DEC) {
        if (row < rows) {
          if constexpr (sizeof(HT) == 4) {
            reinterpret_cast<float4*>(sm.stile + row * SROW)[qq] = make_float4(o[0], o[1], o[2], o[3]);
          } else {
            reinterpret_cast<uint2*>(sm.stile + row * SROW)[qq] =
                make_uint2(pack_bf16x2(o[0], o[1]), pack_bf16x2(o[2], o[3]));
          }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) sm.agg[row * 20 + 4 * qq + k] = 0.0f;  // for the next tile
        __syncthreads();
        {
          constexpr int V16 = RB / 16;
          uint4* gb = reinterpret_cast<uint4*>(Hout + (size_t)r0 * 16);
          for (int k = t; k < rows * V16; k += TM_THREADS)
            gb[k] = reinterpret_cast<const uint4*>(sm.stile + (k / V16) * SROW)[k % V16];
        }
      } else {
        if (row < rows) {
#pragma unroll
          for (int k = 0; k < 4; ++k) sm.agg[row * 20 + 4 * qq + k] = o[k];
        }
        __syncthreads();
        if (row < rows) {
          float full[16];
#pragma unroll
          for (int k = 0; k < 16; ++k) full[k] = sm.agg[row * 20 + k];
          sm.zpart[row][qq] = tma_decode_q(full, dw, qq);
        }
        __syncthreads();
        if (row < rows && qq == 0) {
          float* z = static_cast<float*>(tma_colptr(zp));
          z[r0 + row] = ((((dw.b2 + sm.zpart[row][0]) + sm.zpart[row][1]) + sm.zpart[row][2]) + sm.zpart[row][3]) *
                        s_back;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) sm.agg[row * 20 + 4 * qq + k] = 0.0f;  // for the next tile
      }
    }
    __syncthreads();  // the stage, the partials and the aggregate are free again
  }
  pdl_release();
}

// ------------------------------------------------------------------ host side

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// The tensor map of an [n][16] hidden block: a box of one row of 16 values.
template <class HT>
static int encode_hidden_map(CUtensorMap* m, const HT* H, int n) {
  auto enc = tensor_map_encoder();
  GNP_REQUIRE(enc, "k_gconv_tma: cuTensorMapEncodeTiled is not available");
  GNP_REQUIRE((reinterpret_cast<uintptr_t>(H) & 15) == 0, "k_gconv_tma: hidden block not 16-byte aligned");
  const cuuint64_t dims[2] = {16, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)HTraits<HT>::ROW_BYTES};
  const cuuint32_t box[2] = {16, 1};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r =
      enc(m, sizeof(HT) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 2,
          const_cast<HT*>(H), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  GNP_REQUIRE(r == CUDA_SUCCESS, "k_gconv_tma: cuTensorMapEncodeTiled failed (%d)", (int)r);
  return GNP_OK;
}

static int sm_count() {
  static int c = 0;
  if (!c) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c <= 0) c = NUM_SMS_GB300;
  }
  return c;
}

void tma_sched_free(TmaSched& s) {
  dev_free(s.items);
  dev_free(s.off);
  s = TmaSched{};
}

// Items of `grid` blocks for chunks of at most cap nonzeros: tiles go to the least-loaded
// block in decreasing order of nonzeros (+32 for the epilogue); each block then takes its
// tiles in increasing order, split into chunks.
int tma_sched_build(const std::vector<int>& rp, int n, int cap, int grid, TmaSched& out) {
  const int ntiles = (n + TM_ROWS - 1) / TM_ROWS;
  std::vector<long long> wt(ntiles);
  for (int t = 0; t < ntiles; ++t) {
    const int r0 = t * TM_ROWS, r1 = std::min(n, r0 + TM_ROWS);
    wt[t] = (long long)(rp[r1] - rp[r0]) + 32;
  }
  std::vector<int> order(ntiles);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return wt[x] > wt[y]; });
  using P = std::pair<long long, int>;
  std::priority_queue<P, std::vector<P>, std::greater<P>> heap;
  for (int b = 0; b < grid; ++b) heap.push({0, b});
  std::vector<std::vector<int>> per(grid);
  for (int t : order) {
    P p = heap.top();
    heap.pop();
    per[p.second].push_back(t);
    heap.push({p.first + wt[t], p.second});
  }
  std::vector<int4> items;
  std::vector<int> off(grid + 1, 0);
  for (int b = 0; b < grid; ++b) {
    std::sort(per[b].begin(), per[b].end());
    for (int t : per[b]) {
      const int r0 = t * TM_ROWS, r1 = std::min(n, r0 + TM_ROWS);
      const int e0 = rp[r0], e1 = rp[r1];
      const int nch = std::max(1, (e1 - e0 + cap - 1) / cap);
      for (int k = 0; k < nch; ++k) {
        const int a = e0 + k * cap, z = std::min(e1, a + cap);
        items.push_back(make_int4(t, a, std::max(a, z), (k == 0 ? 1 : 0) | (k == nch - 1 ? 2 : 0)));
      }
    }
    off[b + 1] = (int)items.size();
  }
  tma_sched_free(out);
  GNP_TRY(dev_alloc(&out.items, items.size()));
  GNP_TRY(dev_alloc(&out.off, off.size()));
  GNP_TRY_CUDA(cudaMemcpy(out.items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
  GNP_TRY_CUDA(cudaMemcpy(out.off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
  out.grid = grid;
  out.cap = cap;
  out.nitems = (long long)items.size();
  return GNP_OK;
}

template <class HT>
static int tma_smem_bytes() {
  return (int)sizeof(TmaSmem<HT>) + 128;
}

template <class HT, int FORM, bool DEC>
static int tma_attrs() {
  static bool done = false;
  if (done) return GNP_OK;
  GNP_TRY_CUDA(cudaFuncSetAttribute(k_gconv_tma<HT, FORM, DEC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    tma_smem_bytes<HT>()));
  done = true;
  return GNP_OK;
}

bool tma_active(const gnp_mat* A) {
  if (!A->tma_built) return false;
  const char* e = getenv("GNP_GCONV_TMA");
  return e && e[0] == '1';
}

int tma_prepare(gnp_mat* A) {
  if (A->tma_built) return GNP_OK;
  std::vector<int> h(A->n + 1);
  GNP_TRY_CUDA(cudaMemcpy(h.data(), A->rp, sizeof(int) * (A->n + 1), cudaMemcpyDeviceToHost));
  GNP_TRY(tma_sched_build(h, A->n, TmaCap<float>::CAP, sm_count(), A->tma[0]));
  GNP_TRY(tma_sched_build(h, A->n, TmaCap<uint16_t>::CAP, sm_count(), A->tma[1]));
  GNP_TRY((tma_attrs<float, GNP_LAYER_PAPER, false>()));
  GNP_TRY((tma_attrs<float, GNP_LAYER_PAPER, true>()));
  GNP_TRY((tma_attrs<float, GNP_LAYER_RESID, false>()));
  GNP_TRY((tma_attrs<float, GNP_LAYER_RESID, true>()));
  GNP_TRY((tma_attrs<uint16_t, GNP_LAYER_PAPER, false>()));
  GNP_TRY((tma_attrs<uint16_t, GNP_LAYER_PAPER, true>()));
  GNP_TRY((tma_attrs<uint16_t, GNP_LAYER_RESID, false>()));
  GNP_TRY((tma_attrs<uint16_t, GNP_LAYER_RESID, true>()));
  A->tma_built = true;
  return GNP_OK;
}

template <class HT, int FORM, bool DEC>
static int tma_launch_t(const gnp_mat* A, const float* valhat, const HT* Hin, HT* Hout, ColPtr zp, const double* tau,
                        double sqrt_n, const int* ctl, const LayerW& lw, const DecW& dw, cudaStream_t st) {
  const TmaSched& s = A->tma[sizeof(HT) == 4 ? 0 : 1];
  CUtensorMap m;
  GNP_TRY(encode_hidden_map<HT>(&m, Hin, A->n));
  GNP_TRY_CUDA(launch_pdl(k_gconv_tma<HT, FORM, DEC>, s.grid, tma_smem_bytes<HT>(), st, m,
                          (const int4*)s.items, (const int*)s.off, (const int*)A->rp, (const int*)A->col, valhat, Hin,
                          Hout, zp, tau, sqrt_n, A->n, ctl, lw, dw));
  return GNP_OK;
}

template <class HT>
int tma_layer_launch(const gnp_mat* A, int form, bool dec, const float* valhat, const HT* Hin, HT* Hout, ColPtr zp,
                     const double* tau, double sqrt_n, const int* ctl, const LayerW& lw, const DecW& dw,
                     cudaStream_t st) {
  GNP_REQUIRE(A->tma_built, "k_gconv_tma: schedule not built");
  if (form == GNP_LAYER_PAPER)
    return dec ? tma_launch_t<HT, GNP_LAYER_PAPER, true>(A, valhat, Hin, Hout, zp, tau, sqrt_n, ctl, lw, dw, st)
               : tma_launch_t<HT, GNP_LAYER_PAPER, false>(A, valhat, Hin, Hout, zp, tau, sqrt_n, ctl, lw, dw, st);
  return dec ? tma_launch_t<HT, GNP_LAYER_RESID, true>(A, valhat, Hin, Hout, zp, tau, sqrt_n, ctl, lw, dw, st)
             : tma_launch_t<HT, GNP_LAYER_RESID, false>(A, valhat, Hin, Hout, zp, tau, sqrt_n, ctl, lw, dw, st);
}

template int tma_layer_launch<float>(const gnp_mat*, int, bool, const float*, const float*, float*, ColPtr,
                                     const double*, double, const int*, const LayerW&, const DecW&, cudaStream_t);
template int tma_layer_launch<uint16_t>(const gnp_mat*, int, bool, const float*, const uint16_t*, uint16_t*, ColPtr,
                                        const double*, double, const int*, const LayerW&, const DecW&, cudaStream_t);

}  // namespace gnp

extern "C" int gnp_kernel_faults(int reset) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, gnp::g_kernel_faults, sizeof(int)) != cudaSuccess) return -1;
  if (reset) {
    const int z = 0;
    if (cudaMemcpyToSymbol(gnp::g_kernel_faults, &z, sizeof(int)) != cudaSuccess) return -1;
  }
  return v;
}
