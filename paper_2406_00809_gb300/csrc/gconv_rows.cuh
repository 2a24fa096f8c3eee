// Hidden-row layouts and the per-row Res-GCONV / decoder arithmetic shared by the layer
// kernels (gconv.cu, gconv_tma.cu).
#pragma once

#include "gconv_common.cuh"
#include "internal.h"

namespace gnp {

// ---------------------------------------------------------------- traits

struct TrF32 {  // float32 hidden block: 4 lanes x float4 per 64-byte row
  static constexpr int G = 4, NV = 4, STRIDE = 20;
  using acc = float;
  using val_t = float;
  using x_t = float;
  __device__ __forceinline__ static void load(const float* X, int c, int q, float (&h)[4]) {
    float4 t = __ldg(reinterpret_cast<const float4*>(X + (size_t)c * 16) + q);
    h[0] = t.x; h[1] = t.y; h[2] = t.z; h[3] = t.w;
  }
};

struct TrBF16 {  // bfloat16 hidden block: 2 lanes x 8 values (16 bytes) per 32-byte row
  static constexpr int G = 2, NV = 8, STRIDE = 20;
  using acc = float;
  using val_t = float;
  using x_t = uint16_t;
  __device__ __forceinline__ static void load(const uint16_t* X, int c, int q, float (&h)[8]) {
    uint4 t = __ldg(reinterpret_cast<const uint4*>(X + (size_t)c * 16) + q);
    h[0] = bf16lo(t.x); h[1] = bf16hi(t.x); h[2] = bf16lo(t.y); h[3] = bf16hi(t.y);
    h[4] = bf16lo(t.z); h[5] = bf16hi(t.z); h[6] = bf16lo(t.w); h[7] = bf16hi(t.w);
  }
};

template <class HT> struct HTraits;
template <> struct HTraits<float> {
  using TR = TrF32;
  static constexpr int ROW_BYTES = 64;
  static constexpr int SROW = 20;  // smem staging stride in floats
};
template <> struct HTraits<uint16_t> {
  using TR = TrBF16;
  static constexpr int ROW_BYTES = 32;
  static constexpr int SROW = 12;  // smem staging stride in 32-bit words (48 bytes)
};


// Store one hidden row per thread (float32 values) to a smem staging tile, then the
// block writes the tile to global memory with coalesced 16-byte stores.
template <class HT>
__device__ __forceinline__ void stage_row(uint32_t* stile, int t, const float (&o)[16]) {
  if constexpr (sizeof(HT) == 4) {
    float4* d = reinterpret_cast<float4*>(stile + t * HTraits<HT>::SROW);
    d[0] = make_float4(o[0], o[1], o[2], o[3]);
    d[1] = make_float4(o[4], o[5], o[6], o[7]);
    d[2] = make_float4(o[8], o[9], o[10], o[11]);
    d[3] = make_float4(o[12], o[13], o[14], o[15]);
  } else {
    uint4* d = reinterpret_cast<uint4*>(stile + t * HTraits<HT>::SROW);
    d[0] = make_uint4(pack_bf16x2(o[0], o[1]), pack_bf16x2(o[2], o[3]), pack_bf16x2(o[4], o[5]),
                      pack_bf16x2(o[6], o[7]));
    d[1] = make_uint4(pack_bf16x2(o[8], o[9]), pack_bf16x2(o[10], o[11]),
                      pack_bf16x2(o[12], o[13]), pack_bf16x2(o[14], o[15]));
  }
}

template <class HT>
__device__ __forceinline__ void unstage_row(const uint32_t* stile, int t, float (&o)[16]) {
  if constexpr (sizeof(HT) == 4) {
    const float4* s = reinterpret_cast<const float4*>(stile + t * HTraits<HT>::SROW);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float4 v = s[k];
      o[4 * k] = v.x; o[4 * k + 1] = v.y; o[4 * k + 2] = v.z; o[4 * k + 3] = v.w;
    }
  } else {
    const uint4* s = reinterpret_cast<const uint4*>(stile + t * HTraits<HT>::SROW);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      uint4 v = s[k];
      o[8 * k + 0] = bf16lo(v.x); o[8 * k + 1] = bf16hi(v.x);
      o[8 * k + 2] = bf16lo(v.y); o[8 * k + 3] = bf16hi(v.y);
      o[8 * k + 4] = bf16lo(v.z); o[8 * k + 5] = bf16hi(v.z);
      o[8 * k + 6] = bf16lo(v.w); o[8 * k + 7] = bf16hi(v.w);
    }
  }
}

// Outputs [K0, K0+OPT) of one row: ReLU(h U + agg W) (paper) or h + ReLU(agg W).  Two
// outputs per paired multiply-add (each lane an fmaf, inputs in the same order).
template <int FORM, int K0, int OPT>
__device__ __forceinline__ void layer_part(const float (&h)[16], const float (&agg)[16],
                                           const LayerW& lw, float (&o)[OPT]) {
#pragma unroll
  for (int k = 0; k < OPT; ++k) o[k] = 0.0f;
#pragma unroll
  for (int c = 0; c < 16; ++c) {
#pragma unroll
    for (int k = 0; k < OPT; k += 2)
      ffma2(o[k], o[k + 1], agg[c], agg[c], lw.W[c * 16 + K0 + k], lw.W[c * 16 + K0 + k + 1]);
  }
  if (FORM == GNP_LAYER_PAPER) {
#pragma unroll
    for (int c = 0; c < 16; ++c) {
#pragma unroll
      for (int k = 0; k < OPT; k += 2)
        ffma2(o[k], o[k + 1], h[c], h[c], lw.U[c * 16 + K0 + k], lw.U[c * 16 + K0 + k + 1]);
    }
#pragma unroll
    for (int k = 0; k < OPT; ++k) o[k] = fmaxf(o[k], 0.0f);
  } else {
#pragma unroll
    for (int k = 0; k < OPT; ++k) o[k] = h[K0 + k] + fmaxf(o[k], 0.0f);
  }
}

// Decoder hidden units [K0, K0+KC) of one row: sum_k w2_k ReLU(D1^T o + e1)_k.
template <int K0, int KC>
__device__ __forceinline__ float decode_part(const float (&o)[16], const DecW& dw) {
  float z = 0.0f;
#pragma unroll
  for (int k = K0; k < K0 + KC; ++k) {
    float a = dw.b1[k];
#pragma unroll
    for (int c = 0; c < 16; ++c) a = fmaf(o[c], dw.W1[c * 32 + k], a);
    z = fmaf(fmaxf(a, 0.0f), dw.W2[k], z);
  }
  return z;
}

// Decoder for one row: (w2^T ReLU(D1^T h + e1) + e2) * back.
__device__ __forceinline__ float decode_row(const float (&o)[16], const DecW& dw) {
  float z = dw.b2;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    float a = dw.b1[k];
#pragma unroll
    for (int c = 0; c < 16; ++c) a = fmaf(o[c], dw.W1[c * 32 + k], a);
    z = fmaf(fmaxf(a, 0.0f), dw.W2[k], z);
  }
  return z;
}

}  // namespace gnp
