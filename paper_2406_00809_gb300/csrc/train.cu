// GNP training (Sec. 2.2, Sec. 3 "Hyperparameters"): batched forward with saved
// activations, l1 residual loss, hand-written backward, Adam, best-loss snapshot, and
// the training-pair sampler (half Eq. 5 Arnoldi samples, half N(0, I)).
//
// Batched layout: B right-hand sides node-major, element (i, k) at i*B + k; hidden
// blocks (i, k, c) at (i*B + k)*16 + c, so one CSR gather of node j moves the whole
// contiguous B x 16 block.  R = n*B "rows" for the row-wise kernels.
//
// Backward (App. E: the same products with A_hat and with tall n-row matrices):
//   decoder:  do = dz * tau_k/sqrt(n); dc1 = (do w2^T) * 1[c1 > 0]; dH^L = dc1 D1^T
//   layer l:  Gp = G * 1[pre > 0]; Y = Gp W^T; dX = (Gp U^T | G) + A_hat^T Y, the last
//             product a gather through the canonical CSC of A_hat;
//             dU = sum X^T Gp, dW = sum (A_hat X)^T Gp
//   encoder:  da1 = (dH^0 W2^T) * 1[a1 > 0]; dW2 = sum r1^T dH^0, dW1 = sum u da1
// Weight gradients are column-sum reductions over the R rows (k_wgrad): fixed row
// chunks per block in float32, then a fixed-order float64 sum over blocks.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace gnp {

int arnoldi_basis(gnp_mat* A, const double* v1, int m, double* V_out, double* Hbar_host,
                  int* k_out, cudaStream_t st);  // krylov.cu

struct TrainState {
  int n = 0, B = 0, L = 0;
  long long R = 0;
  // forward activations
  float* u = nullptr;      // [R]
  double* tau = nullptr;   // [B]
  float* Hs = nullptr;     // [(L+1) * R * 16]
  float* AGG = nullptr;    // [L * R * 16]
  float* z = nullptr;      // [R]
  // backward scratch
  float* g16a = nullptr;   // [R*16]
  float* g16b = nullptr;   // [R*16]
  float* y16 = nullptr;    // [R*16]
  float* gp16 = nullptr;   // [R*16]
  float* s32a = nullptr;   // [R*32]
  float* s32b = nullptr;   // [R*32]
  float* r1 = nullptr;     // [R]   (do)
  float* grad = nullptr;   // [count]
  float* partials = nullptr;  // wgrad partials
  int part_cap = 0;
  RedScratch red;          // column norms / loss
  // batch buffers
  float* xb = nullptr;     // [R]
  float* bb = nullptr;     // [R]
  float* rr = nullptr;     // [R]
  float* dz = nullptr;     // [R]
  // optimiser
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* loss = nullptr;       // device scalar: last loss
  float* best_loss = nullptr;  // device scalar
  int* adam_t = nullptr;       // device step counter
  int step = 0;                // host step counter of gnp_train_step
  // sampler
  bool sampler_ready = false;
  int mA = 0;                  // Arnoldi columns actually used
  double* V = nullptr;         // [n*(mA+1)]
  double* Q = nullptr;         // [mA*mA] Z S^-1, row-major
  double* C = nullptr;         // [mA*B]
  double* Hbar = nullptr;      // device copy of H_bar / gamma, column-major (mA+1) x mA
};

void train_free(TrainState* t) {
  if (!t) return;
  float* fs[] = {t->u, t->Hs, t->AGG, t->z, t->g16a, t->g16b, t->y16, t->gp16, t->s32a, t->s32b,
                 t->r1, t->grad, t->partials, t->xb, t->bb, t->rr, t->dz, t->adam_m, t->adam_v, t->loss,
                 t->best_loss};
  for (float* p : fs) if (p) cudaFree(p);
  if (t->tau) cudaFree(t->tau);
  if (t->adam_t) cudaFree(t->adam_t);
  if (t->V) cudaFree(t->V);
  if (t->Q) cudaFree(t->Q);
  if (t->C) cudaFree(t->C);
  if (t->Hbar) cudaFree(t->Hbar);
  red_free(t->red);
  delete t;
}

void train_reset(TrainState* t) {
  if (!t) return;
  const int cnt = weight_count(t->L);
  cudaMemset(t->adam_m, 0, sizeof(float) * cnt);
  cudaMemset(t->adam_v, 0, sizeof(float) * cnt);
  cudaMemset(t->adam_t, 0, sizeof(int));
  const float inf = INFINITY;
  cudaMemcpy(t->best_loss, &inf, sizeof(float), cudaMemcpyHostToDevice);
  t->step = 0;
}

__global__ void k_gather_vals(const float* __restrict__ v, const int* __restrict__ perm, long long nnz,
                              float* __restrict__ out);

static int train_ensure(gnp_model* M, int B) {
  TrainState* t = M->train;
  if (t && t->B == B) return GNP_OK;
  GNP_REQUIRE(B >= 4 && B <= GNP_MAX_BATCH && (B & (B - 1)) == 0,
              "training batch %d must be a power of two in [4, %d]", B, GNP_MAX_BATCH);
  GNP_TRY(mat_build_csc(M->A, 0));
  if (!M->valhat_t) {
    GNP_TRY(dev_alloc(&M->valhat_t, (size_t)std::max<long long>(M->A->nnz, 1)));
    if (M->A->nnz > 0) {
      k_gather_vals<<<4 * NUM_SMS_GB300, 256>>>(M->valhat, M->A->csc.perm, M->A->nnz, M->valhat_t);
      GNP_TRY(check_launch("k_gather_vals"));
      GNP_TRY_CUDA(cudaDeviceSynchronize());
    }
  }
  bool keep_opt = t != nullptr;
  TrainState* nt = new TrainState();
  const int n = M->A->n, L = M->cfg.L;
  const long long R = (long long)n * B;
  nt->n = n;
  nt->B = B;
  nt->L = L;
  nt->R = R;
  const int cnt = weight_count(L);
  int s = GNP_OK;
  do {
    if ((s = dev_alloc(&nt->u, (size_t)R)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->tau, (size_t)B)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->Hs, (size_t)(L + 1) * R * 16)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->AGG, (size_t)std::max(L, 1) * R * 16)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->z, (size_t)R)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->g16a, (size_t)R * 16)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->g16b, (size_t)R * 16)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->y16, (size_t)R * 16)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->gp16, (size_t)R * 16)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->s32a, (size_t)R * 32)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->s32b, (size_t)R * 32)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->r1, (size_t)R)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->grad, (size_t)cnt)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->xb, (size_t)R)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->bb, (size_t)R)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->rr, (size_t)R)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->dz, (size_t)R)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->adam_m, (size_t)cnt)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->adam_v, (size_t)cnt)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->loss, 1)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->best_loss, 1)) != GNP_OK) break;
    if ((s = dev_alloc(&nt->adam_t, 1)) != GNP_OK) break;
    if ((s = red_alloc(nt->red, 4 * NUM_SMS_GB300, GNP_MAX_BATCH)) != GNP_OK) break;
  } while (0);
  if (s != GNP_OK) {
    train_free(nt);
    return s;
  }
  if (keep_opt) {
    // a new batch size keeps the optimiser state and the sampler
    cudaMemcpy(nt->adam_m, t->adam_m, sizeof(float) * cnt, cudaMemcpyDeviceToDevice);
    cudaMemcpy(nt->adam_v, t->adam_v, sizeof(float) * cnt, cudaMemcpyDeviceToDevice);
    cudaMemcpy(nt->adam_t, t->adam_t, sizeof(int), cudaMemcpyDeviceToDevice);
    cudaMemcpy(nt->best_loss, t->best_loss, sizeof(float), cudaMemcpyDeviceToDevice);
    nt->step = t->step;
    std::swap(nt->V, t->V);
    std::swap(nt->Q, t->Q);
    std::swap(nt->Hbar, t->Hbar);
    nt->mA = t->mA;
    nt->sampler_ready = t->sampler_ready;
    train_free(t);
  } else {
    train_reset(nt);
  }
  M->train = nt;
  return GNP_OK;
}

// ---------------------------------------------------------------- Philox / Box-Muller

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 multiplies with
// M0 = 0xD2511F53 (on c0) and M1 = 0xCD9E8D57 (on c2), key bumped by (0x9E3779B9,
// 0xBB67AE85) between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Uniform in (0,1) with at most 24 significant bits: ((r >> 9) + 0.5) * 2^-23.
__device__ __forceinline__ float uniform24(uint32_t r) {
  return ((float)(r >> 9) + 0.5f) * 0x1p-23f;
}

// Element e of stream (seed, step, stream): output e%4 of call e/4, Box-Muller pairs
// (w0, w1) -> [rho cos, rho sin], (w2, w3) -> [rho cos, rho sin].
__device__ __forceinline__ float philox_normal(unsigned long long e, unsigned long long seed,
                                               uint32_t step, uint32_t stream) {
  const unsigned long long idx = e >> 2;
  const uint4 w = philox4x32_10(make_uint4((uint32_t)idx, (uint32_t)(idx >> 32), step, stream),
                                (uint32_t)seed, (uint32_t)(seed >> 32));
  const int lane = (int)(e & 3);
  const uint32_t ra = lane < 2 ? w.x : w.z;
  const uint32_t rb = lane < 2 ? w.y : w.w;
  const float rho = sqrtf(-2.0f * logf(uniform24(ra)));
  float sn, cs;
  sincospif(2.0f * uniform24(rb), &sn, &cs);
  return (lane & 1) ? rho * sn : rho * cs;
}

constexpr uint32_t STREAM_X = 1, STREAM_EPS = 2, STREAM_V1 = 3;

// ---------------------------------------------------------------- generic kernels

// Y[i] = alpha * sum_e vals[e] X[idx[e]] + beta * Yadd[i], for node blocks of W4
// acc += sum_{e in [e0, e1)} vals[e] X[idx[e]] for one node's row of W4 float4: lane
// `lane` of the node's lane group owns float4s lane, lane+LPN, ... (KM of them, W4 =
// LPN*KM or less).  Two nonzeros are in flight at a time; the additions keep the order of
// the nonzeros.
template <int LPN, int KM>
__device__ __forceinline__ void gather_rows(const int* __restrict__ idx, const float* __restrict__ vals,
                                            const float4* __restrict__ X, int W4, int lane, int e0, int e1,
                                            float4 (&acc)[KM]) {
  int e = e0;
  for (; e + 2 <= e1; e += 2) {
    const int j0 = __ldg(idx + e), j1 = __ldg(idx + e + 1);
    const float a0 = __ldg(vals + e), a1 = __ldg(vals + e + 1);
    const float4* x0 = X + (size_t)j0 * W4;
    const float4* x1 = X + (size_t)j1 * W4;
    float4 v0[KM], v1[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      const int f = lane + LPN * k;
      if (f < W4) {
        v0[k] = __ldg(x0 + f);
        v1[k] = __ldg(x1 + f);
      }
    }
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      const int f = lane + LPN * k;
      if (f < W4) {
        acc[k].x = fmaf(a1, v1[k].x, fmaf(a0, v0[k].x, acc[k].x));
        acc[k].y = fmaf(a1, v1[k].y, fmaf(a0, v0[k].y, acc[k].y));
        acc[k].z = fmaf(a1, v1[k].z, fmaf(a0, v0[k].z, acc[k].z));
        acc[k].w = fmaf(a1, v1[k].w, fmaf(a0, v0[k].w, acc[k].w));
      }
    }
  }
  if (e < e1) {
    const int j = __ldg(idx + e);
    const float a = __ldg(vals + e);
    const float4* xj = X + (size_t)j * W4;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      const int f = lane + LPN * k;
      if (f < W4) {
        const float4 v = __ldg(xj + f);
        acc[k].x = fmaf(a, v.x, acc[k].x);
        acc[k].y = fmaf(a, v.y, acc[k].y);
        acc[k].z = fmaf(a, v.z, acc[k].z);
        acc[k].w = fmaf(a, v.w, acc[k].w);
      }
    }
  }
}

// float4 values (warp per node).  With (ptr, idx, vals) the CSR of A_hat this is
// A_hat X; with the canonical CSC and the CSC-ordered values it is A_hat^T X.
template <int LPN, int KM>
__global__ void __launch_bounds__(256)
k_spmm_nodes(const int* __restrict__ ptr, const int* __restrict__ idx, const float* __restrict__ vals,
             const float4* __restrict__ X, int n, int W4, float alpha, const float4* __restrict__ Yadd,
             float beta, float4* __restrict__ Y) {
  constexpr int NPW = 32 / LPN;  // nodes per warp
  const int lane = threadIdx.x & (LPN - 1);
  const int grp = (threadIdx.x & 31) / LPN;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int i0 = warp * NPW; i0 < n; i0 += nwarps * NPW) {
    const int i = i0 + grp;
    if (i >= n) continue;
    float4 acc[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    gather_rows<LPN, KM>(idx, vals, X, W4, lane, ptr[i], ptr[i + 1], acc);
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      const int f = lane + LPN * k;
      if (f < W4) {
        float4 o = make_float4(alpha * acc[k].x, alpha * acc[k].y, alpha * acc[k].z, alpha * acc[k].w);
        if (Yadd) {
          const float4 a = Yadd[(size_t)i * W4 + f];
          o.x = fmaf(beta, a.x, o.x);
          o.y = fmaf(beta, a.y, o.y);
          o.z = fmaf(beta, a.z, o.z);
          o.w = fmaf(beta, a.w, o.w);
        }
        Y[(size_t)i * W4 + f] = o;
      }
    }
  }
}

// Y = alpha A X (+ beta Yadd) for node rows of W4 float4 (W4 = 1..256): a lane group per
// node, LPN = min(W4, 32) lanes, several nodes per warp when the rows are narrow.
static int spmm_nodes(const int* ptr, const int* idx, const float* vals, const float4* X, int n, int W4,
                      float alpha, const float4* Yadd, float beta, float4* Y, cudaStream_t st) {
  const int lpn = W4 >= 32 ? 32 : W4;
  const int npw = 32 / lpn;
  const int grid = std::max(1, std::min((n + 8 * npw - 1) / (8 * npw), 16 * NUM_SMS_GB300));
#define GNP_SPMM(L, K) k_spmm_nodes<L, K><<<grid, 256, 0, st>>>(ptr, idx, vals, X, n, W4, alpha, Yadd, beta, Y)
  if (W4 <= 1) GNP_SPMM(1, 1);
  else if (W4 <= 2) GNP_SPMM(2, 1);
  else if (W4 <= 4) GNP_SPMM(4, 1);
  else if (W4 <= 8) GNP_SPMM(8, 1);
  else if (W4 <= 16) GNP_SPMM(16, 1);
  else if (W4 <= 32) GNP_SPMM(32, 1);
  else if (W4 <= 64) GNP_SPMM(32, 2);
  else if (W4 <= 128) GNP_SPMM(32, 4);
  else GNP_SPMM(32, 8);
#undef GNP_SPMM
  return check_launch("k_spmm_nodes");
}

// Values of A_hat in the CSC order (perm[k] = CSR position of CSC entry k).
__global__ void k_gather_vals(const float* __restrict__ v, const int* __restrict__ perm, long long nnz,
                              float* __restrict__ out) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz;
       k += (long long)gridDim.x * blockDim.x)
    out[k] = v[perm[k]];
}

// tau_k = ||b[:, k]||_2 for the B columns of a node-major batch (B divides 256).
__global__ void __launch_bounds__(256)
k_col_norms(const float* __restrict__ b, long long R, int B, double* __restrict__ partials,
            unsigned* counter, double* __restrict__ tau) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < R;
       e += (long long)gridDim.x * blockDim.x) {
    const double v = b[e];
    acc += v * v;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  if ((int)threadIdx.x < B) {
    double t = 0.0;
    for (int k = threadIdx.x; k < 256; k += B) t += sh[k];
    partials[(size_t)blockIdx.x * B + threadIdx.x] = t;
  }
  if (last_block_arrive(counter)) {
    __shared__ double tot[GNP_MAX_BATCH];
    reduce_partials(partials, gridDim.x, B, tot);
    if ((int)threadIdx.x < B) tau[threadIdx.x] = sqrt(tot[threadIdx.x]);
    if (threadIdx.x == 0) *counter = 0;
  }
}

// tau_k = sqrt(n) for every column: the ablation without the scaling s makes both
// factors of Eq. 8 one.
__global__ void k_fill_tau(double* __restrict__ tau, int B, double sqrt_n) {
  for (int k = threadIdx.x; k < B; k += blockDim.x) tau[k] = sqrt_n;
}

// loss = mean |r| over R entries; r <- sign(r) in place (sign(0) = 0).
__global__ void __launch_bounds__(256)
k_l1(float* __restrict__ r, long long R, double* __restrict__ partials, unsigned* counter,
     float* __restrict__ loss) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < R;
       e += (long long)gridDim.x * blockDim.x) {
    const float v = r[e];
    acc += fabs((double)v);
    r[e] = (v > 0.f) ? 1.f : ((v < 0.f) ? -1.f : 0.f);
  }
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
  if (last_block_arrive(counter)) {
    __shared__ double tot[1];
    reduce_partials(partials, gridDim.x, 1, tot);
    if (threadIdx.x == 0) {
      *loss = (float)(tot[0] / (double)R);
      *counter = 0;
    }
  }
}

// ---------------------------------------------------------------- forward kernels

// u = (sqrt(n)/tau_k) b; H0 = W2^T ReLU(W1 u + b1) + b2 (thread per row).
__global__ void __launch_bounds__(256)
k_enc_batch(const float* __restrict__ b, const double* __restrict__ tau, long long R, int B, double sqrt_n,
            const float* __restrict__ w, float* __restrict__ u_out, float* __restrict__ H0) {
  __shared__ float sw[ENC_COUNT];
  for (int k = threadIdx.x; k < ENC_COUNT; k += blockDim.x) sw[k] = w[k];
  __syncthreads();
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < R;
       r += (long long)gridDim.x * blockDim.x) {
    const double tv = tau[r % B];
    const float u = (float)(tv > 0.0 ? b[r] * (sqrt_n / tv) : 0.0);
    u_out[r] = u;
    float h[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) h[c] = sw[ENC_B2 + c];
    for (int k = 0; k < 32; ++k) {
      const float a = fmaxf(fmaf(u, sw[ENC_W1 + k], sw[ENC_B1 + k]), 0.0f);
#pragma unroll
      for (int c = 0; c < 16; ++c) h[c] = fmaf(a, sw[ENC_W2 + k * 16 + c], h[c]);
    }
    float4* o = reinterpret_cast<float4*>(H0 + r * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = make_float4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
  }
}

// One Res-GCONV layer on the batch: AGG = A_hat X (saved), Out = layer(X, AGG).
// Warp per node (gather of the node block), then lane per batch column.
template <int FORM, int B>
__global__ void __launch_bounds__(256)
k_layer_batch(const int* __restrict__ rp, const int* __restrict__ col, const float* __restrict__ vh,
              const float* __restrict__ X, float* __restrict__ AGG, float* __restrict__ Out, int n,
              const float* __restrict__ lw) {
  constexpr int W4 = B * 4;                  // float4 per node block
  constexpr int KM = (W4 + 31) / 32;         // float4 per lane in the gather
  constexpr int P = B >= 32 ? 1 : 32 / B;    // lanes per batch column in the epilogue
  constexpr int OP = 16 / P;                 // outputs per lane
  constexpr int CPL = B > 32 ? B / 32 : 1;   // batch columns per lane
  extern __shared__ __align__(16) float smf[];
  float* sU = smf;
  float* sW = smf + 256;
  float* sblk = smf + 512;  // per warp: AGG block [B*16] then X block [B*16]
  for (int k = threadIdx.x; k < 512; k += blockDim.x) smf[k] = lw[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  float* sA = sblk + (size_t)wl * (2 * B * 16);
  float* sX = sA + B * 16;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const float4* X4 = reinterpret_cast<const float4*>(X);
  const int k0 = (lane % P) * OP;
  for (int i = warp; i < n; i += nwarps) {
    float4 acc[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    gather_rows<32, KM>(col, vh, X4, W4, lane, rp[i], rp[i + 1], acc);
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      const int f = lane + 32 * k;
      if (f < W4) {
        reinterpret_cast<float4*>(AGG)[(size_t)i * W4 + f] = acc[k];
        reinterpret_cast<float4*>(sA)[f] = acc[k];
        reinterpret_cast<float4*>(sX)[f] = __ldg(X4 + (size_t)i * W4 + f);
      }
    }
    __syncwarp();
#pragma unroll
    for (int cc = 0; cc < CPL; ++cc) {
      const int bq = lane / P + 32 * cc;
      const float* xa = sX + bq * 16;
      const float* ga = sA + bq * 16;
      float o[OP];
#pragma unroll
      for (int k = 0; k < OP; ++k) o[k] = 0.f;
#pragma unroll 4
      for (int c = 0; c < 16; ++c) {
        const float gc = ga[c];
#pragma unroll
        for (int k = 0; k < OP; ++k) o[k] = fmaf(gc, sW[c * 16 + k0 + k], o[k]);
      }
      if (FORM == GNP_LAYER_PAPER) {
#pragma unroll 4
        for (int c = 0; c < 16; ++c) {
          const float xc = xa[c];
#pragma unroll
          for (int k = 0; k < OP; ++k) o[k] = fmaf(xc, sU[c * 16 + k0 + k], o[k]);
        }
#pragma unroll
        for (int k = 0; k < OP; ++k) o[k] = fmaxf(o[k], 0.f);
      } else {
#pragma unroll
        for (int k = 0; k < OP; ++k) o[k] = xa[k0 + k] + fmaxf(o[k], 0.f);
      }
      float* out = Out + ((size_t)i * B + bq) * 16 + k0;
      if constexpr (OP >= 4) {
#pragma unroll
        for (int q = 0; q < OP / 4; ++q)
          reinterpret_cast<float4*>(out)[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
      } else {
        reinterpret_cast<float2*>(out)[0] = make_float2(o[0], o[1]);
      }
    }
    __syncwarp();
  }
}

// z = (w2^T ReLU(D1^T h + e1) + e2) * tau_k / sqrt(n) (thread per row).
__global__ void __launch_bounds__(256)
k_dec_batch(const float* __restrict__ HL, const double* __restrict__ tau, long long R, int B, double sqrt_n,
            const float* __restrict__ wd, float* __restrict__ z) {
  __shared__ float sw[DEC_COUNT];
  for (int k = threadIdx.x; k < DEC_COUNT; k += blockDim.x) sw[k] = wd[k];
  __syncthreads();
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < R;
       r += (long long)gridDim.x * blockDim.x) {
    float h[16];
    const float4* hp = reinterpret_cast<const float4*>(HL + r * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 v = hp[q];
      h[4 * q] = v.x; h[4 * q + 1] = v.y; h[4 * q + 2] = v.z; h[4 * q + 3] = v.w;
    }
    float o = sw[576];
    for (int k = 0; k < 32; ++k) {
      float a = sw[512 + k];
#pragma unroll
      for (int c = 0; c < 16; ++c) a = fmaf(h[c], sw[c * 32 + k], a);
      o = fmaf(fmaxf(a, 0.f), sw[544 + k], o);
    }
    const double tv = tau[r % B];
    z[r] = o * (float)(tv > 0.0 ? tv / sqrt_n : 0.0);
  }
}

// ---------------------------------------------------------------- backward kernels

// Decoder backward (thread per row): do, dc1 = dq * 1[c1 > 0], q = ReLU(c1) saved for
// the weight gradients, dH^L = dc1 D1^T.
__global__ void __launch_bounds__(256)
k_dec_bwd(const float* __restrict__ HL, const float* __restrict__ dz, const double* __restrict__ tau,
          long long R, int B, double sqrt_n, const float* __restrict__ wd, float* __restrict__ do_out,
          float* __restrict__ q_out, float* __restrict__ dc1_out, float* __restrict__ dH) {
  __shared__ __align__(16) float sw[DEC_COUNT + 3];
  for (int k = threadIdx.x; k < DEC_COUNT; k += blockDim.x) sw[k] = wd[k];
  __syncthreads();
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < R;
       r += (long long)gridDim.x * blockDim.x) {
    float h[16];
    const float4* hp = reinterpret_cast<const float4*>(HL + r * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 v = hp[q];
      h[4 * q] = v.x; h[4 * q + 1] = v.y; h[4 * q + 2] = v.z; h[4 * q + 3] = v.w;
    }
    const double tv = tau[r % B];
    const float dov = dz[r] * (float)(tv > 0.0 ? tv / sqrt_n : 0.0);
    do_out[r] = dov;
    float g[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) g[c] = 0.f;
    float4* qo = reinterpret_cast<float4*>(q_out + r * 32);
    float4* dco = reinterpret_cast<float4*>(dc1_out + r * 32);
    // four hidden units at a time: one 16-byte weight load serves four FMAs
#pragma unroll 2
    for (int k4 = 0; k4 < 8; ++k4) {
      float4 a = *reinterpret_cast<const float4*>(sw + 512 + 4 * k4);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const float4 w = *reinterpret_cast<const float4*>(sw + c * 32 + 4 * k4);
        a.x = fmaf(h[c], w.x, a.x);
        a.y = fmaf(h[c], w.y, a.y);
        a.z = fmaf(h[c], w.z, a.z);
        a.w = fmaf(h[c], w.w, a.w);
      }
      const float4 w2 = *reinterpret_cast<const float4*>(sw + 544 + 4 * k4);
      const float4 dc = make_float4(a.x > 0.f ? dov * w2.x : 0.f, a.y > 0.f ? dov * w2.y : 0.f,
                                    a.z > 0.f ? dov * w2.z : 0.f, a.w > 0.f ? dov * w2.w : 0.f);
      qo[k4] = make_float4(fmaxf(a.x, 0.f), fmaxf(a.y, 0.f), fmaxf(a.z, 0.f), fmaxf(a.w, 0.f));
      dco[k4] = dc;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const float4 w = *reinterpret_cast<const float4*>(sw + c * 32 + 4 * k4);
        g[c] = fmaf(dc.x, w.x, g[c]);
        g[c] = fmaf(dc.y, w.y, g[c]);
        g[c] = fmaf(dc.z, w.z, g[c]);
        g[c] = fmaf(dc.w, w.w, g[c]);
      }
    }
    float4* o = reinterpret_cast<float4*>(dH + r * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = make_float4(g[4 * q], g[4 * q + 1], g[4 * q + 2], g[4 * q + 3]);
  }
}

// Layer backward, row part: Gp = G * 1[pre > 0] (pre recomputed from X and AGG exactly
// as the forward did), Y = Gp W^T, local = Gp U^T (paper) or G (residual).  Four threads
// per row, thread j owning entries 4j..4j+3 of every output: it loads quarter j of the
// AGG, X and G rows, takes the other quarters of AGG and X from its quad with shuffles,
// forms its four pre-activations from a 16 x 4 slice of W and of U, its quarter of Gp,
// gathers the other three quarters of Gp from its quad, and forms entries 4j..4j+3 of Y
// and local from the same slices of W^T and U^T (kept transposed in shared memory, so
// every 16-byte weight load of a quad is a broadcast without bank conflicts).
template <int FORM>
__global__ void __launch_bounds__(256)
k_layer_bwd_rows(const float* __restrict__ X, const float* __restrict__ AGG, const float* __restrict__ G,
                 long long R, const float* __restrict__ lw, float* __restrict__ Gp_out,
                 float* __restrict__ Y_out, float* __restrict__ local_out) {
  __shared__ __align__(16) float sU[256], sW[256], sUt[256], sWt[256];
  for (int k = threadIdx.x; k < 256; k += blockDim.x) {
    const int c = k >> 4, o = k & 15;
    sU[k] = lw[k];
    sW[k] = lw[256 + k];
    sUt[o * 16 + c] = lw[k];
    sWt[o * 16 + c] = lw[256 + k];
  }
  __syncthreads();
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int j = (int)(tid & 3);
  const int qbase = (threadIdx.x & 31) & ~3;  // first lane of this quad
  // lanes past the last row stay for the shuffles with a clamped row and store nothing
  const bool ok = (tid >> 2) < R;
  const long long r = ok ? (tid >> 2) : R - 1;
  const float4* W4 = reinterpret_cast<const float4*>(sW);
  const float4* U4 = reinterpret_cast<const float4*>(sU);
  const float4* Wt4 = reinterpret_cast<const float4*>(sWt);
  const float4* Ut4 = reinterpret_cast<const float4*>(sUt);
  // each thread loads its own quarter of the AGG, X and G rows (one 16-byte load each,
  // all in flight together) and takes the other quarters from its quad
  const float4 a_own = __ldg(reinterpret_cast<const float4*>(AGG + r * 16) + j);
  const float4 x_own = FORM == GNP_LAYER_PAPER ? __ldg(reinterpret_cast<const float4*>(X + r * 16) + j)
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 g = __ldg(reinterpret_cast<const float4*>(G + r * 16) + j);
  float4 pre = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float av[4] = {__shfl_sync(0xffffffffu, a_own.x, qbase + q), __shfl_sync(0xffffffffu, a_own.y, qbase + q),
                         __shfl_sync(0xffffffffu, a_own.z, qbase + q), __shfl_sync(0xffffffffu, a_own.w, qbase + q)};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float4 w = W4[(4 * q + e) * 4 + j];
      pre.x = fmaf(av[e], w.x, pre.x);
      pre.y = fmaf(av[e], w.y, pre.y);
      pre.z = fmaf(av[e], w.z, pre.z);
      pre.w = fmaf(av[e], w.w, pre.w);
    }
  }
  if (FORM == GNP_LAYER_PAPER) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float xv[4] = {__shfl_sync(0xffffffffu, x_own.x, qbase + q),
                           __shfl_sync(0xffffffffu, x_own.y, qbase + q),
                           __shfl_sync(0xffffffffu, x_own.z, qbase + q),
                           __shfl_sync(0xffffffffu, x_own.w, qbase + q)};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float4 u = U4[(4 * q + e) * 4 + j];
        pre.x = fmaf(xv[e], u.x, pre.x);
        pre.y = fmaf(xv[e], u.y, pre.y);
        pre.z = fmaf(xv[e], u.z, pre.z);
        pre.w = fmaf(xv[e], u.w, pre.w);
      }
    }
  }
  const float4 gp = make_float4(pre.x > 0.f ? g.x : 0.f, pre.y > 0.f ? g.y : 0.f, pre.z > 0.f ? g.z : 0.f,
                                pre.w > 0.f ? g.w : 0.f);
  if (ok) reinterpret_cast<float4*>(Gp_out + r * 16)[j] = gp;
  // the whole Gp row from the quad
  float gv[16];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    gv[4 * q] = __shfl_sync(0xffffffffu, gp.x, qbase + q);
    gv[4 * q + 1] = __shfl_sync(0xffffffffu, gp.y, qbase + q);
    gv[4 * q + 2] = __shfl_sync(0xffffffffu, gp.z, qbase + q);
    gv[4 * q + 3] = __shfl_sync(0xffffffffu, gp.w, qbase + q);
  }
  float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 loc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float4 w = Wt4[k * 4 + j];  // W[4j..4j+3][k]
    y.x = fmaf(gv[k], w.x, y.x);
    y.y = fmaf(gv[k], w.y, y.y);
    y.z = fmaf(gv[k], w.z, y.z);
    y.w = fmaf(gv[k], w.w, y.w);
    if (FORM == GNP_LAYER_PAPER) {
      const float4 u = Ut4[k * 4 + j];
      loc.x = fmaf(gv[k], u.x, loc.x);
      loc.y = fmaf(gv[k], u.y, loc.y);
      loc.z = fmaf(gv[k], u.z, loc.z);
      loc.w = fmaf(gv[k], u.w, loc.w);
    }
  }
  if (ok) {
    reinterpret_cast<float4*>(Y_out + r * 16)[j] = y;
    reinterpret_cast<float4*>(local_out + r * 16)[j] = FORM == GNP_LAYER_PAPER ? loc : g;
  }
}

// The same with two rows per thread (rows r and r + 256 of a 512-row block, so that each
// load instruction of a warp is coalesced).  Every lane of a warp needs the same weight at
// the same time, so a 16-byte weight load from shared memory is one broadcast, and each
// feeds the multiply-adds of both rows: the weight bytes the shared-memory pipe delivers
// per multiply-add (what bounds these kernels) are a quarter of the quad form's and half
// of one row per thread.  The rows' AGG, X and G (then Gp, Y, local) stay in registers.
// Same arithmetic per output as the quad form (inputs in the same order): the results
// are identical.
template <int FORM>
__global__ void __launch_bounds__(256)
k_layer_bwd_row2(const float* __restrict__ X, const float* __restrict__ AGG, const float* __restrict__ G, long long R,
                 const float* __restrict__ lw, float* __restrict__ Gp_out, float* __restrict__ Y_out,
                 float* __restrict__ local_out) {
  __shared__ __align__(16) float sU[256], sW[256], sUt[256], sWt[256];
  for (int k = threadIdx.x; k < 256; k += blockDim.x) {
    const int c = k >> 4, o = k & 15;
    sU[k] = lw[k];
    sW[k] = lw[256 + k];
    sUt[o * 16 + c] = lw[k];
    sWt[o * 16 + c] = lw[256 + k];
  }
  __syncthreads();
  const long long rA = blockIdx.x * 512LL + threadIdx.x;
  if (rA >= R) return;
  const bool two = rA + 256 < R;
  const long long rB = two ? rA + 256 : rA;  // a lone last row is computed twice, stored once
  const float4* W4 = reinterpret_cast<const float4*>(sW);
  const float4* U4 = reinterpret_cast<const float4*>(sU);
  const float4* Wt4 = reinterpret_cast<const float4*>(sWt);
  const float4* Ut4 = reinterpret_cast<const float4*>(sUt);
  float a[2][16], x[2][16], g[2][16];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const long long r = h ? rB : rA;
    const float4* ap = reinterpret_cast<const float4*>(AGG + r * 16);
    const float4* xp = reinterpret_cast<const float4*>(X + r * 16);
    const float4* gq = reinterpret_cast<const float4*>(G + r * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 t = __ldg(ap + q);
      a[h][4 * q] = t.x; a[h][4 * q + 1] = t.y; a[h][4 * q + 2] = t.z; a[h][4 * q + 3] = t.w;
      const float4 u = FORM == GNP_LAYER_PAPER ? __ldg(xp + q) : make_float4(0.f, 0.f, 0.f, 0.f);
      x[h][4 * q] = u.x; x[h][4 * q + 1] = u.y; x[h][4 * q + 2] = u.z; x[h][4 * q + 3] = u.w;
      const float4 v = __ldg(gq + q);
      g[h][4 * q] = v.x; g[h][4 * q + 1] = v.y; g[h][4 * q + 2] = v.z; g[h][4 * q + 3] = v.w;
    }
  }
  float gp[2][16];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float4 pre[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const float4 w = W4[c * 4 + j];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        pre[h].x = fmaf(a[h][c], w.x, pre[h].x);
        pre[h].y = fmaf(a[h][c], w.y, pre[h].y);
        pre[h].z = fmaf(a[h][c], w.z, pre[h].z);
        pre[h].w = fmaf(a[h][c], w.w, pre[h].w);
      }
    }
    if (FORM == GNP_LAYER_PAPER) {
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const float4 u = U4[c * 4 + j];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          pre[h].x = fmaf(x[h][c], u.x, pre[h].x);
          pre[h].y = fmaf(x[h][c], u.y, pre[h].y);
          pre[h].z = fmaf(x[h][c], u.z, pre[h].z);
          pre[h].w = fmaf(x[h][c], u.w, pre[h].w);
        }
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      gp[h][4 * j] = pre[h].x > 0.f ? g[h][4 * j] : 0.f;
      gp[h][4 * j + 1] = pre[h].y > 0.f ? g[h][4 * j + 1] : 0.f;
      gp[h][4 * j + 2] = pre[h].z > 0.f ? g[h][4 * j + 2] : 0.f;
      gp[h][4 * j + 3] = pre[h].w > 0.f ? g[h][4 * j + 3] : 0.f;
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (h == 1 && !two) break;
    float4* o = reinterpret_cast<float4*>(Gp_out + (h ? rB : rA) * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = make_float4(gp[h][4 * q], gp[h][4 * q + 1], gp[h][4 * q + 2], gp[h][4 * q + 3]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float4 y[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
    float4 loc[2] = {make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f)};
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float4 w = Wt4[k * 4 + j];
      const float4 u = FORM == GNP_LAYER_PAPER ? Ut4[k * 4 + j] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        y[h].x = fmaf(gp[h][k], w.x, y[h].x);
        y[h].y = fmaf(gp[h][k], w.y, y[h].y);
        y[h].z = fmaf(gp[h][k], w.z, y[h].z);
        y[h].w = fmaf(gp[h][k], w.w, y[h].w);
        if (FORM == GNP_LAYER_PAPER) {
          loc[h].x = fmaf(gp[h][k], u.x, loc[h].x);
          loc[h].y = fmaf(gp[h][k], u.y, loc[h].y);
          loc[h].z = fmaf(gp[h][k], u.z, loc[h].z);
          loc[h].w = fmaf(gp[h][k], u.w, loc[h].w);
        }
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && !two) break;
      const long long r = h ? rB : rA;
      reinterpret_cast<float4*>(Y_out + r * 16)[j] = y[h];
      reinterpret_cast<float4*>(local_out + r * 16)[j] =
          FORM == GNP_LAYER_PAPER ? loc[h] : make_float4(g[h][4 * j], g[h][4 * j + 1], g[h][4 * j + 2], g[h][4 * j + 3]);
    }
  }
}

// ---- tensor-core form of the layer backward
//
// Per warp, tiles of 32 rows: pre = [AGG | X] [W; U] (32 x 32 by 32 x 16) and then
// [Y | local] = Gp [W^T | U^T] (32 x 16 by 16 x 32) on mma.sync m16n8k8 with TF32 operands
// in three products (a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, hi = the operand rounded to
// TF32, lo = the TF32 rounding of its remainder), which keeps float32 accuracy.  The weight
// fragments stay in registers for the whole kernel; the row tiles pass through shared
// memory (padded rows, so that the fragment loads are free of bank conflicts) from
// coalesced 16-byte loads.  The residual form has pre = AGG W, Y = Gp W^T, local = G.
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d += a b in three TF32 products (the small ones first)
__device__ __forceinline__ void mma3_tf32(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                          const uint32_t (&bh)[2], const uint32_t (&bl)[2]) {
  mma_tf32(d, al, bh[0], bh[1]);
  mma_tf32(d, ah, bl[0], bl[1]);
  mma_tf32(d, ah, bh[0], bh[1]);
}

// The A fragment (rows 16 mt + {g, g + 8}, columns 8 ks + {t, t + 4}) of a shared tile with
// row stride ST, split into hi and lo.
template <int ST>
__device__ __forceinline__ void frag_a(const float* tile, int mt, int ks, int g, int t, uint32_t (&hi)[4],
                                       uint32_t (&lo)[4]) {
  const float* p = tile + (16 * mt + g) * ST + 8 * ks + t;
  tf32_split(p[0], hi[0], lo[0]);
  tf32_split(p[8 * ST], hi[1], lo[1]);
  tf32_split(p[4], hi[2], lo[2]);
  tf32_split(p[8 * ST + 4], hi[3], lo[3]);
}

template <int FORM>
__global__ void __launch_bounds__(256)
k_layer_bwd_tc(const float* __restrict__ X, const float* __restrict__ AGG, const float* __restrict__ G, long long R,
               const float* __restrict__ lw, float* __restrict__ Gp_out, float* __restrict__ Y_out,
               float* __restrict__ local_out) {
  constexpr bool PAPER = FORM == GNP_LAYER_PAPER;
  constexpr int KA = PAPER ? 32 : 16;   // inputs of pre: [AGG | X] or AGG
  constexpr int NKS1 = KA / 8;
  constexpr int NNT2 = PAPER ? 4 : 2;   // output tiles of phase 2: [Y | local] or Y
  constexpr int AST = KA + 4;           // padded row strides (floats)
  constexpr int GST = 20;
  static_assert(GST <= AST, "the Gp tile reuses the [AGG | X] tile's space");
  __shared__ __align__(16) float sA[8][32 * AST];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  // weight fragments: phase 1 B1[k][n] = [W; U][k][n] (k input, n output); phase 2
  // B2[k][n] = [W^T | U^T][k][n] = W[n][k] (n < 16) or U[n - 16][k]
  uint32_t b1h[NKS1][2][2], b1l[NKS1][2][2];
#pragma unroll
  for (int ks = 0; ks < NKS1; ++ks)
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int k = 8 * ks + t + 4 * e, nn = 8 * nt + g;
        const float v = k < 16 ? lw[256 + k * 16 + nn] : lw[(k - 16) * 16 + nn];
        tf32_split(v, b1h[ks][nt][e], b1l[ks][nt][e]);
      }
  uint32_t b2h[2][NNT2][2], b2l[2][NNT2][2];
#pragma unroll
  for (int ks = 0; ks < 2; ++ks)
#pragma unroll
    for (int nt = 0; nt < NNT2; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int k = 8 * ks + t + 4 * e, nn = 8 * nt + g;
        const float v = nn < 16 ? lw[256 + nn * 16 + k] : lw[(nn - 16) * 16 + k];
        tf32_split(v, b2h[ks][nt][e], b2l[ks][nt][e]);
      }
  float* At = sA[w];
  float* Gt = sA[w];  // after phase 1 the [AGG | X] tile is dead: the Gp tile takes its place
  const long long ntile = (R + 31) / 32;
  const float4* AG4 = reinterpret_cast<const float4*>(AGG);
  const float4* X4 = reinterpret_cast<const float4*>(X);
  for (long long tile = blockIdx.x * 8LL + w; tile < ntile; tile += gridDim.x * 8LL) {
    const long long r0 = tile * 32;
    const int rows = (int)min(32LL, R - r0);
    // stage [AGG | X] (coalesced 16-byte loads; rows past the end as zeros)
#pragma unroll
    for (int q = lane; q < 32 * KA / 4; q += 32) {
      const int r = q / (KA / 4), c4 = q % (KA / 4);
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < rows) v = c4 < 4 ? __ldg(AG4 + (r0 + r) * 4 + c4) : __ldg(X4 + (r0 + r) * 4 + (c4 - 4));
      *reinterpret_cast<float4*>(At + r * AST + 4 * c4) = v;
    }
    __syncwarp();
    float acc1[2][2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc1[mt][nt][i] = 0.f;
#pragma unroll
    for (int ks = 0; ks < NKS1; ++ks)
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        uint32_t ah[4], al[4];
        frag_a<AST>(At, mt, ks, g, t, ah, al);
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) mma3_tf32(acc1[mt][nt], ah, al, b1h[ks][nt], b1l[ks][nt]);
      }
    __syncwarp();  // every lane has read its phase-1 fragments
    // Gp = G where pre > 0 (the C layout: rows 16 mt + g (+8), columns 8 nt + 2t, +1)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          const int r = 16 * mt + g + 8 * hf, c = 8 * nt + 2 * t;
          float2 gv = make_float2(0.f, 0.f);
          if (r < rows) gv = __ldg(reinterpret_cast<const float2*>(G + (r0 + r) * 16 + c));
          const float2 gp = make_float2(acc1[mt][nt][2 * hf] > 0.f ? gv.x : 0.f,
                                        acc1[mt][nt][2 * hf + 1] > 0.f ? gv.y : 0.f);
          if (r < rows) {
            *reinterpret_cast<float2*>(Gp_out + (r0 + r) * 16 + c) = gp;
            if (!PAPER) *reinterpret_cast<float2*>(local_out + (r0 + r) * 16 + c) = gv;
          }
          *reinterpret_cast<float2*>(Gt + r * GST + c) = gp;
        }
    __syncwarp();
    float acc2[2][NNT2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < NNT2; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc2[mt][nt][i] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 2; ++ks)
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        uint32_t ah[4], al[4];
        frag_a<GST>(Gt, mt, ks, g, t, ah, al);
#pragma unroll
        for (int nt = 0; nt < NNT2; ++nt) mma3_tf32(acc2[mt][nt], ah, al, b2h[ks][nt], b2l[ks][nt]);
      }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < NNT2; ++nt)
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {
          const int r = 16 * mt + g + 8 * hf, c = 8 * (nt & 1) + 2 * t;
          if (r < rows) {
            float* dst = nt < 2 ? Y_out : local_out;
            *reinterpret_cast<float2*>(dst + (r0 + r) * 16 + c) =
                make_float2(acc2[mt][nt][2 * hf], acc2[mt][nt][2 * hf + 1]);
          }
        }
    __syncwarp();  // the tiles are free for the next rows
  }
}

// The layer backward of the training step: two rows per thread in float32 (the default),
// or with GNP_TRAIN_BWD=tc / quad in the environment the tensor-core form or four threads
// per row, for comparison (64^3 step: 22.8 ms, tc 23.9, quad 31.5).  Read at every launch.
static int bwd_form() {
  const char* e = getenv("GNP_TRAIN_BWD");
  if (e && strcmp(e, "quad") == 0) return 2;
  if (e && strcmp(e, "tc") == 0) return 0;
  return 1;
}

// Encoder backward (thread per row): r1 = ReLU(a1) and da1 = (dH0 W2^T) * 1[a1 > 0].
__global__ void __launch_bounds__(256)
k_enc_bwd(const float* __restrict__ u, const float* __restrict__ dH0, long long R, const float* __restrict__ w,
          float* __restrict__ r1_out, float* __restrict__ da1_out) {
  __shared__ __align__(16) float sw[ENC_COUNT];
  for (int k = threadIdx.x; k < ENC_COUNT; k += blockDim.x) sw[k] = w[k];
  __syncthreads();
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < R;
       r += (long long)gridDim.x * blockDim.x) {
    float g[16];
    const float4* gp = reinterpret_cast<const float4*>(dH0 + r * 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float4 v = gp[q];
      g[4 * q] = v.x; g[4 * q + 1] = v.y; g[4 * q + 2] = v.z; g[4 * q + 3] = v.w;
    }
    const float uv = u[r];
    float4* ro = reinterpret_cast<float4*>(r1_out + r * 32);
    float4* dao = reinterpret_cast<float4*>(da1_out + r * 32);
#pragma unroll 2
    for (int k4 = 0; k4 < 8; ++k4) {
      float a[4], d[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = 4 * k4 + j;
        a[j] = fmaf(uv, sw[ENC_W1 + k], sw[ENC_B1 + k]);
        float dd = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 wv = *reinterpret_cast<const float4*>(sw + ENC_W2 + k * 16 + 4 * q);
          dd = fmaf(g[4 * q], wv.x, dd);
          dd = fmaf(g[4 * q + 1], wv.y, dd);
          dd = fmaf(g[4 * q + 2], wv.z, dd);
          dd = fmaf(g[4 * q + 3], wv.w, dd);
        }
        d[j] = dd;
      }
      ro[k4] = make_float4(fmaxf(a[0], 0.f), fmaxf(a[1], 0.f), fmaxf(a[2], 0.f), fmaxf(a[3], 0.f));
      dao[k4] = make_float4(a[0] > 0.f ? d[0] : 0.f, a[1] > 0.f ? d[1] : 0.f, a[2] > 0.f ? d[2] : 0.f,
                            a[3] > 0.f ? d[3] : 0.f);
    }
  }
}

// Weight gradient C = sum_r A'[r]^T B[r] over the R rows, A' = [A[r, :P], 1] (the ones
// column gives the bias row P, the column sums of B).  A split-K reduction: block b owns
// rows [b*WG_CHUNK, (b+1)*WG_CHUNK) and streams them through shared memory in tiles of
// WG_KT rows, the next tile's loads in flight while the current one is used.  Thread
// (g, p, q0) accumulates outputs (p, q0..q0+TN) over the rows g, g+RG, ... of every
// tile (TN = 4 columns per thread: one broadcast A load and one 16-byte B load per four
// FMAs); the RG row-group partials are added in a fixed order at the end, and
// k_wgrad_final adds the block partials in float64, also in a fixed order.  Tiles of
// 128 rows (two 16-byte loads of each operand in flight per thread) and 1,024-row chunks
// (twice the blocks of 2,048) keep enough bytes in flight to stream the operands.
constexpr int WG_CHUNK = 1024;
constexpr int WG_KT = 128;

template <int P, int Q>
struct WgShape {
  static constexpr int TN = Q >= 4 ? 4 : 1;
  static constexpr int NQ = Q / TN;
  static constexpr int NP = P + 1;
  static constexpr int TPG = NP * NQ;  // threads per row group
  static constexpr int RG = 256 / TPG;
  static_assert(RG >= 1 && Q % TN == 0, "output tile larger than a block");
  static constexpr int A4 = WG_KT * P / 4;  // float4 per tile of A
  static constexpr int B4 = WG_KT * Q / 4;
  static constexpr int LA = (A4 + 255) / 256;  // float4 loads per thread
  static constexpr int LB = (B4 + 255) / 256;
};

// A2 (may be null): A's rows are [A[r, :P/2], A2[r, :P/2]] (two row-major arrays of P/2
// columns each), so that one pass over B gives the gradients of two weight matrices that
// share it (the layer's U and W).
template <int P, int Q>
__global__ void __launch_bounds__(256)
k_wgrad(const float* __restrict__ A, const float* __restrict__ A2, const float* __restrict__ Bm, long long R,
        float* __restrict__ partials) {
  using S = WgShape<P, Q>;
  constexpr int TN = S::TN, NQ = S::NQ, NP = S::NP, TPG = S::TPG, RG = S::RG;
  __shared__ __align__(16) float sA[WG_KT * P + 4];
  __shared__ __align__(16) float sB[WG_KT * Q];
  __shared__ float sred[RG > 1 ? RG * NP * Q : 1];
  const int t = threadIdx.x;
  const int g = t / TPG, o = t % TPG;
  const int p = o / NQ, q0 = (o % NQ) * TN;
  const bool active = g < RG;
  const long long r0 = (long long)blockIdx.x * WG_CHUNK;
  const int rows = (int)min((long long)WG_CHUNK, R - r0);  // a multiple of 4 (R = n B, B >= 4)
  const int ntiles = (rows + WG_KT - 1) / WG_KT;
  float acc[TN];
#pragma unroll
  for (int k = 0; k < TN; ++k) acc[k] = 0.f;
  float4 ra[S::LA], rb[S::LB];
  auto load = [&](int kt) {
    const int nr = min(WG_KT, rows - kt * WG_KT);
    const float4* b4 = reinterpret_cast<const float4*>(Bm + (r0 + (long long)kt * WG_KT) * Q);
    if (A2 == nullptr) {
      const float4* a4 = reinterpret_cast<const float4*>(A + (r0 + (long long)kt * WG_KT) * P);
#pragma unroll
      for (int u = 0; u < S::LA; ++u) {
        const int i = t + 256 * u;
        ra[u] = (i < S::A4 && i < nr * P / 4) ? __ldg(a4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    } else {  // float4 i of the tile: row i / (P/4), its half from A or A2
      constexpr int H4 = P / 8;  // float4 per half row
      const float4* a4 = reinterpret_cast<const float4*>(A + (r0 + (long long)kt * WG_KT) * (P / 2));
      const float4* c4 = reinterpret_cast<const float4*>(A2 + (r0 + (long long)kt * WG_KT) * (P / 2));
#pragma unroll
      for (int u = 0; u < S::LA; ++u) {
        const int i = t + 256 * u;
        const int row = i / (2 * H4), k = i % (2 * H4);
        const float4* src = k < H4 ? a4 + row * H4 + k : c4 + row * H4 + (k - H4);
        ra[u] = (i < S::A4 && i < nr * P / 4) ? __ldg(src) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int u = 0; u < S::LB; ++u) {
      const int i = t + 256 * u;
      rb[u] = (i < S::B4 && i < nr * Q / 4) ? __ldg(b4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  load(0);
  for (int kt = 0; kt < ntiles; ++kt) {
    __syncthreads();  // the previous tile is consumed
#pragma unroll
    for (int u = 0; u < S::LA; ++u) {
      const int i = t + 256 * u;
      if (i < S::A4) reinterpret_cast<float4*>(sA)[i] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < S::LB; ++u) {
      const int i = t + 256 * u;
      if (i < S::B4) reinterpret_cast<float4*>(sB)[i] = rb[u];
    }
    __syncthreads();
    if (kt + 1 < ntiles) load(kt + 1);
    // rows past the end of the chunk were loaded as zeros: they add nothing, except to
    // the bias row, whose A' entry is 1 but whose B row is zero
    if (active) {
#pragma unroll 4
      for (int rr = g; rr < WG_KT; rr += RG) {
        const float av = p < P ? sA[rr * P + p] : 1.0f;
        if constexpr (TN == 4) {
          const float4 bv = *reinterpret_cast<const float4*>(sB + rr * Q + q0);
          acc[0] = fmaf(av, bv.x, acc[0]);
          acc[1] = fmaf(av, bv.y, acc[1]);
          acc[2] = fmaf(av, bv.z, acc[2]);
          acc[3] = fmaf(av, bv.w, acc[3]);
        } else {
          acc[0] = fmaf(av, sB[rr * Q + q0], acc[0]);
        }
      }
    }
  }
  float* out = partials + (size_t)blockIdx.x * NP * Q;
  if constexpr (RG == 1) {
    if (active) {
#pragma unroll
      for (int k = 0; k < TN; ++k) out[p * Q + q0 + k] = acc[k];
    }
  } else {
    if (active) {
#pragma unroll
      for (int k = 0; k < TN; ++k) sred[g * NP * Q + p * Q + q0 + k] = acc[k];
    }
    __syncthreads();
    for (int e = t; e < NP * Q; e += 256) {
      float v = 0.f;
#pragma unroll
      for (int gg = 0; gg < RG; ++gg) v += sred[gg * NP * Q + e];
      out[e] = v;
    }
  }
}

// Fixed-order float64 sum of the block partials, one warp per output (lanes stride the
// blocks, then a fixed shuffle tree); rows 0..P-1 -> W (P x Q row-major), row P -> bias
// (may be null).
__global__ void __launch_bounds__(256)
k_wgrad_final(const float* __restrict__ partials, int nblocks, int P, int Q, float* __restrict__ Wout,
              float* __restrict__ bias) {
  const int PQ = (P + 1) * Q;
  const int lane = threadIdx.x & 31;
  const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (o >= PQ) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += (double)partials[(size_t)b * PQ + o];
  s = warp_sum(s);
  if (lane == 0) {
    const int p = o / Q, q = o % Q;
    if (p < P) Wout[p * Q + q] = (float)s;
    else if (bias) bias[q] = (float)s;
  }
}

// Adam (bias corrected) with the best-loss snapshot of the weights *before* the update.
__global__ void k_adam(float* __restrict__ w, float* __restrict__ wbest, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, int count, const float* __restrict__ loss,
                       float* __restrict__ best, int* __restrict__ tstep, float lr, float b1, float b2,
                       float eps) {
  __shared__ int improve;
  __shared__ int t;
  if (threadIdx.x == 0) {
    improve = (*loss < *best) ? 1 : 0;
    t = *tstep + 1;
  }
  __syncthreads();
  const double c1 = 1.0 - pow((double)b1, (double)t);
  const double c2 = 1.0 - pow((double)b2, (double)t);
  for (int k = threadIdx.x; k < count; k += blockDim.x) {
    const float wk = w[k];
    if (improve) wbest[k] = wk;
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float mh = (float)(mk / c1);
    const float vh = (float)(vk / c2);
    w[k] = wk - lr * mh / (sqrtf(vh) + eps);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (improve) *best = *loss;
    *tstep = t;
  }
}

// ---------------------------------------------------------------- sampler kernels

__global__ void k_philox_words(const uint4* __restrict__ ctr, uint32_t k0, uint32_t k1, int count,
                               uint4* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = philox4x32_10(ctr[i], k0, k1);
}

__global__ void k_normal_vec(double* __restrict__ out, int n, unsigned long long seed, uint32_t step,
                             uint32_t stream) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = (double)philox_normal((unsigned long long)i, seed, step, stream);
}

// One-block one-sided Jacobi SVD (Hestenes) of H_bar ((k+1) x k, column-major, k <= 64):
// right singular vectors Z, singular values s; then Q = Z S^-1 in the canonical form
// (descending s, largest-|entry| of each z positive, 1/s = 0 for s < 1e-14 s_max).
constexpr int SVD_MAX = 64;

__global__ void __launch_bounds__(256)
k_jacobi_svd(const double* __restrict__ Hbar, int k, double* __restrict__ Qout) {
  __shared__ double Bm[(SVD_MAX + 1) * SVD_MAX];
  __shared__ double Zs[SVD_MAX * SVD_MAX];
  __shared__ double sv[SVD_MAX];
  __shared__ int order[SVD_MAX];
  __shared__ int rotated;
  const int ld = k + 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int t = threadIdx.x; t < ld * k; t += blockDim.x) Bm[t] = Hbar[t];
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) Zs[t] = (t / k == t % k) ? 1.0 : 0.0;
  __syncthreads();
  const int kk = (k + 1) & ~1;  // players of the round-robin (one dummy when k is odd)
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int round = 0; round < kk - 1; ++round) {
      for (int pr = wid; pr < kk / 2; pr += nw) {
        auto pos = [&](int x) { return x == 0 ? 0 : ((x - 1 + round) % (kk - 1)) + 1; };
        int p = pos(pr), q = pos(kk - 1 - pr);
        if (p > q) { int tmp = p; p = q; q = tmp; }
        if (q >= k) continue;
        double* bp = Bm + p * ld;
        double* bq = Bm + q * ld;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < ld; i += 32) {
          al += bp[i] * bp[i];
          be += bq[i] * bq[i];
          ga += bp[i] * bq[i];
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga != 0.0 && fabs(ga) > 1e-15 * sqrt(al * be)) {
          const double zeta = (be - al) / (2.0 * ga);
          const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + tt * tt);
          const double s = c * tt;
          for (int i = lane; i < ld; i += 32) {
            const double a = bp[i], b = bq[i];
            bp[i] = c * a - s * b;
            bq[i] = s * a + c * b;
          }
          double* zp = Zs + p * k;
          double* zq = Zs + q * k;
          for (int i = lane; i < k; i += 32) {
            const double a = zp[i], b = zq[i];
            zp[i] = c * a - s * b;
            zq[i] = s * a + c * b;
          }
          if (lane == 0) rotated = 1;
        }
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  // singular values = column norms
  for (int j = wid; j < k; j += nw) {
    double s = 0.0;
    for (int i = lane; i < ld; i += 32) s += Bm[j * ld + i] * Bm[j * ld + i];
    s = warp_sum(s);
    if (lane == 0) sv[j] = sqrt(s);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int j = 0; j < k; ++j) order[j] = j;
    for (int a = 1; a < k; ++a) {  // insertion sort, descending
      int o = order[a];
      int b = a - 1;
      while (b >= 0 && sv[order[b]] < sv[o]) {
        order[b + 1] = order[b];
        --b;
      }
      order[b + 1] = o;
    }
  }
  __syncthreads();
  const double smax = sv[order[0]];
  for (int jj = wid; jj < k; jj += nw) {
    const int j = order[jj];
    const double* z = Zs + j * k;
    // canonical sign: the largest-magnitude entry positive (first one on ties)
    int imax = 0;
    double vmax = -1.0;
    if (lane == 0) {
      for (int i = 0; i < k; ++i)
        if (fabs(z[i]) > vmax) { vmax = fabs(z[i]); imax = i; }
    }
    imax = __shfl_sync(0xffffffffu, imax, 0);
    const double sg = z[imax] < 0.0 ? -1.0 : 1.0;
    const double inv = (sv[j] >= 1e-14 * smax && sv[j] > 0.0) ? 1.0 / sv[j] : 0.0;
    for (int i = lane; i < k; i += 32) Qout[i * k + jj] = sg * z[i] * inv;  // row-major Q[i][jj]
  }
}

// C = Q E for the Eq. 5 draws of this step: E[j][c] = normal(j*Ba + c, stream 2).
__global__ void k_sampler_coef(const double* __restrict__ Q, int mA, int Ba, unsigned long long seed,
                               uint32_t step, double* __restrict__ C) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < mA * Ba; t += gridDim.x * blockDim.x) {
    const int j = t / Ba, c = t % Ba;
    double s = 0.0;
    for (int l = 0; l < mA; ++l)
      s += Q[j * mA + l] * (double)philox_normal((unsigned long long)l * Ba + c, seed, step, STREAM_EPS);
    C[t] = s;
  }
}

// x[:, :Ba] = V_m C (float64 sums, float32 store); x[:, Ba:] ~ N(0, I) (stream 1,
// element (i, c) at index i*Bg + c).
__global__ void k_sampler_x(const double* __restrict__ V, int n, int mA, const double* __restrict__ C, int B,
                            int Ba, unsigned long long seed, uint32_t step, float* __restrict__ x) {
  const int Bg = B - Ba;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * B;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / B), c = (int)(e % B);
    float val;
    if (c < Ba) {
      double s = 0.0;
      for (int j = 0; j < mA; ++j) s += V[(size_t)j * n + i] * C[j * Ba + c];
      val = (float)s;
    } else {
      val = philox_normal((unsigned long long)i * Bg + (c - Ba), seed, step, STREAM_X);
    }
    x[e] = val;
  }
}

// ---------------------------------------------------------------- host drivers

static int grid_rows(long long R) {
  long long b = (R + 255) / 256;
  return (int)std::min<long long>(std::max<long long>(b, 1), 8LL * NUM_SMS_GB300);
}

static int layer_smem(int B) { return (512 + 8 * 2 * B * 16) * (int)sizeof(float); }

template <int FORM, int B>
static int layer_batch_one(int grid, int smem, cudaStream_t st, const int* rp, const int* col, const float* vh,
                           const float* X, float* AG, float* Out, int n, const float* lw) {
  static int done = 0;
  if (done < smem) {
    GNP_TRY_CUDA(cudaFuncSetAttribute(k_layer_batch<FORM, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    done = smem;
  }
  k_layer_batch<FORM, B><<<grid, 256, smem, st>>>(rp, col, vh, X, AG, Out, n, lw);
  return check_launch("k_layer_batch");
}

template <int FORM>
static int layer_batch_form(int B, int grid, int smem, cudaStream_t st, const int* rp, const int* col,
                            const float* vh, const float* X, float* AG, float* Out, int n, const float* lw) {
  switch (B) {
    case 4: return layer_batch_one<FORM, 4>(grid, smem, st, rp, col, vh, X, AG, Out, n, lw);
    case 8: return layer_batch_one<FORM, 8>(grid, smem, st, rp, col, vh, X, AG, Out, n, lw);
    case 16: return layer_batch_one<FORM, 16>(grid, smem, st, rp, col, vh, X, AG, Out, n, lw);
    case 32: return layer_batch_one<FORM, 32>(grid, smem, st, rp, col, vh, X, AG, Out, n, lw);
    case 64: return layer_batch_one<FORM, 64>(grid, smem, st, rp, col, vh, X, AG, Out, n, lw);
    default: set_error("k_layer_batch: batch %d is not a power of two in [4, 64]", B); return GNP_ERR_INVALID_ARG;
  }
}

static int layer_batch_launch(int form, int B, int grid, int smem, cudaStream_t st, const int* rp, const int* col,
                              const float* vh, const float* X, float* AG, float* Out, int n, const float* lw) {
  return form == GNP_LAYER_PAPER ? layer_batch_form<GNP_LAYER_PAPER>(B, grid, smem, st, rp, col, vh, X, AG, Out, n, lw)
                                 : layer_batch_form<GNP_LAYER_RESID>(B, grid, smem, st, rp, col, vh, X, AG, Out, n, lw);
}

// Forward on the batch b (device, node-major [n*B]); activations saved in T.
static int forward_batch(gnp_model* M, const float* b, cudaStream_t st) {
  TrainState* T = M->train;
  const gnp_mat* A = M->A;
  const int n = A->n, B = T->B, L = M->cfg.L;
  const long long R = T->R;
  const double sqrt_n = std::sqrt((double)n);
  const int nb = red_blocks(R);
  if (M->cfg.no_scale)
    k_fill_tau<<<1, 64, 0, st>>>(T->tau, B, sqrt_n);  // u = b, z = network output
  else
    k_col_norms<<<nb, 256, 0, st>>>(b, R, B, T->red.partials, T->red.counter, T->tau);
  k_enc_batch<<<grid_rows(R), 256, 0, st>>>(b, T->tau, R, B, sqrt_n, M->w_dev, T->u, T->Hs);
  const int smem = layer_smem(B);
  const int wgrid = std::min((n + 7) / 8, 16 * NUM_SMS_GB300);
  for (int l = 0; l < L; ++l) {
    const float* X = T->Hs + (size_t)l * R * 16;
    float* Out = T->Hs + (size_t)(l + 1) * R * 16;
    float* AG = T->AGG + (size_t)l * R * 16;
    const float* lw = M->w_dev + layer_off(l);
    GNP_TRY(layer_batch_launch(M->cfg.form, B, wgrid, smem, st, A->rp, A->col, M->valhat, X, AG, Out, n, lw));
  }
  k_dec_batch<<<grid_rows(R), 256, 0, st>>>(T->Hs + (size_t)L * R * 16, T->tau, R, B, sqrt_n,
                                            M->w_dev + dec_off(L), T->z);
  return check_launch("forward_batch");
}

// k_wgrad for P x Q = 512 outputs (the layer's [X | AGG]^T Gp, 32 x 16, and the decoder's
// 16 x 32) with a 4 x 4 register tile per lane: one warp owns the whole output, lane l
// the rows 4 (l / (Q/4)) .. +3 and columns 4 (l % (Q/4)) .. +3, so a staged row costs the
// warp two 16-byte shared loads for 16 multiply-adds per lane (k_wgrad's one output
// column per thread was bound by its shared-memory loads).  The 8 warps split each tile's
// rows; their sums meet in shared memory in warp order.  Same partials layout as k_wgrad
// (row P = the bias), reduced by k_wgrad_final.
template <int P, int Q>
__global__ void __launch_bounds__(256)
k_wgrad_t(const float* __restrict__ A, const float* __restrict__ A2, const float* __restrict__ Bm, long long R,
          float* __restrict__ partials) {
  using S = WgShape<P, Q>;
  constexpr int NQB = Q / 4, NPB = P / 4;
  static_assert(P % 4 == 0 && Q % 4 == 0 && NPB * NQB == 32, "one 4 x 4 tile per lane");
  constexpr int NOUT = (P + 1) * Q;
  __shared__ __align__(16) float sA[WG_KT * P + 4];
  __shared__ __align__(16) float sB[WG_KT * Q];
  __shared__ float sred[8 * NOUT];
  const int t = threadIdx.x;
  const int w = t >> 5, lane = t & 31;
  const int pb = lane / NQB, qb = lane % NQB;
  const long long r0 = (long long)blockIdx.x * WG_CHUNK;
  const int rows = (int)min((long long)WG_CHUNK, R - r0);
  const int ntiles = (rows + WG_KT - 1) / WG_KT;
  float acc[4][4];
  float bacc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[i][k] = 0.f;
  float4 ra[S::LA], rb[S::LB];
  auto load = [&](int kt) {
    const int nr = min(WG_KT, rows - kt * WG_KT);
    const float4* b4 = reinterpret_cast<const float4*>(Bm + (r0 + (long long)kt * WG_KT) * Q);
    if (A2 == nullptr) {
      const float4* a4 = reinterpret_cast<const float4*>(A + (r0 + (long long)kt * WG_KT) * P);
#pragma unroll
      for (int u = 0; u < S::LA; ++u) {
        const int i = t + 256 * u;
        ra[u] = (i < S::A4 && i < nr * P / 4) ? __ldg(a4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    } else {
      constexpr int H4 = P / 8;
      const float4* a4 = reinterpret_cast<const float4*>(A + (r0 + (long long)kt * WG_KT) * (P / 2));
      const float4* c4 = reinterpret_cast<const float4*>(A2 + (r0 + (long long)kt * WG_KT) * (P / 2));
#pragma unroll
      for (int u = 0; u < S::LA; ++u) {
        const int i = t + 256 * u;
        const int row = i / (2 * H4), k = i % (2 * H4);
        const float4* src = k < H4 ? a4 + row * H4 + k : c4 + row * H4 + (k - H4);
        ra[u] = (i < S::A4 && i < nr * P / 4) ? __ldg(src) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int u = 0; u < S::LB; ++u) {
      const int i = t + 256 * u;
      rb[u] = (i < S::B4 && i < nr * Q / 4) ? __ldg(b4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  load(0);
  for (int kt = 0; kt < ntiles; ++kt) {
    __syncthreads();  // the previous tile is consumed
#pragma unroll
    for (int u = 0; u < S::LA; ++u) {
      const int i = t + 256 * u;
      if (i < S::A4) reinterpret_cast<float4*>(sA)[i] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < S::LB; ++u) {
      const int i = t + 256 * u;
      if (i < S::B4) reinterpret_cast<float4*>(sB)[i] = rb[u];
    }
    __syncthreads();
    if (kt + 1 < ntiles) load(kt + 1);
    // rows past the end of the chunk were staged as zeros and add nothing
#pragma unroll 4
    for (int rr = w; rr < WG_KT; rr += 8) {
      const float4 av = *reinterpret_cast<const float4*>(sA + rr * P + 4 * pb);
      const float4 bv = *reinterpret_cast<const float4*>(sB + rr * Q + 4 * qb);
      const float a4[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        acc[i][0] = fmaf(a4[i], bv.x, acc[i][0]);
        acc[i][1] = fmaf(a4[i], bv.y, acc[i][1]);
        acc[i][2] = fmaf(a4[i], bv.z, acc[i][2]);
        acc[i][3] = fmaf(a4[i], bv.w, acc[i][3]);
      }
      if (pb == 0) {
        bacc[0] += bv.x;
        bacc[1] += bv.y;
        bacc[2] += bv.z;
        bacc[3] += bv.w;
      }
    }
  }
  float* my = sred + w * NOUT;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int k = 0; k < 4; ++k) my[(4 * pb + i) * Q + 4 * qb + k] = acc[i][k];
  if (pb == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) my[P * Q + 4 * qb + k] = bacc[k];
  }
  __syncthreads();
  float* out = partials + (size_t)blockIdx.x * NOUT;
  for (int e = t; e < NOUT; e += 256) {
    float v = 0.f;
#pragma unroll
    for (int ww = 0; ww < 8; ++ww) v += sred[ww * NOUT + e];
    out[e] = v;
  }
}

// The weight-gradient reduction: the tiled form where P x Q = 512 (GNP_TRAIN_WGRAD=col in
// the environment keeps the one-column-per-thread form, for comparison).
static bool wgrad_col() {
  static const char* e = getenv("GNP_TRAIN_WGRAD");
  static const bool c = e && strcmp(e, "col") == 0;
  return c;
}

template <int P, int Q>
static int wgrad(TrainState* T, const float* A, const float* Bm, float* Wout, float* bias, cudaStream_t st,
                 const float* A2 = nullptr) {
  const int nblk = (int)((T->R + WG_CHUNK - 1) / WG_CHUNK);
  const int PQ = (P + 1) * Q;
  if (T->part_cap < nblk * 33 * 32) {
    if (T->partials) cudaFree(T->partials);
    T->partials = nullptr;
    GNP_TRY(dev_alloc(&T->partials, (size_t)nblk * 33 * 32));
    T->part_cap = nblk * 33 * 32;
  }
  if constexpr (P * Q == 512 && P % 4 == 0 && Q % 4 == 0) {
    if (!wgrad_col()) k_wgrad_t<P, Q><<<nblk, 256, 0, st>>>(A, A2, Bm, T->R, T->partials);
    else k_wgrad<P, Q><<<nblk, 256, 0, st>>>(A, A2, Bm, T->R, T->partials);
  } else {
    k_wgrad<P, Q><<<nblk, 256, 0, st>>>(A, A2, Bm, T->R, T->partials);
  }
  k_wgrad_final<<<(PQ * 32 + 255) / 256, 256, 0, st>>>(T->partials, nblk, P, Q, Wout, bias);
  return check_launch("wgrad");
}

// Backward of the saved forward given dL/dz (device [R]); gradient blob -> T->grad.
static int backward_batch(gnp_model* M, const float* dz, cudaStream_t st) {
  TrainState* T = M->train;
  const gnp_mat* A = M->A;
  const int n = A->n, B = T->B, L = M->cfg.L;
  const long long R = T->R;
  const double sqrt_n = std::sqrt((double)n);
  float* g = T->grad;
  const float* HL = T->Hs + (size_t)L * R * 16;
  // decoder: do -> r1, q -> s32a, dc1 -> s32b, dH^L -> g16a
  k_dec_bwd<<<grid_rows(R), 256, 0, st>>>(HL, dz, T->tau, R, B, sqrt_n, M->w_dev + dec_off(L), T->r1, T->s32a,
                                          T->s32b, T->g16a);
  float* gd = g + dec_off(L);
  GNP_TRY((wgrad<16, 32>(T, HL, T->s32b, gd, gd + 512, st)));          // dD1, de1
  GNP_TRY((wgrad<32, 1>(T, T->s32a, T->r1, gd + 544, gd + 576, st)));   // dD2, de2
  float* G = T->g16a;
  float* Gn = T->g16b;
  const int wgrid = std::min((n + 7) / 8, 16 * NUM_SMS_GB300);
  for (int l = L - 1; l >= 0; --l) {
    const float* X = T->Hs + (size_t)l * R * 16;
    const float* AG = T->AGG + (size_t)l * R * 16;
    const float* lw = M->w_dev + layer_off(l);
    const int bf = bwd_form();
    if (bf == 0) {
      const int tiles = (int)std::min<long long>((R + 31) / 32, 1LL << 30);
      const int grid = std::min((tiles + 7) / 8, 4 * NUM_SMS_GB300 * 4);
      if (M->cfg.form == GNP_LAYER_PAPER)
        k_layer_bwd_tc<GNP_LAYER_PAPER><<<grid, 256, 0, st>>>(X, AG, G, R, lw, T->gp16, T->y16, Gn);
      else
        k_layer_bwd_tc<GNP_LAYER_RESID><<<grid, 256, 0, st>>>(X, AG, G, R, lw, T->gp16, T->y16, Gn);
    } else if (bf == 2) {
      if (M->cfg.form == GNP_LAYER_PAPER)
        k_layer_bwd_rows<GNP_LAYER_PAPER><<<(int)((R + 63) / 64), 256, 0, st>>>(X, AG, G, R, lw, T->gp16, T->y16,
                                                                               Gn);
      else
        k_layer_bwd_rows<GNP_LAYER_RESID><<<(int)((R + 63) / 64), 256, 0, st>>>(X, AG, G, R, lw, T->gp16, T->y16,
                                                                               Gn);
    } else if (M->cfg.form == GNP_LAYER_PAPER) {
      k_layer_bwd_row2<GNP_LAYER_PAPER><<<(int)((R + 511) / 512), 256, 0, st>>>(X, AG, G, R, lw, T->gp16, T->y16, Gn);
    } else {
      k_layer_bwd_row2<GNP_LAYER_RESID><<<(int)((R + 511) / 512), 256, 0, st>>>(X, AG, G, R, lw, T->gp16, T->y16, Gn);
    }
    // dX = local + A_hat^T Y (gather through the canonical CSC)
    GNP_TRY(spmm_nodes(A->csc.ptr, A->csc.idx, M->valhat_t, reinterpret_cast<const float4*>(T->y16), n, B * 4,
                       1.0f, reinterpret_cast<const float4*>(Gn), 1.0f, reinterpret_cast<float4*>(Gn), st));
    float* gl = g + layer_off(l);
    if (M->cfg.form == GNP_LAYER_PAPER) {
      GNP_TRY((wgrad<32, 16>(T, X, T->gp16, gl, nullptr, st, AG)));  // dU (rows 0-15), dW (16-31)
    } else {
      GNP_TRY_CUDA(cudaMemsetAsync(gl, 0, sizeof(float) * 256, st));
      GNP_TRY((wgrad<16, 16>(T, AG, T->gp16, gl + 256, nullptr, st)));  // dW
    }
    std::swap(G, Gn);
  }
  // encoder: r1 -> s32a, da1 -> s32b
  k_enc_bwd<<<grid_rows(R), 256, 0, st>>>(T->u, G, R, M->w_dev, T->s32a, T->s32b);
  GNP_TRY((wgrad<32, 16>(T, T->s32a, G, g + ENC_W2, g + ENC_B2, st)));  // dW2, db2
  GNP_TRY((wgrad<1, 32>(T, T->u, T->s32b, g + ENC_W1, g + ENC_B1, st))); // dW1, db1
  return check_launch("backward_batch");
}

static int sampler_prepare(gnp_model* M, cudaStream_t st) {
  TrainState* T = M->train;
  if (T->sampler_ready) return GNP_OK;
  const int n = M->A->n;
  const int m = M->cfg.arnoldi_m;
  GNP_REQUIRE(m >= 1 && m <= SVD_MAX, "arnoldi_m = %d outside [1, %d]", m, SVD_MAX);
  double* v1 = nullptr;
  GNP_TRY(dev_alloc(&v1, (size_t)n));
  k_normal_vec<<<grid_rows(n), 256, 0, st>>>(v1, n, M->cfg.seed, 0u, STREAM_V1);
  if (!T->V) GNP_TRY(dev_alloc(&T->V, (size_t)n * (m + 1)));
  std::vector<double> Hh((size_t)(m + 1) * m, 0.0);
  int k = 0;
  int s = arnoldi_basis(M->A, v1, m, T->V, Hh.data(), &k, st);
  dev_free(v1);
  if (s != GNP_OK) return s;
  GNP_REQUIRE(k >= 1, "sampler: Arnoldi broke down at the first step");
  // H_bar of A_hat = H_bar of A / gamma (same basis V); compact to (k+1) x k
  std::vector<double> Hk((size_t)(k + 1) * k);
  for (int j = 0; j < k; ++j)
    for (int i = 0; i <= k; ++i)  // upper Hessenberg: zero below the subdiagonal
      Hk[(size_t)j * (k + 1) + i] = i <= j + 1 ? Hh[(size_t)j * (m + 1) + i] / M->gamma : 0.0;
  if (T->Hbar) cudaFree(T->Hbar);
  T->Hbar = nullptr;
  if (T->Q) cudaFree(T->Q);
  T->Q = nullptr;
  GNP_TRY(dev_alloc(&T->Hbar, Hk.size()));
  GNP_TRY(dev_alloc(&T->Q, (size_t)k * k));
  GNP_TRY_CUDA(cudaMemcpyAsync(T->Hbar, Hk.data(), sizeof(double) * Hk.size(), cudaMemcpyHostToDevice, st));
  k_jacobi_svd<<<1, 256, 0, st>>>(T->Hbar, k, T->Q);
  GNP_TRY(check_launch("k_jacobi_svd"));
  GNP_TRY_CUDA(cudaStreamSynchronize(st));
  T->mA = k;
  T->sampler_ready = true;
  return GNP_OK;
}

// The batch of step `step`: sample_mode 0 (Sec. 3) fills the first B/2 columns with
// Eq. 5 samples and the rest with N(0, I); modes 1 and 2 (the Sec. 4 ablations) fill all
// B columns with N(0, I) (read as x in mode 1, as b in mode 2).
static int sample_batch(gnp_model* M, int step, float* x, cudaStream_t st) {
  TrainState* T = M->train;
  const int n = M->A->n, B = T->B;
  const int Ba = M->cfg.sample_mode == 0 ? B / 2 : 0;
  int mA = 0;
  if (Ba > 0) {
    GNP_TRY(sampler_prepare(M, st));
    mA = T->mA;
    if (!T->C) GNP_TRY(dev_alloc(&T->C, (size_t)SVD_MAX * GNP_MAX_BATCH));
    k_sampler_coef<<<1, 256, 0, st>>>(T->Q, mA, Ba, M->cfg.seed, (uint32_t)step, T->C);
  }
  k_sampler_x<<<grid_rows((long long)n * B), 256, 0, st>>>(T->V, n, mA, T->C, B, Ba, M->cfg.seed,
                                                           (uint32_t)step, x);
  return check_launch("sample_batch");
}

// Forward on T->bb, loss, dz, backward, Adam.  No host synchronisation.
static int train_from_b(gnp_model* M, cudaStream_t st) {
  TrainState* T = M->train;
  const gnp_mat* A = M->A;
  const int n = A->n, B = T->B;
  const long long R = T->R;
  const int wgrid = std::min((n + 7) / 8, 16 * NUM_SMS_GB300);
  const int W4 = B / 4;
  GNP_TRY(forward_batch(M, T->bb, st));
  // r = A_hat z - b; loss = mean |r|; s = sign(r); dz = A_hat^T s / (n B)
  GNP_TRY(spmm_nodes(A->rp, A->col, M->valhat, reinterpret_cast<const float4*>(T->z), n, W4, 1.0f,
                     reinterpret_cast<const float4*>(T->bb), -1.0f, reinterpret_cast<float4*>(T->rr), st));
  k_l1<<<red_blocks(R), 256, 0, st>>>(T->rr, R, T->red.partials, T->red.counter, T->loss);
  GNP_TRY(spmm_nodes(A->csc.ptr, A->csc.idx, M->valhat_t, reinterpret_cast<const float4*>(T->rr), n, W4,
                     (float)(1.0 / (double)R), nullptr, 0.0f, reinterpret_cast<float4*>(T->dz), st));
  GNP_TRY(backward_batch(M, T->dz, st));
  const int cnt = weight_count(M->cfg.L);
  k_adam<<<1, 1024, 0, st>>>(M->w_dev, M->w_best, T->grad, T->adam_m, T->adam_v, cnt, T->loss, T->best_loss,
                             T->adam_t, M->cfg.lr, M->cfg.beta1, M->cfg.beta2, M->cfg.eps);
  M->host_stale = true;
  ++M->version;
  return check_launch("train step");
}

// b = A_hat x, then train_from_b.
static int train_pairs(gnp_model* M, const float* x, cudaStream_t st) {
  TrainState* T = M->train;
  const gnp_mat* A = M->A;
  const int n = A->n;
  const int wgrid = std::min((n + 7) / 8, 16 * NUM_SMS_GB300);
  GNP_TRY(spmm_nodes(A->rp, A->col, M->valhat, reinterpret_cast<const float4*>(x), n, T->B / 4, 1.0f, nullptr,
                     0.0f, reinterpret_cast<float4*>(T->bb), st));
  return train_from_b(M, st);
}

// One step on the model's own sampler (sample_mode 2 samples b directly).
static int train_step_own(gnp_model* M, cudaStream_t st) {
  TrainState* T = M->train;
  const int step = T->step++;
  if (M->cfg.sample_mode == 2) {
    GNP_TRY(sample_batch(M, step, T->bb, st));
    return train_from_b(M, st);
  }
  GNP_TRY(sample_batch(M, step, T->xb, st));
  return train_pairs(M, T->xb, st);
}

static int train_prepare(gnp_model* M, int B, cudaStream_t st) {
  (void)st;
  return train_ensure(M, B);
}

}  // namespace gnp

using namespace gnp;

extern "C" {

int gnp_philox4x32_10(const unsigned* ctr_dev, unsigned key0, unsigned key1, int count, unsigned* out_dev,
                      void* stream) {
  GNP_REQUIRE(ctr_dev && out_dev && count >= 0, "gnp_philox4x32_10: bad argument");
  if (count == 0) return GNP_OK;
  k_philox_words<<<(count + 255) / 256, 256, 0, as_stream(stream)>>>(
      reinterpret_cast<const uint4*>(ctr_dev), key0, key1, count, reinterpret_cast<uint4*>(out_dev));
  return check_launch("k_philox_words");
}

int gnp_set_weights_device(gnp_model* M, const float* w_dev, int count, void* stream) {
  GNP_REQUIRE(M && w_dev, "gnp_set_weights_device: null argument");
  GNP_REQUIRE(count == weight_count(M->cfg.L), "gnp_set_weights_device: %d floats, expected %d", count,
              weight_count(M->cfg.L));
  cudaStream_t st = as_stream(stream);
  GNP_TRY_CUDA(cudaMemcpyAsync(M->w_dev, w_dev, sizeof(float) * count, cudaMemcpyDeviceToDevice, st));
  GNP_TRY_CUDA(cudaMemcpyAsync(M->w_best, w_dev, sizeof(float) * count, cudaMemcpyDeviceToDevice, st));
  M->host_stale = true;
  ++M->version;
  return GNP_OK;
}

int gnp_forward_batch(gnp_model* M, const float* b_dev, int B, float* z_dev, void* stream) {
  GNP_REQUIRE(M && b_dev && z_dev, "gnp_forward_batch: null argument");
  cudaStream_t st = as_stream(stream);
  GNP_TRY(train_prepare(M, B, st));
  GNP_TRY(forward_batch(M, b_dev, st));
  GNP_TRY_CUDA(cudaMemcpyAsync(z_dev, M->train->z, sizeof(float) * M->train->R, cudaMemcpyDeviceToDevice, st));
  return GNP_OK;
}

int gnp_backward_batch(gnp_model* M, const float* dz_dev, float* grad_dev, void* stream) {
  GNP_REQUIRE(M && dz_dev && grad_dev, "gnp_backward_batch: null argument");
  GNP_REQUIRE(M->train != nullptr, "gnp_backward_batch: no forward_batch before");
  cudaStream_t st = as_stream(stream);
  GNP_TRY(backward_batch(M, dz_dev, st));
  GNP_TRY_CUDA(cudaMemcpyAsync(grad_dev, M->train->grad, sizeof(float) * weight_count(M->cfg.L),
                               cudaMemcpyDeviceToDevice, st));
  return GNP_OK;
}

int gnp_sample_batch(gnp_model* M, int step, float* x_dev, void* stream) {
  GNP_REQUIRE(M && x_dev, "gnp_sample_batch: null argument");
  GNP_REQUIRE(step >= 0, "gnp_sample_batch: step < 0");
  cudaStream_t st = as_stream(stream);
  GNP_TRY(train_prepare(M, M->cfg.batch, st));
  return sample_batch(M, step, x_dev, st);
}

int gnp_train_step_pairs(gnp_model* M, const float* x_dev, int B, float* loss_out, void* stream) {
  GNP_REQUIRE(M && x_dev, "gnp_train_step_pairs: null argument");
  cudaStream_t st = as_stream(stream);
  GNP_TRY(train_prepare(M, B, st));
  GNP_TRY(train_pairs(M, x_dev, st));
  if (loss_out) {
    GNP_TRY_CUDA(cudaMemcpyAsync(loss_out, M->train->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    GNP_TRY_CUDA(cudaStreamSynchronize(st));
  }
  return GNP_OK;
}

int gnp_train_step(gnp_model* M, float* loss_out, void* stream) {
  GNP_REQUIRE(M, "gnp_train_step: null model");
  cudaStream_t st = as_stream(stream);
  GNP_TRY(train_prepare(M, M->cfg.batch, st));
  TrainState* T = M->train;
  GNP_TRY(train_step_own(M, st));
  if (loss_out) {
    GNP_TRY_CUDA(cudaMemcpyAsync(loss_out, T->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    GNP_TRY_CUDA(cudaStreamSynchronize(st));
  }
  return GNP_OK;
}

int gnp_train_release(gnp_model* M) {
  GNP_REQUIRE(M, "gnp_train_release: null model");
  GNP_TRY(model_sync_host(M));
  train_free(M->train);
  M->train = nullptr;
  return GNP_OK;
}

int gnp_train_history(gnp_model* M, int steps, float* losses_out, float* best_loss_out, void* stream) {
  GNP_REQUIRE(M && steps >= 0, "gnp_train: bad argument");
  cudaStream_t st = as_stream(stream);
  GNP_TRY(train_prepare(M, M->cfg.batch, st));
  TrainState* T = M->train;
  if (M->cfg.sample_mode == 0) GNP_TRY(sampler_prepare(M, st));
  float* hist = nullptr;
  if (losses_out && steps > 0) GNP_TRY(dev_alloc(&hist, (size_t)steps));
  int e = GNP_OK;
  for (int s = 0; s < steps && e == GNP_OK; ++s) {
    e = train_step_own(M, st);
    if (e == GNP_OK && hist && cudaMemcpyAsync(hist + s, T->loss, sizeof(float), cudaMemcpyDeviceToDevice, st) !=
                                   cudaSuccess) {
      set_error("gnp_train: loss copy failed");
      e = GNP_ERR_CUDA;
    }
  }
  if (e == GNP_OK && hist &&
      cudaMemcpyAsync(losses_out, hist, sizeof(float) * steps, cudaMemcpyDeviceToHost, st) != cudaSuccess) {
    set_error("gnp_train: loss history copy failed");
    e = GNP_ERR_CUDA;
  }
  if (e == GNP_OK && best_loss_out &&
      cudaMemcpyAsync(best_loss_out, T->best_loss, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess) {
    set_error("gnp_train: best loss copy failed");
    e = GNP_ERR_CUDA;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && e == GNP_OK) {
    set_error("gnp_train: %s", cudaGetErrorString(cudaGetLastError()));
    e = GNP_ERR_CUDA;
  }
  dev_free(hist);
  return e;
}

int gnp_train(gnp_model* M, int steps, float* best_loss_out, void* stream) {
  return gnp_train_history(M, steps, nullptr, best_loss_out, stream);
}

}  // extern "C"
