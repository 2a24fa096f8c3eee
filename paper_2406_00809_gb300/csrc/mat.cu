// Sparse matrix objects: upload with validation, the transpose (CSC) built on the
// device, the gamma normalisation factor of Eq. 6, and the float64 SpMV entry point.
#include <algorithm>
#include <vector>

#include "internal.h"

namespace gnp {

// ---------------------------------------------------------------- CSC build

__global__ void k_count_cols(const int* __restrict__ col, long long nnz, int* __restrict__ cnt) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz;
       e += (long long)gridDim.x * blockDim.x)
    atomicAdd(cnt + col[e], 1);
}

// Exclusive scan of cnt[0..n) into ptr[0..n] in three launches: per-block scans of
// 1024 entries, a scan of the block totals by one block, and the add-back.
constexpr int SCAN_B = 1024;

__device__ int block_exclusive_scan(int v, int* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int t = lane < (blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    sh[lane] = t;  // inclusive scan of warp totals
  }
  __syncthreads();
  int base = w > 0 ? sh[w - 1] : 0;
  int total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  sh[32] = total;
  return base + x - v;
}

__global__ void k_scan_blocks(const int* __restrict__ cnt, int n, int* __restrict__ ptr,
                              int* __restrict__ totals) {
  __shared__ int sh[33];
  int i = blockIdx.x * SCAN_B + threadIdx.x;
  int v = i < n ? cnt[i] : 0;
  int ex = block_exclusive_scan(v, sh);
  __syncthreads();
  if (i < n) ptr[i] = ex;
  if (threadIdx.x == 0) totals[blockIdx.x] = sh[32];
}

__global__ void k_scan_totals(int* totals, int nb) {
  __shared__ int sh[33];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += SCAN_B) {
    int i = base + threadIdx.x;
    int v = i < nb ? totals[i] : 0;
    int ex = block_exclusive_scan(v, sh);
    __syncthreads();
    int c = carry;
    if (i < nb) totals[i] = ex + c;
    __syncthreads();
    if (threadIdx.x == 0) carry = c + sh[32];
    __syncthreads();
  }
}

__global__ void k_scan_add(int* ptr, int n, const int* totals, long long nnz) {
  int i = blockIdx.x * SCAN_B + threadIdx.x;
  if (i < n) ptr[i] += totals[blockIdx.x];
  if (i == 0) ptr[n] = (int)nnz;
}

__global__ void k_scatter_csc(const int* __restrict__ rp, const int* __restrict__ col, int n,
                              const int* __restrict__ ptr, int* __restrict__ fill,
                              int* __restrict__ idx, int* __restrict__ perm) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    for (int e = rp[r]; e < rp[r + 1]; ++e) {
      int c = col[e];
      int pos = ptr[c] + atomicAdd(fill + c, 1);
      idx[pos] = r;
      perm[pos] = e;
    }
  }
}

// Canonical order inside each column: by row, then by CSR position (insertion sort;
// columns are short for the matrices this library targets, and this runs once).
__global__ void k_sort_csc(const int* __restrict__ ptr, int n, int* __restrict__ idx,
                           int* __restrict__ perm) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    int a = ptr[c], b = ptr[c + 1];
    for (int i = a + 1; i < b; ++i) {
      int ki = idx[i], pi = perm[i];
      int j = i - 1;
      while (j >= a && (idx[j] > ki || (idx[j] == ki && perm[j] > pi))) {
        idx[j + 1] = idx[j];
        perm[j + 1] = perm[j];
        --j;
      }
      idx[j + 1] = ki;
      perm[j + 1] = pi;
    }
  }
}

int mat_build_csc(gnp_mat* A, cudaStream_t st) {
  if (A->csc.ptr) return GNP_OK;
  const int n = A->n;
  const long long nnz = A->nnz;
  int *cnt = nullptr, *totals = nullptr, *fill = nullptr;
  const int nb = (n + SCAN_B - 1) / SCAN_B;
  int s = GNP_OK;
  if ((s = dev_alloc(&A->csc.ptr, (size_t)n + 1)) != GNP_OK) return s;
  if ((s = dev_alloc(&A->csc.idx, (size_t)std::max<long long>(nnz, 1))) != GNP_OK) return s;
  if ((s = dev_alloc(&A->csc.perm, (size_t)std::max<long long>(nnz, 1))) != GNP_OK) return s;
  if ((s = dev_alloc(&cnt, (size_t)n)) != GNP_OK) return s;
  if ((s = dev_alloc(&fill, (size_t)n)) != GNP_OK) { dev_free(cnt); return s; }
  if ((s = dev_alloc(&totals, (size_t)nb)) != GNP_OK) { dev_free(cnt); dev_free(fill); return s; }
  cudaMemsetAsync(cnt, 0, sizeof(int) * n, st);
  cudaMemsetAsync(fill, 0, sizeof(int) * n, st);
  const int gb = 4 * NUM_SMS_GB300;
  if (nnz > 0) k_count_cols<<<gb, 256, 0, st>>>(A->col, nnz, cnt);
  k_scan_blocks<<<nb, SCAN_B, 0, st>>>(cnt, n, A->csc.ptr, totals);
  k_scan_totals<<<1, SCAN_B, 0, st>>>(totals, nb);
  k_scan_add<<<nb, SCAN_B, 0, st>>>(A->csc.ptr, n, totals, nnz);
  if (nnz > 0) {
    k_scatter_csc<<<gb, 256, 0, st>>>(A->rp, A->col, n, A->csc.ptr, fill, A->csc.idx, A->csc.perm);
    k_sort_csc<<<gb, 256, 0, st>>>(A->csc.ptr, n, A->csc.idx, A->csc.perm);
  }
  s = check_launch("csc build");
  cudaError_t e = cudaStreamSynchronize(st);
  dev_free(cnt);
  dev_free(fill);
  dev_free(totals);
  if (s != GNP_OK) return s;
  if (e != cudaSuccess) {
    set_error("csc build: %s", cudaGetErrorString(e));
    return GNP_ERR_CUDA;
  }
  return GNP_OK;
}

// ---------------------------------------------------------------- gamma (Eq. 6)

// gamma = min(max_i sum_j |a_ij|, max_j sum_i |a_ij|).  Thread i sums row i (CSR) and
// column i (CSC, canonical order) sequentially; maxima are order independent.
__global__ void k_gamma(const int* __restrict__ rp, const double* __restrict__ val,
                        const int* __restrict__ cptr, const int* __restrict__ cperm, int n,
                        double* __restrict__ partials, unsigned* counter, double* out) {
  __shared__ double sh[2][32];
  double rmax = 0.0, cmax = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double rs = 0.0, cs = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) rs += fabs(val[e]);
    for (int k = cptr[i]; k < cptr[i + 1]; ++k) cs += fabs(val[cperm[k]]);
    rmax = fmax(rmax, rs);
    cmax = fmax(cmax, cs);
  }
  rmax = warp_max(rmax);
  cmax = warp_max(cmax);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) { sh[0][w] = rmax; sh[1][w] = cmax; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int k = 0; k < nw; ++k) { a = fmax(a, sh[0][k]); b = fmax(b, sh[1][k]); }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
  if (last_block_arrive(counter)) {
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int k = 0; k < (int)gridDim.x; ++k) {
        a = fmax(a, __ldcg(partials + 2 * k));
        b = fmax(b, __ldcg(partials + 2 * k + 1));
      }
      *out = fmin(a, b);
      *counter = 0;
    }
  }
}

int gamma_launch(gnp_mat* A, double* gamma_dev, cudaStream_t st) {
  GNP_TRY(mat_build_csc(A, st));
  const int nb = std::min(4 * NUM_SMS_GB300, std::max(1, (A->n + 255) / 256));
  GNP_TRY(red_alloc(A->red, 4 * NUM_SMS_GB300, 2));
  k_gamma<<<nb, 256, 0, st>>>(A->rp, A->val, A->csc.ptr, A->csc.perm, A->n, A->red.partials,
                              A->red.counter, gamma_dev);
  return check_launch("k_gamma");
}

}  // namespace gnp

using namespace gnp;

extern "C" {

int gnp_mat_create(int n, long long nnz, const int* row_ptr, const int* col, const double* val,
                   int on_device, void* stream, gnp_mat** out) {
  GNP_REQUIRE(out != nullptr, "gnp_mat_create: out is null");
  *out = nullptr;
  GNP_REQUIRE(n >= 1, "gnp_mat_create: n = %d must be >= 1", n);
  GNP_REQUIRE(nnz >= 0 && nnz < (1LL << 31), "gnp_mat_create: nnz = %lld out of range", nnz);
  GNP_REQUIRE(row_ptr && (nnz == 0 || (col && val)), "gnp_mat_create: null array");
  cudaStream_t st = as_stream(stream);
  // validate on the host (device input is copied down once for the check)
  std::vector<int> h_rp((size_t)n + 1), h_col((size_t)nnz);
  if (on_device) {
    GNP_TRY_CUDA(cudaMemcpy(h_rp.data(), row_ptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost));
    if (nnz) GNP_TRY_CUDA(cudaMemcpy(h_col.data(), col, sizeof(int) * nnz, cudaMemcpyDeviceToHost));
  } else {
    std::copy(row_ptr, row_ptr + n + 1, h_rp.begin());
    if (nnz) std::copy(col, col + nnz, h_col.begin());
  }
  if (h_rp[0] != 0 || (long long)h_rp[n] != nnz) {
    set_error("gnp_mat_create: row_ptr[0] = %d, row_ptr[n] = %d, nnz = %lld", h_rp[0], h_rp[n], nnz);
    return GNP_ERR_INVALID_CSR;
  }
  for (int i = 0; i < n; ++i)
    if (h_rp[i + 1] < h_rp[i]) {
      set_error("gnp_mat_create: row_ptr decreases at row %d", i);
      return GNP_ERR_INVALID_CSR;
    }
  for (long long e = 0; e < nnz; ++e)
    if (h_col[e] < 0 || h_col[e] >= n) {
      set_error("gnp_mat_create: col[%lld] = %d outside [0, %d)", e, h_col[e], n);
      return GNP_ERR_INVALID_CSR;
    }
  gnp_mat* A = new gnp_mat();
  A->n = n;
  A->nnz = nnz;
  for (int i = 0; i < n; ++i) A->max_deg = std::max(A->max_deg, h_rp[i + 1] - h_rp[i]);
  cudaGetDevice(&A->device);
  int s = GNP_OK;
  if ((s = dev_alloc(&A->rp, (size_t)n + 1)) != GNP_OK ||
      (s = dev_alloc(&A->col, (size_t)nnz + NNZ_PAD)) != GNP_OK ||
      (s = dev_alloc(&A->val, (size_t)nnz + NNZ_PAD)) != GNP_OK) {
    gnp_mat_destroy(A);
    return s;
  }
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemsetAsync(A->col + nnz, 0, sizeof(int) * NNZ_PAD, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(A->val + nnz, 0, sizeof(double) * NNZ_PAD, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(A->rp, row_ptr, sizeof(int) * (n + 1), kind, st);
  if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(A->col, col, sizeof(int) * nnz, kind, st);
  if (e == cudaSuccess && nnz) e = cudaMemcpyAsync(A->val, val, sizeof(double) * nnz, kind, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_error("gnp_mat_create: copy failed: %s", cudaGetErrorString(e));
    gnp_mat_destroy(A);
    return GNP_ERR_CUDA;
  }
  *out = A;
  return GNP_OK;
}

void gnp_mat_destroy(gnp_mat* A) {
  if (!A) return;
  solver_free(A->solver);
  A->solver = nullptr;
  multi_solver_free(A->msolver);
  A->msolver = nullptr;
  dev_free(A->rp);
  dev_free(A->col);
  dev_free(A->val);
  dev_free(A->csc.ptr);
  dev_free(A->csc.idx);
  dev_free(A->csc.perm);
  dev_free(A->scratch_d);
  red_free(A->red);
  tma_sched_free(A->tma[0]);
  tma_sched_free(A->tma[1]);
  delete A;
}

int gnp_mat_info(const gnp_mat* A, int* n, long long* nnz) {
  GNP_REQUIRE(A != nullptr, "gnp_mat_info: null matrix");
  if (n) *n = A->n;
  if (nnz) *nnz = A->nnz;
  return GNP_OK;
}

int gnp_gamma(const gnp_mat* Ac, double* gamma_out, void* stream) {
  GNP_REQUIRE(Ac && gamma_out, "gnp_gamma: null argument");
  gnp_mat* A = const_cast<gnp_mat*>(Ac);
  cudaStream_t st = as_stream(stream);
  if (!A->scratch_d) GNP_TRY(dev_alloc(&A->scratch_d, (size_t)A->n));
  GNP_TRY(gamma_launch(A, A->scratch_d, st));
  GNP_TRY_CUDA(cudaMemcpyAsync(gamma_out, A->scratch_d, sizeof(double), cudaMemcpyDeviceToHost, st));
  GNP_TRY_CUDA(cudaStreamSynchronize(st));
  return GNP_OK;
}

int gnp_spmv(const gnp_mat* A, const double* x_dev, double* y_dev, void* stream) {
  GNP_REQUIRE(A && x_dev && y_dev, "gnp_spmv: null argument");
  GNP_REQUIRE(x_dev != y_dev, "gnp_spmv: x and y must not overlap");
  return spmv_launch(A, x_dev, nullptr, y_dev, as_stream(stream));
}

}  // extern "C"
