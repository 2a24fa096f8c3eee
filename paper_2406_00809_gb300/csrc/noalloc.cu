// gnp_gamma_noalloc: gamma = min(max row abs-sum, max column abs-sum) (Eq. 6) straight
// from a caller's device CSR, with every byte of scratch in a fixed file-scope device
// array instead of cudaMalloc.
//
// Who needs it: callers that must not allocate device memory when they call in --
// applications whose device memory is owned by an arena or pool of their own (an outside
// cudaMalloc would escape their accounting and limits), plug-ins that a host framework
// hands only a stream and its own buffers, and real-time loops that cannot take the
// implicit device synchronisation of cudaMalloc/cudaFree.  gnp_gamma needs a gnp_mat
// (which allocates a device copy and a transpose); this variant needs nothing but the CSR.
//
// The scratch (column sums, block partials, an arrival counter, an error flag) lives in
// g_noalloc_scratch, NOALLOC_BYTES = 8,398,592 bytes (8 MiB + 9,984 B), which every GPU
// that loads the library holds until the process exits.  Host code must not pass
// g_noalloc_scratch itself to a kernel (on the host that name is only a stand-in); the
// device address comes from cudaGetSymbolAddress, looked up once per device ordinal by
// the first call on that device and cached for the life of the process (the cache does
// not survive cudaDeviceReset of that device).
//
// The column sums are formed with float64 atomicAdd, so their summation order, and with
// it the last bits of gamma, can differ from call to call; every other reduction of the
// library runs in a fixed order.
#include <mutex>

#include "internal.h"

namespace gnp {

constexpr int NOALLOC_MAX_N = 1 << 20;          // largest n accepted
constexpr int NOALLOC_BLOCKS = 4 * NUM_SMS_GB300;  // grid of the reduction kernels
constexpr size_t NOALLOC_BYTES =
    sizeof(double) * NOALLOC_MAX_N + sizeof(double) * 2 * NOALLOC_BLOCKS + 256;  // + counter, flag
static_assert(NOALLOC_BYTES == 8398592, "the documented scratch size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

struct NoallocView {
  double* colsum;    // [NOALLOC_MAX_N]
  double* partials;  // [2 * NOALLOC_BLOCKS]
  unsigned* counter; // arrival counter of the last-block reduction
  unsigned* bad;     // set when the CSR is malformed (row pointers or column indices)
};

// Zero the column sums of this call and the arrival counter.
__global__ void k_noalloc_clear(double* __restrict__ colsum, int n, unsigned* counter, unsigned* bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) colsum[i] = 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *counter = 0u;
    *bad = 0u;
  }
}

// Row absolute sums (their maximum per block) and column absolute sums (atomically).
// The caller's CSR is not validated on the host, so every access stays inside the
// buffers the sizes describe: a row's range is clamped to [0, nnz) and column indices
// outside [0, n) are skipped.  Row pointers that do not start at 0, decrease or do not
// end at nnz, and out-of-range columns, set *bad (gamma becomes NaN).
__global__ void k_noalloc_rows(const int* __restrict__ rp, const int* __restrict__ col,
                               const double* __restrict__ val, int n, int nnz, double* __restrict__ colsum,
                               double* __restrict__ partials, unsigned* bad) {
  __shared__ double sh[32];
  double rmax = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double rs = 0.0;
    int e0 = rp[i], e1 = rp[i + 1];
    if (e0 > e1 || (i == 0 && e0 != 0) || (i == n - 1 && e1 != nnz)) *bad = 1u;
    e0 = max(e0, 0);
    e1 = min(e1, nnz);
    for (int e = e0; e < e1; ++e) {
      const double a = fabs(val[e]);
      const int c = col[e];
      rs += a;
      if ((unsigned)c < (unsigned)n) atomicAdd(colsum + c, a);
      else *bad = 1u;  // the caller's CSR is not validated on the host: skip, report
    }
    rmax = fmax(rmax, rs);
  }
  rmax = warp_max(rmax);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) sh[w] = rmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int k = 0; k < nw; ++k) a = fmax(a, sh[k]);
    partials[2 * blockIdx.x] = a;
  }
}

// Column maxima; the last block forms gamma = min(max row sum, max column sum).
__global__ void k_noalloc_cols(const double* __restrict__ colsum, int n, double* __restrict__ partials,
                               unsigned* counter, const unsigned* bad, double* __restrict__ gamma) {
  __shared__ double sh[32];
  double cmax = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    cmax = fmax(cmax, colsum[i]);
  cmax = warp_max(cmax);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) sh[w] = cmax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int k = 0; k < nw; ++k) a = fmax(a, sh[k]);
    partials[2 * blockIdx.x + 1] = a;
  }
  if (last_block_arrive(counter)) {
    if (threadIdx.x == 0) {
      double r = 0.0, c = 0.0;
      for (int k = 0; k < (int)gridDim.x; ++k) {
        r = fmax(r, __ldcg(partials + 2 * k));
        c = fmax(c, __ldcg(partials + 2 * k + 1));
      }
      *gamma = *bad ? __longlong_as_double(0x7ff8000000000000LL) : fmin(r, c);  // NaN: bad CSR
      *counter = 0u;
    }
  }
}

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[64];  // device address of the scratch, per device ordinal

static int noalloc_view(NoallocView& v) {
  int dev = 0;
  GNP_TRY_CUDA(cudaGetDevice(&dev));
  GNP_REQUIRE(dev >= 0 && dev < 64, "gnp_gamma_noalloc: device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("gnp_gamma_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return GNP_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  unsigned char* base = static_cast<unsigned char*>(g_noalloc_addr[dev]);
  v.colsum = reinterpret_cast<double*>(base);
  v.partials = reinterpret_cast<double*>(base + sizeof(double) * NOALLOC_MAX_N);
  v.counter = reinterpret_cast<unsigned*>(base + sizeof(double) * NOALLOC_MAX_N +
                                          sizeof(double) * 2 * NOALLOC_BLOCKS);
  v.bad = v.counter + 1;
  return GNP_OK;
}

}  // namespace gnp

using namespace gnp;

extern "C" int gnp_gamma_noalloc(int n, long long nnz, const int* row_ptr_dev, const int* col_dev,
                                 const double* val_dev, double* gamma_dev, void* stream) {
  GNP_REQUIRE(row_ptr_dev && gamma_dev && (nnz == 0 || (col_dev && val_dev)),
              "gnp_gamma_noalloc: null argument");
  GNP_REQUIRE(n >= 1 && n <= NOALLOC_MAX_N,
              "gnp_gamma_noalloc: n = %d outside [1, %d], the size of its fixed scratch", n, NOALLOC_MAX_N);
  GNP_REQUIRE(nnz >= 0 && nnz < (1LL << 31), "gnp_gamma_noalloc: nnz = %lld out of range", nnz);
  NoallocView v;
  GNP_TRY(noalloc_view(v));
  cudaStream_t st = as_stream(stream);
  const int nb = std::min(NOALLOC_BLOCKS, std::max(1, (n + 255) / 256));
  k_noalloc_clear<<<nb, 256, 0, st>>>(v.colsum, n, v.counter, v.bad);
  k_noalloc_rows<<<nb, 256, 0, st>>>(row_ptr_dev, col_dev, val_dev, n, (int)nnz, v.colsum, v.partials, v.bad);
  k_noalloc_cols<<<nb, 256, 0, st>>>(v.colsum, n, v.partials, v.counter, v.bad, gamma_dev);
  return check_launch("gnp_gamma_noalloc");
}
