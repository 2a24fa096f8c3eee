// Error reporting, status names and small allocation helpers.
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstring>

#include "internal.h"

namespace gnp {

static thread_local char g_err[1024] = "no error";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("launch of %s failed: %s", what, cudaGetErrorString(e));
    return GNP_ERR_CUDA;
  }
  return GNP_OK;
}

int red_alloc(RedScratch& r, int max_blocks, int max_k) {
  if (r.partials && r.max_blocks >= max_blocks && r.max_k >= max_k) return GNP_OK;
  red_free(r);
  GNP_TRY(dev_alloc(&r.partials, (size_t)max_blocks * max_k));
  GNP_TRY(dev_alloc(&r.counter, 1));
  GNP_TRY_CUDA(cudaMemset(r.counter, 0, sizeof(unsigned)));
  r.max_blocks = max_blocks;
  r.max_k = max_k;
  return GNP_OK;
}

void red_free(RedScratch& r) {
  dev_free(r.partials);
  dev_free(r.counter);
  r.max_blocks = r.max_k = 0;
}

}  // namespace gnp

extern "C" {

const char* gnp_status_string(int s) {
  switch (s) {
    case GNP_OK: return "GNP_OK";
    case GNP_ERR_INVALID_ARG: return "GNP_ERR_INVALID_ARG";
    case GNP_ERR_INVALID_CSR: return "GNP_ERR_INVALID_CSR";
    case GNP_ERR_OOM: return "GNP_ERR_OOM";
    case GNP_ERR_CUDA: return "GNP_ERR_CUDA";
    case GNP_ERR_BREAKDOWN: return "GNP_ERR_BREAKDOWN";
    case GNP_ERR_STAGNATION: return "GNP_ERR_STAGNATION";
    case GNP_ERR_RESIDUAL_MISMATCH: return "GNP_ERR_RESIDUAL_MISMATCH";
    case GNP_ERR_NOT_CONVERGED: return "GNP_ERR_NOT_CONVERGED";
    case GNP_ERR_TIMEOUT: return "GNP_ERR_TIMEOUT";
    case GNP_ERR_NAN: return "GNP_ERR_NAN";
    case GNP_ERR_BUSY: return "GNP_ERR_BUSY";
    default: return "GNP_ERR_UNKNOWN";
  }
}

const char* gnp_last_error(void) { return gnp::g_err; }

// Sec. 3 "Evaluation metrics": areas under the log10 relative-residual curve above
// log10 rtol, per iteration (from i = 0) and per unit of time (from i = 1, each term
// weighted by the time that iteration took).
static double log_excess(double r, double lrtol) { return std::log10(r > 0.0 ? r : DBL_MIN) - lrtol; }

double gnp_iter_auc(const double* res_history, int len, double rtol) {
  if (!res_history || len < 1 || !(rtol > 0.0)) return NAN;
  const double lr = std::log10(rtol);
  double s = 0.0;
  for (int i = 0; i < len; ++i) s += log_excess(res_history[i], lr);
  return s;
}

double gnp_time_auc(const double* res_history, const double* time_history, int len, double rtol) {
  if (!res_history || !time_history || len < 1 || !(rtol > 0.0)) return NAN;
  const double lr = std::log10(rtol);
  double s = 0.0;
  for (int i = 1; i < len; ++i) s += log_excess(res_history[i], lr) * (time_history[i] - time_history[i - 1]);
  return s;
}

int gnp_weight_count(int L) {
  if (L < 0 || L > GNP_MAX_LAYERS) return -1;
  return gnp::weight_count(L);
}

}  // extern "C"
