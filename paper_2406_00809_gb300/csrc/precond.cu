// Right preconditioners other than the GNP for FGMRES: Jacobi and inner GMRES, the
// simple baselines the paper compares the GNP with (Sec. 3 "Compared methods"), and the
// gnp_precond handle that also wraps a GNP or the identity.
//
//   k_diag_inv    1 / a_ii per row (a row without a stored or with a zero diagonal
//                 gets 1, so z_i = v_i there).  Once, at creation.
//   k_jacobi_col  z = D^-1 v, v first normalised by the outer step's scale (fused, so
//                 the Jacobi step costs one read of v and dinv and two writes).
// Inner GMRES runs on krylov.cu's kernels (inner_gmres_launch).
#include <algorithm>

#include "solver.h"

struct gnp_precond {
  gnp_mat* A = nullptr;
  int kind = GNP_PRECOND_IDENTITY;
  gnp_model* M = nullptr;          // GNP (not owned)
  double* dinv = nullptr;          // Jacobi [n]
  gnp::InnerGmres* inner = nullptr;
  float* zf = nullptr;             // GNP: float32 output of gnp_precond_apply before widening
};

namespace gnp {

__global__ void __launch_bounds__(RED_THREADS)
k_diag_inv(const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val, int n,
           double* __restrict__ dinv) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k)
      if (col[k] == i) d += val[k];  // duplicates of a diagonal entry add up, as in A x
    dinv[i] = d != 0.0 ? 1.0 / d : 1.0;
  }
}

__global__ void __launch_bounds__(RED_THREADS)
k_jacobi_col(const double* __restrict__ dinv, ColPtr vp, DevState* outer, ColPtr zp, int n) {
  if (outer && !outer->active) return;
  const int jv = vp.jptr ? *vp.jptr : 0;
  const int jz = zp.jptr ? *zp.jptr : 0;
  double* v = reinterpret_cast<double*>(static_cast<char*>(vp.base) + (size_t)(jv + vp.off) * vp.stride);
  double* z = reinterpret_cast<double*>(static_cast<char*>(zp.base) + (size_t)(jz + zp.off) * zp.stride);
  const double s = outer ? outer->vscale : 1.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double t = v[i];
    if (outer) {
      t = t / s;
      v[i] = t;
    }
    z[i] = t * dinv[i];
  }
}

__global__ void k_widen(const float* __restrict__ a, double* __restrict__ b, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = (double)a[i];
}

int jacobi_launch(const double* dinv, ColPtr v, DevState* outer, ColPtr z, int n, cudaStream_t st) {
  k_jacobi_col<<<red_blocks(n), RED_THREADS, 0, st>>>(dinv, v, outer, z, n);
  return check_launch("k_jacobi_col");
}

Prec precond_view(gnp_precond* P) {
  Prec v;
  v.kind = P->kind;
  v.M = P->M;
  v.dinv = P->dinv;
  v.inner = P->inner;
  v.key = P;
  return v;
}

const gnp_mat* precond_matrix(const gnp_precond* P) { return P->A; }

}  // namespace gnp

using namespace gnp;

extern "C" void gnp_precond_destroy(gnp_precond* P) {
  if (!P) return;
  dev_free(P->dinv);
  dev_free(P->zf);
  inner_gmres_free(P->inner);
  delete P;
}

extern "C" int gnp_precond_create(gnp_mat* A, int kind, gnp_model* M, int inner_iters, double inner_rtol,
                                  gnp_precond** out) {
  GNP_REQUIRE(A && out, "gnp_precond_create: null argument");
  *out = nullptr;
  GNP_REQUIRE(kind >= GNP_PRECOND_IDENTITY && kind <= GNP_PRECOND_GMRES, "gnp_precond_create: kind %d", kind);
  if (kind == GNP_PRECOND_GNP) {
    GNP_REQUIRE(M, "gnp_precond_create: GNP kind needs a model");
    GNP_REQUIRE(M->A == A, "gnp_precond_create: the model was built for another matrix");
  }
  if (kind == GNP_PRECOND_GMRES) {
    GNP_REQUIRE(inner_iters >= 1 && inner_iters <= GNP_MAX_RESTART, "gnp_precond_create: inner_iters %d out of [1, %d]",
                inner_iters, GNP_MAX_RESTART);
    GNP_REQUIRE(inner_rtol >= 0.0, "gnp_precond_create: inner_rtol < 0");
  }
  gnp_precond* P = new gnp_precond();
  P->A = A;
  P->kind = kind;
  P->M = kind == GNP_PRECOND_GNP ? M : nullptr;
  int e = GNP_OK;
  if (kind == GNP_PRECOND_JACOBI) {
    e = dev_alloc(&P->dinv, (size_t)A->n);
    if (e == GNP_OK) {
      k_diag_inv<<<red_blocks(A->n), RED_THREADS>>>(A->rp, A->col, A->val, A->n, P->dinv);
      e = check_launch("k_diag_inv");
      if (e == GNP_OK && cudaDeviceSynchronize() != cudaSuccess) {
        set_error("gnp_precond_create: %s", cudaGetErrorString(cudaGetLastError()));
        e = GNP_ERR_CUDA;
      }
    }
  } else if (kind == GNP_PRECOND_GMRES) {
    e = inner_gmres_create(A->n, inner_iters, inner_rtol, &P->inner);
  } else if (kind == GNP_PRECOND_GNP) {
    e = dev_alloc(&P->zf, (size_t)A->n);
  }
  if (e != GNP_OK) {
    gnp_precond_destroy(P);
    return e;
  }
  *out = P;
  return GNP_OK;
}

extern "C" int gnp_precond_apply(gnp_precond* P, const double* v, double* z, void* stream) {
  GNP_REQUIRE(P && v && z, "gnp_precond_apply: null argument");
  GNP_REQUIRE(v != z, "gnp_precond_apply: v and z must be distinct");
  cudaStream_t st = as_stream(stream);
  const int n = P->A->n;
  if (n == 0) return GNP_OK;
  ColPtr vc{const_cast<double*>(v), 0, nullptr, 0};
  ColPtr zc{z, 0, nullptr, 0};
  switch (P->kind) {
    case GNP_PRECOND_IDENTITY:
      GNP_TRY_CUDA(cudaMemcpyAsync(z, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
      return GNP_OK;
    case GNP_PRECOND_JACOBI:
      return jacobi_launch(P->dinv, vc, nullptr, zc, n, st);
    case GNP_PRECOND_GMRES:
      return inner_gmres_launch(P->A, P->inner, vc, nullptr, zc, st);
    default: {
      GNP_TRY(apply_prepare(P->M));
      ColPtr zf{P->zf, 0, nullptr, 0};
      GNP_TRY(apply_launch(P->M, vc, nullptr, zf, nullptr, nullptr, st));
      k_widen<<<red_blocks(n), RED_THREADS, 0, st>>>(P->zf, z, n);
      return check_launch("k_widen");
    }
  }
}
