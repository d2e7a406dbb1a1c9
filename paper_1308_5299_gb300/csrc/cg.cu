// Diagonal-preconditioned conjugate gradients on A (the method the paper
// compares against, Sections 1 and 2.4): the preconditioner is the inverse
// of diag(A) = 1/C_l + b_l^2 diag(Y^T N^-1 Y), the latter the Delta m = 0
// ring-formula term (Section 3.3, Eq. Ni-dense).  FP64 throughout; A is the
// plan's FP64 apply_A.  The stop rule is the one of CR-Solve (Fig. code:mg):
// r^T S^-1 r < eps b^T S^-1 b.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "levels.h"

namespace cr {

static int cg_prepare(cr_plan* P) {
  const int64_t nlm = n_lm(P->lmax);
  if (!P->d_pcinv) {
    CR_CUDA(cudaMalloc(&P->d_pcinv, nlm * sizeof(double)));
    std::vector<double> ones(P->lmax + 1, 1.0);
    int rc = inv_diag_A(P, ones, P->d_pcinv);
    if (rc) return rc;
  }
  for (int i = 0; i < 4; ++i)
    if (!P->cgv[i]) CR_CUDA(cudaMalloc(&P->cgv[i], nlm * sizeof(double2)));
  if (!P->d_cgdot) CR_CUDA(cudaMalloc(&P->d_cgdot, 4 * sizeof(double)));
  return CR_OK;
}

// q = A p in FP64 on the observation grid
static int apply_A64(cr_plan* P, const void* p, void* q) {
  return do_sandwich<double>(P, P->obs, P->lmax, p, q, P->d_bl, P->d_ninv, P->d_bl, P->d_sinv, nullptr, nullptr);
}

// z = d * r (d real per coefficient)
static int precond(cr_plan* P, const void* r, void* z) {
  const int64_t nlm = n_lm(P->lmax);
  CR_CUDA(cudaMemsetAsync(z, 0, nlm * sizeof(double2), P->stream));
  return launch_diag_axpy<double>(z, r, P->d_pcinv, nlm, P->stream);
}

static int dots(cr_plan* P, int n, const void* const* a, const void* const* b, const double* const* w,
                double* out) {
  for (int i = 0; i < n; ++i) {
    int rc = launch_dot<double>(a[i], b[i], w[i], P->lmax, P->d_cgdot + i, P->d_dotpart, P->stream);
    if (rc) return rc;
  }
  CR_CUDA(cudaMemcpyAsync(out, P->d_cgdot, n * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  CR_CUDA(cudaStreamSynchronize(P->stream));
  return CR_OK;
}

int cg_solve(cr_plan* P, void* x, const void* b, double eps, int maxit, int* it_out, double* relres_out,
             double* history) {
  int rc = cg_prepare(P);
  if (rc) return rc;
  const int L = P->lmax;
  const int64_t nlm = n_lm(L);
  const size_t bytes = nlm * sizeof(double2);
  void *r = P->cgv[0], *z = P->cgv[1], *pv = P->cgv[2], *q = P->cgv[3];
  double d[2];
  {
    const void* a1[1] = {b};
    const double* w1[1] = {P->d_sinv};
    if ((rc = dots(P, 1, a1, a1, w1, d))) return rc;
  }
  const double bsb = d[0];
  CR_CUDA(cudaMemsetAsync(x, 0, bytes, P->stream));
  if (it_out) *it_out = 0;
  if (relres_out) *relres_out = 0.0;
  if (!(bsb > 0.0)) return CR_OK;
  CR_CUDA(cudaMemcpyAsync(r, b, bytes, cudaMemcpyDeviceToDevice, P->stream));
  if ((rc = precond(P, r, z))) return rc;
  CR_CUDA(cudaMemcpyAsync(pv, z, bytes, cudaMemcpyDeviceToDevice, P->stream));
  {
    const void* a1[1] = {r};
    const void* b1[1] = {z};
    const double* w1[1] = {nullptr};
    if ((rc = dots(P, 1, a1, b1, w1, d))) return rc;
  }
  double rz = d[0], rel = 1.0;
  int k;
  for (k = 1; k <= maxit; ++k) {
    {
      TimerScope ts(P->timing, P->stream, "cg_apply_A");
      if ((rc = apply_A64(P, pv, q))) return rc;
    }
    {
      const void* a1[1] = {pv};
      const void* b1[1] = {q};
      const double* w1[1] = {nullptr};
      if ((rc = dots(P, 1, a1, b1, w1, d))) return rc;
    }
    if (!(d[0] > 0.0)) return fail(CR_ENONFINITE, "cg: non-positive curvature p^T A p");
    const double alpha = rz / d[0];
    if ((rc = launch_axpby(x, alpha, pv, 1.0, nlm, P->stream))) return rc;  // x += alpha p
    if ((rc = launch_axpby(r, -alpha, q, 1.0, nlm, P->stream))) return rc;  // r -= alpha q
    if ((rc = precond(P, r, z))) return rc;
    {
      const void* a2[2] = {r, r};
      const void* b2[2] = {r, z};
      const double* w2[2] = {P->d_sinv, nullptr};
      if ((rc = dots(P, 2, a2, b2, w2, d))) return rc;
    }
    rel = std::sqrt(std::max(d[0], 0.0) / bsb);
    if (history) history[k - 1] = rel;
    if (!std::isfinite(rel)) {
      if (it_out) *it_out = k;
      if (relres_out) *relres_out = rel;
      return fail(CR_ENONFINITE, "cg: non-finite residual");
    }
    if (rel * rel < eps) break;
    const double beta = d[1] / rz;
    rz = d[1];
    if ((rc = launch_axpby(pv, 1.0, z, beta, nlm, P->stream))) return rc;  // p = z + beta p
  }
  if (it_out) *it_out = std::min(k, maxit);
  if (relres_out) *relres_out = rel;
  if (k > maxit) return fail(CR_EMAXITER, "cg: iteration cap reached before the tolerance");
  return CR_OK;
}

}  // namespace cr
