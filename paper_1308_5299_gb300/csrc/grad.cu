// Gradients of a constrained realization and of the Wiener-filter
// log-likelihood with respect to C_l and the inverse-noise map (the system
// of Section 2.3, Eq. system-explicit, differentiated; A is symmetric, so the
// adjoint solve lambda = A^-1 g reuses CR-Solve).
//
// With x = A^-1 b, b = B Y^T (N^-1 d + N^-1/2 w2) + S^-1/2 w1 and a loss L(x)
// of gradient g (dL = <g, dx>), lambda = A^-1 g gives
//   dL/dC_l = C_l^-2 <lambda, x>_l - 1/2 C_l^-3/2 <lambda, w1>_l,
//   dL/dn_i = -(Y B lambda)_i (Y B x)_i + (Y B lambda)_i (d_i + w2_i / (2 sqrt n_i)),
// <.,.>_l the real inner product restricted to multipole l (w1 in complex
// storage: w_l0, (w_re + i w_im) / sqrt2).  The Wiener-filter data term
// -1/2 (d^T N^-1 d - b^T A^-1 b), b = B Y^T N^-1 d, has
//   d/dC_l = 1/2 C_l^-2 <xh, xh>_l,  d/dn_i = -1/2 (d_i - (Y B xh)_i)^2,
// xh = A^-1 b.  Both are instances of the two kernels below.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "levels.h"
#include "philox.cuh"

namespace cr {

// out_l (+)= alpha C_l^-2 <u, v>_l + beta C_l^-3/2 <u, w1>_l + kappa (2l+1) / C_l
// (0 where C_l = 0)
__global__ void grad_cl_kernel(const double2* u, const double2* v, const double* sinv, int L, double alpha,
                               double beta, double kappa, uint64_t seed, uint32_t rhs, int acc, double* out) {
  const int l = blockIdx.x;
  __shared__ double red[256];
  double s1 = 0.0, s2 = 0.0;
  for (int m = threadIdx.x; m <= l; m += blockDim.x) {
    const int64_t i = lm_off(L, m) + (l - m);
    const double2 a = u[i];
    const double w = (m == 0) ? 1.0 : 2.0;
    if (v) {
      const double2 c = v[i];
      s1 += w * (a.x * c.x + (m ? a.y * c.y : 0.0));
    }
    if (beta != 0.0) {
      const double wr = draw_normal(seed, 3u, rhs, 2 * (uint64_t)i);
      if (m == 0) {
        s2 += a.x * wr;
      } else {
        const double wi = draw_normal(seed, 3u, rhs, 2 * (uint64_t)i + 1);
        s2 += w * M_SQRT1_2 * (a.x * wr + a.y * wi);
      }
    }
  }
  // fixed-order block reduction (deterministic)
  red[threadIdx.x] = s1;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double t1 = red[0];
  __syncthreads();
  red[threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double si = sinv[l];
    const double g = (si > 0.0) ? alpha * si * si * t1 + beta * si * sqrt(si) * red[0] + kappa * (2.0 * l + 1.0) * si
                                : 0.0;
    out[l] = acc ? out[l] + g : g;
  }
}

// out_i (+)= alpha p_i q_i + p_i (gamma d_i + delta w2_i / sqrt n_i) + eps d_i^2 + kappa / n_i
// (the w2 and 1/n terms only where n_i > 0; q may be null: its term is 0)
__global__ void grad_ninv_kernel(const double* p, const double* q, const double* d, const double* ninv, double alpha,
                                 double gamma, double delta, double eps, double kappa, uint64_t seed, uint32_t rhs,
                                 int acc, int64_t npix, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
    const double pi = p[i];
    double r = q ? alpha * pi * q[i] : 0.0;
    if (d) {
      const double di = d[i];
      r += gamma * pi * di + eps * di * di;
    }
    const double n = ninv[i];
    if (delta != 0.0 && n > 0.0) r += delta * pi * draw_normal(seed, 4u, rhs, (uint64_t)i) / sqrt(n);
    if (kappa != 0.0 && n > 0.0) r += kappa / n;
    out[i] = acc ? out[i] + r : r;
  }
}

// Rademacher probes: element k of stream s for probe j takes word k & 3 of
// Philox4x32-10 at counter (k >> 2, k >> 34, s, j); sign + for an even word.
__device__ __forceinline__ double rademacher(uint64_t seed, uint32_t stream, uint32_t j, uint64_t k) {
  const U4 x = philox4x32_10((uint32_t)(k >> 2), (uint32_t)(k >> 34), stream, j, (uint32_t)seed, (uint32_t)(seed >> 32));
  return (x.x[k & 3] & 1u) ? -1.0 : 1.0;
}

// coefficient probe in the real orthonormal basis: a_l0 = z, a_lm = (z_re + i z_im) / sqrt2
__global__ void probe_alm_kernel(const double* sinv, int L, uint64_t seed, uint32_t j, double2* out) {
  const int m = blockIdx.x;
  const int64_t o = lm_off(L, m);
  for (int l = m + threadIdx.x; l <= L; l += blockDim.x) {
    const int64_t i = o + (l - m);
    double2 v = make_double2(0.0, 0.0);
    if (sinv[l] > 0.0) {
      const double zr = rademacher(seed, 5u, j, 2 * (uint64_t)i);
      if (m == 0) {
        v.x = zr;
      } else {
        v.x = zr * M_SQRT1_2;
        v.y = rademacher(seed, 5u, j, 2 * (uint64_t)i + 1) * M_SQRT1_2;
      }
    }
    out[i] = v;
  }
}

// pixel probe on observed pixels (n_i > 0)
__global__ void probe_map_kernel(const double* ninv, int64_t npix, uint64_t seed, uint32_t j, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = ninv[i] > 0.0 ? rademacher(seed, 6u, j, (uint64_t)i) : 0.0;
}

// sum_i n_i a_i b_i, fixed-order two-pass reduction
__global__ void wdot_partial_kernel(const double* a, const double* b, const double* n, int64_t npix, double* part) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x)
    s += n[i] * a[i] * b[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

}  // namespace cr

using namespace cr;

extern "C" int cr_grad_cl(cr_plan* plan, const void* u, const void* v, double alpha, double beta, double kappa,
                          uint64_t seed, int rhs, int accumulate, double* out) {
  if (!plan || !u || !out) return fail(CR_EINVAL, "cr_grad_cl: null argument");
  if (!plan->has_op) return fail(CR_EINVAL, "cr_grad_cl: the plan needs C_l");
  if (rhs < 0) return fail(CR_EINVAL, "cr_grad_cl: rhs < 0");
  const int L = plan->lmax;
  { grad_cl_kernel<<<L + 1, 256, 0, plan->stream>>>((const double2*)u, (const double2*)v, plan->d_sinv, L, alpha,
                                                     beta, kappa, seed, (uint32_t)rhs, accumulate ? 1 : 0, out);
    count_launch(); }
  CR_CHECK_LAUNCH("grad_cl_kernel");
  CR_CUDA(cudaStreamSynchronize(plan->stream));
  return CR_OK;
}

extern "C" int cr_grad_ninv(cr_plan* plan, const void* u, const void* v, const double* d, double alpha, double gamma,
                            double delta, double eps, double kappa, uint64_t seed, int rhs, int accumulate,
                            double* out) {
  if (!plan || !u || !out) return fail(CR_EINVAL, "cr_grad_ninv: null argument");
  if (!plan->has_op) return fail(CR_EINVAL, "cr_grad_ninv: the plan needs C_l, b_l and N^-1");
  if (rhs < 0) return fail(CR_EINVAL, "cr_grad_ninv: rhs < 0");
  const Grid& g = plan->obs;
  double *p = nullptr, *q = nullptr;
  CR_CUDA(cudaMalloc(&p, g.npix * sizeof(double)));
  cudaError_t e = cudaMalloc(&q, g.npix * sizeof(double));
  if (e != cudaSuccess) {
    cudaFree(p);
    return cuda_fail(e, "cudaMalloc(grad maps)");
  }
  int rc = do_synth<double>(plan, g, plan->lmax, u, p, plan->d_bl);
  if (!rc && v) rc = do_synth<double>(plan, g, plan->lmax, v, q, plan->d_bl);
  if (!rc) {
    { grad_ninv_kernel<<<1024, 256, 0, plan->stream>>>(p, v ? q : nullptr, d, plan->d_ninv, alpha, gamma, delta, eps,
                                                        kappa, seed, (uint32_t)rhs, accumulate ? 1 : 0, g.npix, out);
      count_launch(); }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(plan->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "grad_ninv_kernel");
  }
  cudaFree(p);
  cudaFree(q);
  return rc;
}

extern "C" int cr_map_wdot(cr_plan* plan, const double* a, const double* b, double* out) {
  if (!plan || !a || !b || !out) return fail(CR_EINVAL, "cr_map_wdot: null argument");
  if (!plan->has_op) return fail(CR_EINVAL, "cr_map_wdot: the plan needs N^-1");
  const int nb = 512;
  double* part = nullptr;
  CR_CUDA(cudaMalloc(&part, nb * sizeof(double)));
  { wdot_partial_kernel<<<nb, 256, 0, plan->stream>>>(a, b, plan->d_ninv, plan->obs.npix, part); count_launch(); }
  cudaError_t e = cudaGetLastError();
  std::vector<double> h(nb);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, nb * sizeof(double), cudaMemcpyDeviceToHost, plan->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(plan->stream);
  cudaFree(part);
  if (e != cudaSuccess) return cuda_fail(e, "cr_map_wdot");
  double s = 0.0;
  for (double v : h) s += v;
  *out = s;
  return CR_OK;
}

extern "C" int cr_alm_dot(cr_plan* plan, const void* u, const void* v, int weighted, double* out) {
  if (!plan || !u || !v || !out) return fail(CR_EINVAL, "cr_alm_dot: null argument");
  if (weighted && !plan->has_op) return fail(CR_EINVAL, "cr_alm_dot: S^-1 weighting needs C_l");
  double* d = nullptr;
  CR_CUDA(cudaMalloc(&d, sizeof(double)));
  int rc = launch_dot<double>(u, v, weighted ? plan->d_sinv : nullptr, plan->lmax, d, plan->d_dotpart, plan->stream);
  cudaError_t e = cudaSuccess;
  if (!rc) e = cudaMemcpyAsync(out, d, sizeof(double), cudaMemcpyDeviceToHost, plan->stream);
  if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(plan->stream);
  cudaFree(d);
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "cr_alm_dot");
  return rc;
}

extern "C" int cr_probe(cr_plan* plan, uint64_t seed, int kind, int j, void* out) {
  if (!plan || !out || j < 0) return fail(CR_EINVAL, "cr_probe: null argument or j < 0");
  if (!plan->has_op) return fail(CR_EINVAL, "cr_probe: the plan needs C_l and N^-1");
  if (kind == CR_PROBE_ALM) {
    { probe_alm_kernel<<<plan->lmax + 1, 128, 0, plan->stream>>>(plan->d_sinv, plan->lmax, seed, (uint32_t)j,
                                                                  (double2*)out); count_launch(); }
  } else if (kind == CR_PROBE_MAP) {
    { probe_map_kernel<<<1024, 256, 0, plan->stream>>>(plan->d_ninv, plan->obs.npix, seed, (uint32_t)j, (double*)out);
      count_launch(); }
  } else {
    return fail(CR_EINVAL, "cr_probe: kind must be CR_PROBE_ALM or CR_PROBE_MAP");
  }
  CR_CHECK_LAUNCH("probe kernel");
  CR_CUDA(cudaStreamSynchronize(plan->stream));
  return CR_OK;
}
