// Right-hand sides of the CR system (Section 2.3):
//   b = B Y^T N^-1 d + S^-1/2 omega_1 + B Y^T N^-1/2 omega_2,
// omega_1 ~ N(0, I) in the real orthonormal coefficient basis, omega_2 ~
// N(0, I) per pixel (N^-1/2 = 0 under the mask); without the omega terms b
// is the Wiener-filter right-hand side.  With d = 0, Cov(b) = A, so
// x = A^-1 b carries the fluctuations of a constrained realization.
//
// Normals: Philox4x32-10 (Salmon, Moraes, Dror, Shaw 2011) from its
// published round function and key schedule, Box-Muller in FP64.  Element k
// of stream s for right-hand side j: counter (k >> 2, 0, s, j), key (seed low,
// seed high), slot k & 3 of the pairs (x0, x1) -> 0, 1 and (x2, x3) -> 2, 3,
// u = (x + 1/2) 2^-32, z = sqrt(-2 ln u_a) (cos, sin)(2 pi u_b).  Streams:
// 3 = omega_1 (element 2 i + part of coefficient i), 4 = omega_2 (pixel i).
#include <cmath>

#include "common.cuh"
#include "kernels.h"
#include "philox.cuh"

namespace cr {

// map_i = N^-1_i d_i + sqrt(N^-1_i) omega_2,i
__global__ void draw_map_kernel(const double* ninv, const double* d, int fluct, int plain, uint64_t seed, uint32_t rhs,
                                int64_t npix, double* map) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
    const double n = ninv[i];
    double v = d ? (plain ? d[i] : n * d[i]) : 0.0;
    if (fluct) v += sqrt(fmax(n, 0.0)) * draw_normal(seed, 4u, rhs, (uint64_t)i);
    map[i] = v;
  }
}

// b_lm += C_l^-1/2 omega_1 (active l only; real basis: a_l0 = w, a_lm = (w_re + i w_im) / sqrt2)
__global__ void draw_prior_kernel(const double* sinv, int L, uint64_t seed, uint32_t rhs, double2* b) {
  const int m = blockIdx.x;
  const int64_t o = lm_off(L, m);
  for (int l = m + threadIdx.x; l <= L; l += blockDim.x) {
    const double si = sinv[l];
    if (!(si > 0.0)) continue;
    const int64_t i = o + (l - m);
    const double wr = draw_normal(seed, 3u, rhs, 2 * (uint64_t)i);
    const double sc = sqrt(si);
    double2 v = b[i];
    if (m == 0) {
      v.x += sc * wr;
    } else {
      const double wi = draw_normal(seed, 3u, rhs, 2 * (uint64_t)i + 1);
      v.x += sc * wr * M_SQRT1_2;
      v.y += sc * wi * M_SQRT1_2;
    }
    b[i] = v;
  }
}

}  // namespace cr

using namespace cr;

extern "C" int cr_draw(cr_plan* plan, uint64_t seed, const void* d, void* b, int nrhs, int flags) {
  if (!plan || !b || nrhs < 1) return fail(CR_EINVAL, "cr_draw: null plan / output or nrhs < 1");
  if (!plan->has_op) return fail(CR_EINVAL, "cr_draw: the plan needs C_l, b_l and N^-1");
  if (flags & ~(CR_DRAW_FLUCT | CR_DRAW_PLAIN)) return fail(CR_EINVAL, "cr_draw: unknown flag");
  const int fluct = (flags & CR_DRAW_FLUCT) ? 1 : 0;
  const int plain = (flags & CR_DRAW_PLAIN) ? 1 : 0;
  const Grid& g = plan->obs;
  const int L = plan->lmax;
  const int64_t nlm = n_lm(L);
  double* map = nullptr;
  CR_CUDA(cudaMalloc(&map, g.npix * sizeof(double)));
  int rc = CR_OK;
  for (int j = 0; j < nrhs && !rc; ++j) {
    double2* bj = reinterpret_cast<double2*>(b) + (int64_t)j * nlm;
    const double* dj = d ? reinterpret_cast<const double*>(d) + (int64_t)j * g.npix : nullptr;
    { draw_map_kernel<<<1024, 256, 0, plan->stream>>>(plan->d_ninv, dj, fluct, plain, seed, (uint32_t)j, g.npix, map);
      count_launch(); }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "draw_map_kernel");
      break;
    }
    rc = do_adjoint<double>(plan, g, L, map, bj, plan->d_bl, nullptr, nullptr, 0);
    if (!rc && fluct) {
      { draw_prior_kernel<<<L + 1, 128, 0, plan->stream>>>(plan->d_sinv, L, seed, (uint32_t)j, bj); count_launch(); }
      e = cudaGetLastError();
      if (e != cudaSuccess) rc = cuda_fail(e, "draw_prior_kernel");
    }
  }
  cudaError_t e = cudaStreamSynchronize(plan->stream);
  cudaFree(map);
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "cr_draw");
  return rc;
}
