// Top-level diagonal smoother and bottom dense level (Section 3.2), both from
// the ring formula of Section 3.3 (Eq. Ni-dense):
//   (Y^T N^-1 Y)_{l1 m1, l2 m2} = sum_k P~_l1m1(z_k) P~_l2m2(z_k) X_k(m1 - m2),
//   X_k(d) = sum_j xi_kj e^{-i d phi_kj}   (per-ring DFT of the N^-1 map).
// For real fields in m >= 0 storage a second term with X_k(m1 + m2) appears:
//   (Y^T N Y a)_{l1 m1} = sum_k P1 sum_{l2 m2} (w_m2 / 2) P2
//                         [a_{l2 m2} X_k(m1 - m2) + conj(a_{l2 m2}) X_k(m1 + m2)].
// Top level: diag(A)_lm ~ 1/C_l + (b_l p_l)^2 sum_k P~_lm(z_k)^2 X_k(0) (the
// Delta m = 0 term), applied as x += (1 - f^1_l) r / diag(A).
// Bottom: the real-basis matrix of A_bottom = D + B M B over l <= l_dense,
// factorised by Cholesky and inverted once (FP64); each bottom solve is one
// dense matrix-vector product.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"
#include "hier.h"
#include "kernels.h"
#include "levels.h"

namespace cr {

// X_k(d) = sum_j n_kj e^{-i d phi_j}, phi_j = pi (2 j + s) / n, d = 0..dmax
__global__ void ring_dft_kernel(const RingFFT* fft, const double2* tab_all, const double* ninv, int dmax, double2* X) {
  const int r = blockIdx.x;
  const RingFFT f = fft[r];
  const double2* tab = tab_all + f.tab;
  const int64_t twon = 2 * (int64_t)f.n;
  __shared__ double sv[256];
  double2 acc = make_double2(0.0, 0.0);
  const int d = threadIdx.x;
  for (int j0 = 0; j0 < f.n; j0 += 256) {
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += blockDim.x) sv[t] = (j0 + t < f.n) ? ninv[f.off + j0 + t] : 0.0;
    __syncthreads();
    if (d <= dmax) {
      const int jn = min(256, f.n - j0);
      for (int t = 0; t < jn; ++t) {
        const int64_t u = ((int64_t)d * (2 * (int64_t)(j0 + t) + f.shift)) % twon;
        const double2 e = tab[u];  // e^{i pi u / n}
        acc.x = fma(sv[t], e.x, acc.x);
        acc.y = fma(-sv[t], e.y, acc.y);
      }
    }
  }
  if (d <= dmax) X[(int64_t)r * (dmax + 1) + d] = acc;
}

// P~_lm(z_pair) for l <= Ld, [pair][lm(Ld)], from the plan's recurrence
// tables and scaled seeds (values while the level is below 0 are negligible).
__global__ void ptab_kernel(const double* z, const double* seed, const int* lev, int ld_seed, const double* c,
                            const double* s, int Lc, int Ld, int npairs, double* out) {
  const int m = blockIdx.x;
  const int p = blockIdx.y * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const double zz = z[p];
  int e = lev[(int64_t)m * ld_seed + p];
  double q1 = 0.0, q2 = -seed[(int64_t)m * ld_seed + p];
  const int64_t oc = lm_off(Lc, m), oo = lm_off(Ld, m);
  const int64_t nlm = n_lm(Ld);
  for (int l = m; l <= Ld; ++l) {
    const double q = fma(c[oc + l - m] * zz, q1, -q2);
    q2 = q1;
    q1 = q;
    if (e < 0 && fabs(q1) > 0x1p300) {
      q1 *= 0x1p-600;
      q2 *= 0x1p-600;
      e += 1;
    }
    // q1 (not q): the state may just have been renormalised
    out[(int64_t)p * nlm + oo + (l - m)] = (e == 0) ? q1 * s[oc + l - m] : 0.0;
  }
}

struct DofMap {
  int l, m, part;  // part 0 = Re (or the m = 0 real value), 1 = Im
};

// Real-basis entries of B (Y^T N^-1 Y) B + D over the active dofs.
__global__ void assemble_dense_kernel(const double* ptab, const double2* X, int dmax, int npairs, int nring, int Ld,
                                      const DofMap* dofs, int nd, const double* bl, const double* dl, double* A) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)nd * nd) return;
  const int r = (int)(e / nd), c = (int)(e % nd);
  const DofMap a = dofs[r], b = dofs[c];
  const int64_t nlm = n_lm(Ld);
  const int64_t i1 = lm_off(Ld, a.m) + (a.l - a.m), i2 = lm_off(Ld, b.m) + (b.l - b.m);
  const int dm = a.m - b.m, sm = a.m + b.m;
  const bool even = ((a.l + a.m + b.l + b.m) & 1) == 0;
  double2 T1 = make_double2(0.0, 0.0), T2 = make_double2(0.0, 0.0);
  for (int p = 0; p < npairs; ++p) {
    const double pp = ptab[(int64_t)p * nlm + i1] * ptab[(int64_t)p * nlm + i2];
    const int rs = nring - 1 - p;
    const bool mid = (rs == p);
    double2 x1 = X[(int64_t)p * (dmax + 1) + abs(dm)];
    double2 x2 = X[(int64_t)p * (dmax + 1) + sm];
    if (!mid) {
      const double sg = even ? 1.0 : -1.0;
      const double2 y1 = X[(int64_t)rs * (dmax + 1) + abs(dm)];
      const double2 y2 = X[(int64_t)rs * (dmax + 1) + sm];
      x1.x += sg * y1.x;
      x1.y += sg * y1.y;
      x2.x += sg * y2.x;
      x2.y += sg * y2.y;
    }
    if (dm < 0) x1.y = -x1.y;  // X(-d) = conj X(d)
    T1.x = fma(pp, x1.x, T1.x);
    T1.y = fma(pp, x1.y, T1.y);
    T2.x = fma(pp, x2.x, T2.x);
    T2.y = fma(pp, x2.y, T2.y);
  }
  // column b: unit real dof -> complex coefficient a2, y = (w/2)(a2 T1 + conj(a2) T2)
  double2 y;
  const double rt2 = 1.4142135623730951;
  if (b.m == 0) {
    y = T1;  // (1/2)(T1 + T2) with T1 = T2 when m2 = 0
  } else if (b.part == 0) {
    y = make_double2((T1.x + T2.x) / rt2, (T1.y + T2.y) / rt2);
  } else {
    // a2 = i / sqrt2: (i T1 - i T2) / sqrt2
    y = make_double2(-(T1.y - T2.y) / rt2, (T1.x - T2.x) / rt2);
  }
  double v;
  if (a.m == 0) v = y.x;
  else v = rt2 * (a.part == 0 ? y.x : y.y);
  v *= bl[a.l] * bl[b.l];
  if (r == c) v += dl[a.l];
  A[(int64_t)r * nd + c] = v;
}

// right-looking Cholesky, one column per pair of launches; fail[0] records
// 1 + the first failing pivot index, fail_val its value
__global__ void chol_col_kernel(double* A, int n, int j, int* fail, double* fail_val) {
  __shared__ double d;
  if (threadIdx.x == 0) {
    const double v = A[(int64_t)j * n + j];
    if ((!(v > 0.0) || !isfinite(v)) && atomicCAS(fail, 0, j + 1) == 0) *fail_val = v;
    d = sqrt(fmax(v, 1e-300));
    A[(int64_t)j * n + j] = d;
  }
  __syncthreads();
  for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[(int64_t)i * n + j] /= d;
}
__global__ void chol_update_kernel(double* A, int n, int j) {
  const int i = j + 1 + blockIdx.y;
  const double aij = A[(int64_t)i * n + j];
  for (int k = j + 1 + blockIdx.x * blockDim.x + threadIdx.x; k <= i; k += gridDim.x * blockDim.x)
    A[(int64_t)i * n + k] -= aij * A[(int64_t)k * n + j];
}
// Linv column c by forward substitution (lower L in A, row-major)
__global__ void tri_inv_kernel(const double* A, int n, double* Li) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int i = 0; i < n; ++i) {
    double s = (i == c) ? 1.0 : 0.0;
    if (i > c)
      for (int k = c; k < i; ++k) s -= A[(int64_t)i * n + k] * Li[(int64_t)k * n + c];
    Li[(int64_t)i * n + c] = (i >= c) ? s / A[(int64_t)i * n + i] : 0.0;
  }
}
// Ainv = Li^T Li  (16x16 tiles)
__global__ void gram_kernel(const double* Li, int n, double* out) {
  __shared__ double ta[16][17], tb[16][17];
  const int r = blockIdx.y * 16 + threadIdx.y, c = blockIdx.x * 16 + threadIdx.x;
  double acc = 0.0;
  for (int k0 = 0; k0 < n; k0 += 16) {
    const int ka = k0 + threadIdx.x, kb = k0 + threadIdx.y;
    ta[threadIdx.y][threadIdx.x] = (r < n && ka < n) ? Li[(int64_t)ka * n + r] : 0.0;
    tb[threadIdx.y][threadIdx.x] = (c < n && kb < n) ? Li[(int64_t)kb * n + c] : 0.0;
    __syncthreads();
    for (int k = 0; k < 16; ++k) acc = fma(ta[threadIdx.y][k], tb[k][threadIdx.x], acc);
    __syncthreads();
  }
  if (r < n && c < n) out[(int64_t)r * n + c] = acc;
}

// bottom solve: x = Ainv b in the real basis; b, x complex in the lmax_d layout
template <typename T>
__global__ void bottom_gemv_kernel(const double* Ainv, const DofMap* dofs, int nd, int Ld,
                                   const typename Tr<T>::C* b, typename Tr<T>::C* x) {
  extern __shared__ double ub[];
  const double rt2 = 1.4142135623730951;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) {
    const DofMap d = dofs[i];
    const typename Tr<T>::C v = b[lm_off(Ld, d.m) + (d.l - d.m)];
    ub[i] = (d.m == 0) ? (double)v.x : rt2 * (double)(d.part == 0 ? v.x : v.y);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int row = blockIdx.x * nw + warp; row < nd; row += gridDim.x * nw) {
    double s = 0.0;
    for (int k = lane; k < nd; k += 32) s = fma(Ainv[(int64_t)row * nd + k], ub[k], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const DofMap d = dofs[row];
      typename Tr<T>::C* dst = x + lm_off(Ld, d.m) + (d.l - d.m);
      if (d.m == 0) {
        dst->x = (T)s;
        dst->y = (T)0;
      } else if (d.part == 0) {
        dst->x = (T)(s / rt2);
      } else {
        dst->y = (T)(s / rt2);
      }
    }
  }
}

static int ring_dft(cr_plan* P, int dmax, double2** X) {
  const Grid& g = P->obs;
  CR_CUDA(cudaMalloc(X, (size_t)g.nring * (dmax + 1) * sizeof(double2)));
  ring_dft_kernel<<<g.nring, 128, 0, P->stream>>>(g.d_fft, g.d_tab, P->d_ninv, dmax, *X);
  CR_CHECK_LAUNCH("ring_dft_kernel");
  return CR_OK;
}

static int ptable(cr_plan* P, int Ld, double** out) {
  const Grid& g = P->obs;
  CR_CUDA(cudaMalloc(out, (size_t)g.npairs * n_lm(Ld) * sizeof(double)));
  dim3 grid(Ld + 1, (g.npairs + 127) / 128);
  ptab_kernel<<<grid, 128, 0, P->stream>>>(g.d_z, g.d_seed, g.d_lev, g.npairs, P->d_c, P->d_s, P->Lcoef, Ld,
                                           g.npairs, *out);
  CR_CHECK_LAUNCH("ptab_kernel");
  return CR_OK;
}

// inv_diag_hp[lm] = (1 - f1_l) / (1/C_l + b_l^2 diag_lm), 0 at inactive l
__global__ void top_inv_kernel(const double* diag, const double* sinv, const double* bl, const double* hp, int L,
                               double* out) {
  const int m = blockIdx.x;
  const int64_t o = lm_off(L, m);
  for (int l = m + threadIdx.x; l <= L; l += blockDim.x) {
    const double d = sinv[l] + bl[l] * bl[l] * diag[o + l - m];
    out[o + l - m] = (sinv[l] > 0.0 && d > 0.0) ? hp[l] / d : 0.0;
  }
}

// X_k(0) = sum_j n_kj per ring
__global__ void ring_sum_kernel(const RingFFT* fft, const double* ninv, double* out) {
  const RingFFT f = fft[blockIdx.x];
  double s = 0.0;
  for (int j = threadIdx.x; j < f.n; j += blockDim.x) s += ninv[f.off + j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    out[blockIdx.x] = t;
  }
}

__global__ void top_inv_from_complex_kernel(const double2* diag, const double* sinv, const double* bl,
                                            const double* hp, int L, double* out) {
  const int m = blockIdx.x;
  const int64_t o = lm_off(L, m);
  for (int l = m + threadIdx.x; l <= L; l += blockDim.x) {
    const double d = sinv[l] + bl[l] * bl[l] * diag[o + l - m].x;
    out[o + l - m] = (sinv[l] > 0.0 && d > 0.0) ? hp[l] / d : 0.0;
  }
}

// out_lm = hp_l / diag(A)_lm (0 where C_l = 0), diag(A) = 1/C_l + b_l^2 times
// the Delta m = 0 ring-formula diagonal of Y^T N^-1 Y; out is device [n_lm].
int inv_diag_A(cr_plan* P, const std::vector<double>& hpl, double* out) {
  const int L = P->lmax;
  const int64_t nlm = n_lm(L);
  double *rs = nullptr, *hp = nullptr;
  double2* diag = nullptr;
  CR_CUDA(cudaMalloc(&rs, P->obs.nring * sizeof(double)));
  { ring_sum_kernel<<<P->obs.nring, 256, 0, P->stream>>>(P->obs.d_fft, P->d_ninv, rs); count_launch(); }
  CR_CHECK_LAUNCH("ring_sum_kernel");
  CR_CUDA(cudaMalloc(&diag, nlm * sizeof(double2)));
  int rc = launch_leg_diag(P, rs, diag);
  if (!rc) {
    CR_CUDA(cudaMalloc(&hp, (L + 1) * sizeof(double)));
    CR_CUDA(cudaMemcpy(hp, hpl.data(), (L + 1) * sizeof(double), cudaMemcpyHostToDevice));
    { top_inv_from_complex_kernel<<<L + 1, 128, 0, P->stream>>>(diag, P->d_sinv, P->d_bl, hp, L, out); count_launch(); }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "top_inv_kernel");
  }
  void* ptrs[] = {rs, hp, diag};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  return rc;
}

int build_top_diag(cr_plan* P, Hierarchy& Hh, const std::vector<double>& f1) {
  const int L = P->lmax;
  const int64_t nlm = n_lm(L);
  std::vector<double> h(L + 1);
  for (int l = 0; l <= L; ++l) h[l] = 1.0 - (l < (int)f1.size() ? f1[l] : 0.0);
  double* out = nullptr;
  CR_CUDA(cudaMalloc(&out, nlm * sizeof(double)));
  int rc = inv_diag_A(P, h, out);
  if (!rc) {
    std::vector<double> hv(nlm);
    cudaError_t e = cudaMemcpy(hv.data(), out, nlm * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = cuda_fail(e, "top diag copy");
    else rc = Hh.inv_diag_hp.assign(hv);
  }
  cudaFree(out);
  return rc;
}

// Real degrees of freedom of the bottom level, in the order of the dense
// matrix: every active (C_l > 0) l with m = 0, then for m = 1..Ld and
// l = m..Ld the real and imaginary parts.  Returned as (l, m, part) triples.
std::vector<int32_t> bottom_dof_map(const cr_plan* P, int Ld) {
  std::vector<int32_t> d;
  for (int l = 0; l <= Ld; ++l)
    if (P->h_cl[l] > 0) d.insert(d.end(), {l, 0, 0});
  for (int m = 1; m <= Ld; ++m)
    for (int l = m; l <= Ld; ++l)
      if (P->h_cl[l] > 0) d.insert(d.end(), {l, m, 0, l, m, 1});
  return d;
}

int build_bottom(cr_plan* P, Hierarchy& Hh) {
  const int Ld = Hh.ld;
  const std::vector<int32_t> flat = bottom_dof_map(P, Ld);
  std::vector<DofMap> dofs(flat.size() / 3);
  for (size_t i = 0; i < dofs.size(); ++i) dofs[i] = {flat[3 * i], flat[3 * i + 1], flat[3 * i + 2]};
  const int nd = (int)dofs.size();
  Hh.nd = nd;
  if (nd == 0) return CR_OK;
  std::vector<double> bd(Ld + 1), dd(Ld + 1);
  for (int l = 0; l <= Ld; ++l) {
    const double f = Hh.fb[l];
    bd[l] = P->h_cl[l] > 0 ? f * P->h_bl[l] : 0.0;
    dd[l] = P->h_cl[l] > 0 ? f * f / P->h_cl[l] : 0.0;
  }
  double2* X = nullptr;
  double *pt = nullptr, *A = nullptr, *Li = nullptr, *dbl = nullptr, *ddl = nullptr;
  DofMap* d_dofs = nullptr;
  int* d_fail = nullptr;
  double* d_fail_val = nullptr;
  if (2 * Ld + 1 > 128) return fail(CR_EINVAL, "bottom level: lmax_dense must be <= 63");
  int rc = ring_dft(P, 2 * Ld, &X);
  if (!rc) rc = ptable(P, Ld, &pt);
  if (!rc) {
    CR_CUDA(cudaMalloc(&d_dofs, nd * sizeof(DofMap)));
    CR_CUDA(cudaMemcpy(d_dofs, dofs.data(), nd * sizeof(DofMap), cudaMemcpyHostToDevice));
    CR_CUDA(cudaMalloc(&dbl, (Ld + 1) * sizeof(double)));
    CR_CUDA(cudaMalloc(&ddl, (Ld + 1) * sizeof(double)));
    CR_CUDA(cudaMemcpy(dbl, bd.data(), (Ld + 1) * sizeof(double), cudaMemcpyHostToDevice));
    CR_CUDA(cudaMemcpy(ddl, dd.data(), (Ld + 1) * sizeof(double), cudaMemcpyHostToDevice));
    CR_CUDA(cudaMalloc(&A, (size_t)nd * nd * sizeof(double)));
    CR_CUDA(cudaMalloc(&Li, (size_t)nd * nd * sizeof(double)));
    CR_CUDA(cudaMalloc(&d_fail, sizeof(int)));
    CR_CUDA(cudaMalloc(&d_fail_val, sizeof(double)));
    CR_CUDA(cudaMemset(d_fail, 0, sizeof(int)));
    const int64_t ne = (int64_t)nd * nd;
    assemble_dense_kernel<<<(int)((ne + 127) / 128), 128, 0, P->stream>>>(pt, X, 2 * Ld, P->obs.npairs,
                                                                          P->obs.nring, Ld, d_dofs, nd, dbl, ddl, A);
    CR_CHECK_LAUNCH("assemble_dense_kernel");
    if (Hh.nd_alloc != nd) {
      // a changed set of active l: new bottom arrays
      void* old[] = {Hh.d_Abottom, Hh.d_Ainv, Hh.d_dof_lm};
      for (void* q : old)
        if (q) cudaFree(q);
      Hh.d_Abottom = Hh.d_Ainv = nullptr;
      Hh.d_dof_lm = nullptr;
      CR_CUDA(cudaMalloc(&Hh.d_Abottom, (size_t)nd * nd * sizeof(double)));
      CR_CUDA(cudaMalloc(&Hh.d_Ainv, (size_t)nd * nd * sizeof(double)));
      CR_CUDA(cudaMalloc(&Hh.d_dof_lm, nd * sizeof(DofMap)));
      Hh.nd_alloc = nd;
    }
    CR_CUDA(cudaMemcpyAsync(Hh.d_Abottom, A, (size_t)nd * nd * sizeof(double), cudaMemcpyDeviceToDevice, P->stream));
    for (int j = 0; j < nd; ++j) {
      chol_col_kernel<<<1, 256, 0, P->stream>>>(A, nd, j, d_fail, d_fail_val);
      if (j + 1 < nd) {
        dim3 g((nd - j + 255) / 256, nd - j - 1);
        chol_update_kernel<<<g, 256, 0, P->stream>>>(A, nd, j);
      }
    }
    CR_CHECK_LAUNCH("chol kernels");
    tri_inv_kernel<<<(nd + 63) / 64, 64, 0, P->stream>>>(A, nd, Li);
    CR_CHECK_LAUNCH("tri_inv_kernel");
    dim3 gg((nd + 15) / 16, (nd + 15) / 16), bb(16, 16);
    gram_kernel<<<gg, bb, 0, P->stream>>>(Li, nd, Hh.d_Ainv);
    CR_CHECK_LAUNCH("gram_kernel");
    int failed = 0;
    double fval = 0.0;
    CR_CUDA(cudaMemcpyAsync(&failed, d_fail, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
    CR_CUDA(cudaMemcpyAsync(&fval, d_fail_val, sizeof(double), cudaMemcpyDeviceToHost, P->stream));
    CR_CUDA(cudaStreamSynchronize(P->stream));
    if (failed) {
      const DofMap& dm = dofs[failed - 1];
      rc = fail(CR_EICC, "bottom level: dense Cholesky pivot " + std::to_string(failed - 1) + " of " +
                             std::to_string(nd) + " (l=" + std::to_string(dm.l) + " m=" + std::to_string(dm.m) +
                             ") is " + std::to_string(fval));
    }
    CR_CUDA(cudaMemcpy(Hh.d_dof_lm, dofs.data(), nd * sizeof(DofMap), cudaMemcpyHostToDevice));
  }
  void* ptrs[] = {X, pt, A, Li, dbl, ddl, d_dofs, d_fail, d_fail_val};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  return rc;
}

// bottom-level arrays from host copies (checkpoint load)
int bottom_upload(cr_plan* P, Hierarchy& Hh, int nd, const double* a, const double* ainv, const int32_t* dofs) {
  static_assert(sizeof(DofMap) == 3 * sizeof(int32_t), "dof map layout");
  CR_CUDA(cudaStreamSynchronize(P->stream));
  if (Hh.nd_alloc != nd) {
    void* old[] = {Hh.d_Abottom, Hh.d_Ainv, Hh.d_dof_lm};
    for (void* q : old)
      if (q) cudaFree(q);
    Hh.d_Abottom = Hh.d_Ainv = nullptr;
    Hh.d_dof_lm = nullptr;
    CR_CUDA(cudaMalloc(&Hh.d_Abottom, (size_t)nd * nd * sizeof(double)));
    CR_CUDA(cudaMalloc(&Hh.d_Ainv, (size_t)nd * nd * sizeof(double)));
    CR_CUDA(cudaMalloc(&Hh.d_dof_lm, nd * sizeof(DofMap)));
    Hh.nd_alloc = nd;
  }
  CR_CUDA(cudaMemcpy(Hh.d_Abottom, a, (size_t)nd * nd * sizeof(double), cudaMemcpyHostToDevice));
  CR_CUDA(cudaMemcpy(Hh.d_Ainv, ainv, (size_t)nd * nd * sizeof(double), cudaMemcpyHostToDevice));
  CR_CUDA(cudaMemcpy(Hh.d_dof_lm, dofs, nd * sizeof(DofMap), cudaMemcpyHostToDevice));
  return CR_OK;
}

int bottom_matrix(cr_plan* P, double* host, int* nd) {
  Hierarchy& Hh = *P->hier;
  if (nd) *nd = Hh.nd;
  if (host && Hh.nd > 0)
    CR_CUDA(cudaMemcpy(host, Hh.d_Abottom, (size_t)Hh.nd * Hh.nd * sizeof(double), cudaMemcpyDeviceToHost));
  return CR_OK;
}

template <typename T>
int bottom_solve(cr_plan* P, Hierarchy& Hh, const void* b, void* x) {
  const int Ld = Hh.ld;
  CR_CUDA(cudaMemsetAsync(x, 0, n_lm(Ld) * sizeof(typename Tr<T>::C), P->stream));
  if (Hh.nd == 0) return CR_OK;
  const int blocks = std::min(152, (Hh.nd + 7) / 8);
  { bottom_gemv_kernel<T><<<blocks, 256, Hh.nd * sizeof(double), P->stream>>>(
      Hh.d_Ainv, reinterpret_cast<const DofMap*>(Hh.d_dof_lm), Hh.nd, Ld, (const typename Tr<T>::C*)b,
      (typename Tr<T>::C*)x); count_launch(); }
  CR_CHECK_LAUNCH("bottom_gemv_kernel");
  return CR_OK;
}
template int bottom_solve<double>(cr_plan*, Hierarchy&, const void*, void*);
template int bottom_solve<float>(cr_plan*, Hierarchy&, const void*, void*);

}  // namespace cr
