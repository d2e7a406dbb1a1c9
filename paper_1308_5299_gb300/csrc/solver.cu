// Multi-level hierarchy construction, CR-Cycle and CR-Solve (Section 3.2,
// Fig. code:mg), and the C ABI entry points of the multi-level solver.
//
// CR-Cycle(h, x, b) on a spherical-harmonic level h:
//   pre-smoothing   x += S_h(b - A_h x)
//   restriction     r_H = I_h^H (b - A_h x)
//   recursion       c_H = 0; repeat n_rec(h): c_H = CR-Cycle(H, c_H, r_H)
//   correction      x += (I_h^H)^T c_H
//   post-smoothing  x += S_h(b - A_h x)
// with S_0 the top-level diagonal smoother (1 - f^1) diag(A)^-1, S_h for
// pixel levels Y_h^T M_h Y_h, and the bottom level solved densely.  A zero
// starting vector saves the first residual (b itself).  Residuals are fused
// into the adjoint-synthesis epilogue (r = b - A_h x) and the smoothing
// correction into the adjoint epilogue of the level grid (x += ...).
//
// CR-Solve repeats cycles until r^T S^-1 r < eps b^T S^-1 b.  In the mixed
// mode every cycle runs in FP32 on the FP64 residual (iterative refinement):
//   r = b - A x (FP64),  c = CR-Cycle_FP32(0, r),  x += c.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "hier.h"
#include "kernels.h"
#include "levels.h"

namespace cr {

static int lmax_of(const cr_plan* P, int h) {
  const Hierarchy& H = *P->hier;
  if (h == 0) return P->lmax;
  if (h <= H.H) return H.pix[h - 1].lmax_h;
  return H.ld;
}

// per-level operator arrays: B_h and D_h (l-indexed, 0 where C_l = 0), the
// restriction ratio into the next level, and the active mask
struct LevelOps {
  LArr b, d, ratio, act;
};
struct HierOps {
  std::vector<LevelOps> ops;  // [H + 2]
};

static HierOps& ops_of(cr_plan* P) {
  return *reinterpret_cast<HierOps*>(P->hier->ops_store);
}

// Grid and pixel weights of level h's inverse-noise term: the level's
// Gauss-Legendre grid when it has one, else the observation grid.
template <typename T>
static const Grid& noise_grid(cr_plan* P, int h, const T** pix) {
  const Hierarchy& H = *P->hier;
  if (h >= 1 && h <= H.H && H.pix[h - 1].gl) {
    const PixLevel& lev = H.pix[h - 1];
    if constexpr (sizeof(T) == 8) *pix = lev.d_nt;
    else *pix = lev.d_nt32;
    return *lev.gl;
  }
  if constexpr (sizeof(T) == 8) *pix = P->d_ninv;
  else *pix = P->d_ninv32;
  return P->obs;
}

template <typename T>
static int residual(cr_plan* P, int h, const void* x, const void* b, void* r) {
  LevelOps& o = ops_of(P).ops[h];
  const int L = lmax_of(P, h);
  const T* pix = nullptr;
  const Grid& g = noise_grid<T>(P, h, &pix);
  return do_sandwich<T>(P, g, L, x, r, o.b.get<T>(), pix, o.b.get<T>(), o.d.get<T>(), nullptr, b);
}

template <typename T>
static int smooth_add(cr_plan* P, int h, void* x, const void* r) {
  Hierarchy& H = *P->hier;
  const int L = lmax_of(P, h);
  if (h == 0) {
    TimerScope ts(P->timing, P->stream, "top_smoother");
    return launch_diag_axpy<T>(x, r, H.inv_diag_hp.get<T>(), n_lm(L), P->stream);
  }
  PixLevel& lev = H.pix[h - 1];
  T* m1 = reinterpret_cast<T*>(H.map_work);
  T* m2 = reinterpret_cast<T*>(H.map_work2);
  int rc = do_synth<T>(P, *lev.grid, L, r, m1, nullptr);
  if (rc) return rc;
  {
    // algorithmic bytes: every factor block read once forward, once backward
    // (Schwarz: every tile's inverse block once)
    const double bytes = H.smoother_kind == 1 ? lev.pat.ntile * 64.0 * 64.0 * sizeof(float)
                                              : 2.0 * lev.pat.nblocks * 64.0 * 64.0 * sizeof(float);
    TimerScope ts(P->timing, P->stream, "pixel_smoother", bytes);
    TimerScope tl(P->timing, P->stream, "pixel_smoother.n" + std::to_string(lev.nside_h), bytes);
    rc = apply_smoother<T>(P, lev, m1, m2);
  }
  if (rc) return rc;
  return do_adjoint<T>(P, *lev.grid, L, m2, x, ops_of(P).ops[h].act.get<T>(), nullptr, nullptr, 1);
}

template <typename T>
static int cycle(cr_plan* P, int h, void* x, const void* b, bool x_zero, const void* r_in) {
  Hierarchy& H = *P->hier;
  using C = typename Tr<T>::C;
  if (h == H.H + 1) {
    TimerScope ts(P->timing, P->stream, "bottom_solve");
    return bottom_solve<T>(P, H, b, x);
  }
  const int L = lmax_of(P, h), LH = lmax_of(P, h + 1);
  void* r = H.work[h].r;
  int rc;
  if (x_zero) {
    CR_CUDA(cudaMemsetAsync(x, 0, n_lm(L) * sizeof(C), P->stream));
    if ((rc = smooth_add<T>(P, h, x, b))) return rc;
  } else if (r_in) {
    if ((rc = smooth_add<T>(P, h, x, r_in))) return rc;
  } else {
    if ((rc = residual<T>(P, h, x, b, r))) return rc;
    if ((rc = smooth_add<T>(P, h, x, r))) return rc;
  }
  if ((rc = residual<T>(P, h, x, b, r))) return rc;
  LevelOps& o = ops_of(P).ops[h];
  if ((rc = launch_restrict<T>(r, L, H.work[h + 1].b, LH, o.ratio.get<T>(), P->stream))) return rc;
  const int nrec = (h == 0) ? H.n_rec_top : H.pix[h - 1].n_rec;
  for (int i = 0; i < nrec; ++i)
    if ((rc = cycle<T>(P, h + 1, H.work[h + 1].x, H.work[h + 1].b, i == 0, nullptr))) return rc;
  if ((rc = launch_prolong_add<T>(x, L, H.work[h + 1].x, LH, o.ratio.get<T>(), P->stream))) return rc;
  if ((rc = residual<T>(P, h, x, b, r))) return rc;
  return smooth_add<T>(P, h, x, r);
}

// ---------------------------------------------------------------------------
// Batched CR-Cycle: the FP32 cycle above for up to 16 right-hand sides at
// once, every Legendre stage (level operators A_h on their noise grids, the
// pixel levels' Y_h and Y_h^T around the smoother) as one tensor-core
// contraction over the right-hand sides (BF16 operands, FP32 accumulation);
// ring FFTs, pixel smoothers, restriction, prolongation and the bottom solve
// run per right-hand side.  Level h keeps its vectors in tcw[h], contiguous
// [16][n_lm(lmax_h)].

static int ensure_tc_work(cr_plan* P) {
  Hierarchy& H = *P->hier;
  int rc = ensure_smoother_batch(P);
  if (rc) return rc;
  if (!P->d_tc_r64) CR_CUDA(cudaMalloc(&P->d_tc_r64, (size_t)16 * n_lm(P->lmax) * sizeof(double2)));
  if ((int)H.tcw.size() == H.H + 2) return CR_OK;
  H.tcw.assign(H.H + 2, Hierarchy::TcWork());
  for (int h = 0; h <= H.H + 1; ++h) {
    const size_t bytes = (size_t)16 * n_lm(lmax_of(P, h)) * sizeof(float2);
    CR_CUDA(cudaMalloc(&H.tcw[h].x, bytes));
    CR_CUDA(cudaMalloc(&H.tcw[h].b, bytes));
    CR_CUDA(cudaMalloc(&H.tcw[h].r, bytes));
  }
  return CR_OK;
}

// R = B - A_h X for nr right-hand sides (with P->tc_top_f32 the top level's
// residuals run per right-hand side on the FP32 CUDA-core kernels)
static int residual_tc(cr_plan* P, int h, int nr, const float2* X, const float2* B, float2* R) {
  LevelOps& o = ops_of(P).ops[h];
  const int L = lmax_of(P, h);
  if (h == 0 && P->tc_top_f32) {
    const int64_t nlm = n_lm(L);
    for (int r = 0; r < nr; ++r) {
      int rc = residual<float>(P, 0, X + r * nlm, B + r * nlm, R + r * nlm);
      if (rc) return rc;
    }
    return CR_OK;
  }
  const float* pix = nullptr;
  const Grid& g = noise_grid<float>(P, h, &pix);
  int rc = tc_begin(P, g, L, true, false);
  if (rc) return rc;
  TcTail t;
  t.dl_out = o.b.get<float>();
  t.dadd = o.d.get<float>();
  t.xadd = X;
  t.bsub = B;
  t.out = R;
  return tc_sandwich(P, g, L, nr, X, o.b.get<float>(), pix, t);
}

// X += S_h R for nr right-hand sides
static int smooth_add_tc(cr_plan* P, int h, int nr, float2* X, const float2* R) {
  Hierarchy& H = *P->hier;
  const int L = lmax_of(P, h);
  const int64_t nlm = n_lm(L);
  if (h == 0) {
    TimerScope ts(P->timing, P->stream, "top_smoother");
    for (int r = 0; r < nr; ++r) {
      int rc = launch_diag_axpy<float>(X + r * nlm, R + r * nlm, H.inv_diag_hp.get<float>(), nlm, P->stream);
      if (rc) return rc;
    }
    return CR_OK;
  }
  PixLevel& lev = H.pix[h - 1];
  const Grid& g = *lev.grid;
  float* m1 = reinterpret_cast<float*>(H.map_work);
  float* m2 = reinterpret_cast<float*>(H.map_work2);
  int rc = tc_begin(P, g, L, true, false);
  if (!rc) rc = tc_synth_stage(P, g, L, R, nr, nullptr);
  if (!rc && H.smoother_kind == 0 && nr > 1) {
    // every right-hand side's map, then the sweeps for all of them at once
    const int64_t np = g.npix;
    for (int r = 0; r < nr && !rc; ++r) rc = tc_ring(P, g, L, r, 0, nullptr, H.d_mr_m1 + r * np);
    if (!rc) {
      const double bytes = 2.0 * lev.pat.nblocks * 64.0 * 64.0 * sizeof(float);
      TimerScope ts(P->timing, P->stream, "pixel_smoother", bytes);
      rc = apply_smoother_mr<float>(P, lev, nr, H.d_mr_m1, H.d_mr_m2, np);
    }
    for (int r = 0; r < nr && !rc; ++r) rc = tc_ring(P, g, L, r, 1, H.d_mr_m2 + r * np, nullptr);
  }
  for (int r = 0; r < nr && !rc && !(H.smoother_kind == 0 && nr > 1); ++r) {
    if ((rc = tc_ring(P, g, L, r, 0, nullptr, m1))) break;
    {
      const double bytes = H.smoother_kind == 1 ? lev.pat.ntile * 64.0 * 64.0 * sizeof(float)
                                                : 2.0 * lev.pat.nblocks * 64.0 * 64.0 * sizeof(float);
      TimerScope ts(P->timing, P->stream, "pixel_smoother", bytes);
      if ((rc = apply_smoother<float>(P, lev, m1, m2))) break;
    }
    rc = tc_ring(P, g, L, r, 1, m2, nullptr);
  }
  if (rc) return rc;
  TcTail t;
  t.dl_out = ops_of(P).ops[h].act.get<float>();
  t.accumulate = 1;
  t.out = X;
  return tc_adjoint_tail(P, g, L, nr, t);
}

static int cycle_tc(cr_plan* P, int h, int nr, bool x_zero) {
  Hierarchy& H = *P->hier;
  Hierarchy::TcWork& w = H.tcw[h];
  const int L = lmax_of(P, h);
  const int64_t nlm = n_lm(L);
  int rc;
  if (h == H.H + 1) {
    TimerScope ts(P->timing, P->stream, "bottom_solve");
    for (int r = 0; r < nr; ++r)
      if ((rc = bottom_solve<float>(P, H, w.b + r * nlm, w.x + r * nlm))) return rc;
    return CR_OK;
  }
  const int LH = lmax_of(P, h + 1);
  const int64_t nlmH = n_lm(LH);
  Hierarchy::TcWork& wH = H.tcw[h + 1];
  if (x_zero) {
    CR_CUDA(cudaMemsetAsync(w.x, 0, nr * nlm * sizeof(float2), P->stream));
    if ((rc = smooth_add_tc(P, h, nr, w.x, w.b))) return rc;
  } else {
    if ((rc = residual_tc(P, h, nr, w.x, w.b, w.r))) return rc;
    if ((rc = smooth_add_tc(P, h, nr, w.x, w.r))) return rc;
  }
  if ((rc = residual_tc(P, h, nr, w.x, w.b, w.r))) return rc;
  LevelOps& o = ops_of(P).ops[h];
  for (int r = 0; r < nr; ++r)
    if ((rc = launch_restrict<float>(w.r + r * nlm, L, wH.b + r * nlmH, LH, o.ratio.get<float>(), P->stream)))
      return rc;
  const int nrec = (h == 0) ? H.n_rec_top : H.pix[h - 1].n_rec;
  for (int i = 0; i < nrec; ++i)
    if ((rc = cycle_tc(P, h + 1, nr, i == 0))) return rc;
  for (int r = 0; r < nr; ++r)
    if ((rc = launch_prolong_add<float>(w.x + r * nlm, L, wH.x + r * nlmH, LH, o.ratio.get<float>(), P->stream)))
      return rc;
  if ((rc = residual_tc(P, h, nr, w.x, w.b, w.r))) return rc;
  return smooth_add_tc(P, h, nr, w.x, w.r);
}

template <typename T>
int level_apply(cr_plan* P, int h, const void* x, void* y);

// Largest eigenvalue of S_h A_h (self-adjoint in the A_h inner product) by
// power iteration in FP32, Rayleigh quotient <S A v, A v> / <v, A v>.
static int smoother_lambda_max(cr_plan* P, int h, int iters, double* lam) {
  Hierarchy& H = *P->hier;
  const int L = lmax_of(P, h);
  void* v = H.work[h].x;
  void* av = H.work[h].b;
  void* w = H.work[h].r;
  int rc = launch_fill_random(v, L, 0x9e3779b9u + 17u * h, P->stream);
  if (rc) return rc;
  double num = 0.0, den = 1.0, nv = 0.0;
  *lam = 0.0;
  for (int it = 0; it < iters; ++it) {
    if ((rc = level_apply<float>(P, h, v, av))) return rc;
    CR_CUDA(cudaMemsetAsync(w, 0, n_lm(L) * sizeof(float2), P->stream));
    if ((rc = smooth_add<float>(P, h, w, av))) return rc;
    if ((rc = launch_dot<float>(w, av, nullptr, L, H.d_dot, P->d_dotpart, P->stream))) return rc;
    if ((rc = launch_dot<float>(v, av, nullptr, L, H.d_dot + 1, P->d_dotpart, P->stream))) return rc;
    if ((rc = launch_dot<float>(w, w, nullptr, L, H.d_dot + 2, P->d_dotpart, P->stream))) return rc;
    double d3[3];
    CR_CUDA(cudaMemcpyAsync(d3, H.d_dot, 3 * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
    CR_CUDA(cudaStreamSynchronize(P->stream));
    num = d3[0];
    den = d3[1];
    nv = d3[2];
    if (!(den > 0.0) || !(nv > 0.0) || !std::isfinite(num)) break;
    *lam = num / den;
    // v = w / |w|
    if ((rc = launch_scale_copy(w, v, (float)(1.0 / std::sqrt(nv)), n_lm(L), P->stream))) return rc;
  }
  return CR_OK;
}

static int alloc_work(Hierarchy& H, int h, int L) {
  const size_t bytes = n_lm(L) * sizeof(double2);
  CR_CUDA(cudaMalloc(&H.work[h].x, bytes));
  CR_CUDA(cudaMalloc(&H.work[h].b, bytes));
  CR_CUDA(cudaMalloc(&H.work[h].r, bytes));
  CR_CUDA(cudaMemset(H.work[h].x, 0, bytes));
  return CR_OK;
}

__global__ void gl_weight_kernel(double* nt, float* nt32, const double* wr, int nphi, int64_t npix) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = nt[i] * wr[i / nphi];
    nt[i] = v;
    nt32[i] = (float)v;
  }
}

// Section 3.4 (Eqs. Ni-rewrite, Xi): for band limit Lh the operator
// Y_obs^T N^-1 Y_obs sees the inverse-noise map n only through
// xi_LM = (Y_obs^T n)_LM, L <= 2 Lh (the product Y*_lm Y_l'm' expands into
// Y_LM with L <= l + l').  On a Gauss-Legendre grid exact for degree 4 Lh
// (2 Lh + 1 rings, nphi >= 4 Lh + 1) the same operator is
// Y_gl^T diag(w_j nt(n_j)) Y_gl with nt = sum_{L<=2Lh} xi_LM Y_LM.
static int build_gl_level(cr_plan* P, PixLevel& lev) {
  const int Lh = lev.lmax_h, L2 = 2 * Lh;
  int nphi = 2;
  while (nphi < 2 * L2 + 1) nphi <<= 1;
  lev.gl = new Grid();
  std::vector<double> w;
  gl_rings(*lev.gl, L2 + 1, nphi, &w);
  int rc = grid_upload(*lev.gl, L2, P->stream);
  if (!rc) rc = build_start_tables(P, *lev.gl);
  if (!rc) rc = ensure_workspace(P, *lev.gl, L2);
  if (!rc) rc = ensure_workspace(P, P->obs, L2);
  if (rc) return rc;
  const int64_t npix = lev.gl->npix;
  void* xi = nullptr;
  double* d_wr = nullptr;
  CR_CUDA(cudaMalloc(&xi, n_lm(L2) * sizeof(double2)));
  CR_CUDA(cudaMalloc(&lev.d_nt, npix * sizeof(double)));
  CR_CUDA(cudaMalloc(&lev.d_nt32, npix * sizeof(float)));
  CR_CUDA(cudaMalloc(&d_wr, w.size() * sizeof(double)));
  for (auto& v : w) v *= 2.0 * M_PI / nphi;
  CR_CUDA(cudaMemcpy(d_wr, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
  rc = do_adjoint<double>(P, P->obs, L2, P->d_ninv, xi, nullptr, nullptr, nullptr, 0);
  if (!rc) rc = do_synth<double>(P, *lev.gl, L2, xi, lev.d_nt, nullptr);
  if (!rc) {
    gl_weight_kernel<<<1024, 256, 0, P->stream>>>(lev.d_nt, lev.d_nt32, d_wr, nphi, npix);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "gl_weight_kernel");
  }
  cudaFree(xi);
  cudaFree(d_wr);
  return rc;
}

// per-level operator arrays B_h = f_h b_l, D_h = f_h^2 / C_l and the active
// mask (0 where C_l = 0) of every level (Section 3.2, Eq. A_h)
static int upload_level_arrays(cr_plan* P) {
  Hierarchy& H = *P->hier;
  HierOps& hops = ops_of(P);
  auto one = [&](int h, const std::vector<double>& f, int Lh) -> int {
    std::vector<double> b(Lh + 1), d(Lh + 1), act(Lh + 1);
    for (int l = 0; l <= Lh; ++l) {
      const bool a = P->h_cl[l] > 0;
      b[l] = a ? f[l] * P->h_bl[l] : 0.0;
      d[l] = a ? f[l] * f[l] / P->h_cl[l] : 0.0;
      act[l] = a ? 1.0 : 0.0;
    }
    int r2 = hops.ops[h].b.assign(b);
    if (!r2) r2 = hops.ops[h].d.assign(d);
    if (!r2) r2 = hops.ops[h].act.assign(act);
    return r2;
  };
  std::vector<double> ftop(P->lmax + 1, 1.0);
  int rc = one(0, ftop, P->lmax);
  for (int i = 0; !rc && i < H.H; ++i) rc = one(i + 1, H.pix[i].fl, H.pix[i].lmax_h);
  if (!rc) rc = one(H.H + 1, H.fb, H.ld);
  return rc;
}

int build_hierarchy(cr_plan* P, const cr_params* p) {
  Hierarchy* Hp = new Hierarchy();
  P->hier = Hp;
  Hierarchy& H = *Hp;
  HierOps* hops = new HierOps();
  H.ops_store = hops;
  const int L = P->lmax;
  std::vector<LevelSpec> specs;
  int ld = -1;
  if (p->nlevels < 0) {
    default_levels(P->obs.nside, L, 8, specs, &ld);
  } else {
    for (int i = 0; i < p->nlevels; ++i) {
      const cr_level_spec& s = p->levels[i];
      LevelSpec ls;
      ls.nside_h = s.nside_h;
      ls.lmax_h = s.lmax_h;
      ls.n_rec = s.n_rec;
      ls.fl.assign(L + 1, 0.0);
      if (!s.fl) return fail(CR_EINVAL, "levels: every level needs a filter");
      for (int l = 0; l <= std::min(L, s.lmax_h); ++l) ls.fl[l] = s.fl[l];
      if (s.nside_h < 8 || (s.nside_h & (s.nside_h - 1)) || s.nside_h > P->obs.nside || s.lmax_h < 0 ||
          s.lmax_h > L || s.n_rec < 1)
        return fail(CR_EINVAL, "levels: bad nside_h / lmax_h / n_rec");
      specs.push_back(ls);
    }
    ld = p->lmax_dense >= 0 ? p->lmax_dense : (specs.empty() ? std::min(40, L) : std::min(40, specs.back().lmax_h / 2));
  }
  for (size_t i = 1; i < specs.size(); ++i)
    if (specs[i].lmax_h > specs[i - 1].lmax_h) return fail(CR_EINVAL, "levels: band limits must not increase");
  H.H = (int)specs.size();
  H.ld = std::max(0, std::min(ld, specs.empty() ? L : specs.back().lmax_h));
  H.n_rec_top = 1;
  H.pix.resize(H.H);
  H.work.resize(H.H + 2);
  hops->ops.resize(H.H + 2);
  if (p->smoother != 0 && p->smoother != 1) return fail(CR_EINVAL, "levels: smoother must be 0 (ICC) or 1 (Schwarz)");
  H.smoother_kind = p->smoother;
  if (p->smoother_sweep < 0 || p->smoother_sweep > 2) return fail(CR_EINVAL, "levels: smoother_sweep must be 0, 1 or 2");
  H.sweep_mode = p->smoother_sweep;
  const double rf = p->ridge_factor > 0 ? p->ridge_factor : 1.5;
  const int nbis = p->ridge_bisections > 0 ? p->ridge_bisections : 30;
  int rc = CR_OK;
  int64_t max_npix_h = 1;
  // Gauss-Legendre grids for the levels' inverse-noise term (gl_downgrade):
  // decided first, since they may need recurrence tables and observation-grid
  // seeds beyond lmax (up to 2 lmax_h)
  std::vector<int> use_gl(H.H, 0);
  {
    int Lneed = P->Lcoef;
    for (int i = 0; i < H.H; ++i) {
      const int Lh = specs[i].lmax_h;
      // automatic: where the GL grid has at most 3/5 of the observation
      // grid's rings (the Legendre stages cost in proportion to the rings;
      // the GL grid's power-of-two rings need no Bluestein FFTs)
      use_gl[i] = p->gl_downgrade > 0 || (p->gl_downgrade == 0 && 5 * (2 * Lh + 1) <= 3 * P->obs.nring);
      if (use_gl[i]) Lneed = std::max(Lneed, 2 * Lh);
    }
    const bool recoef = Lneed > P->Lcoef, reseed = Lneed > P->obs.Lseed;
    if (recoef && (rc = rebuild_coef(P, Lneed))) return rc;
    if (reseed && (rc = grid_reseed(P->obs, Lneed, P->stream))) return rc;
    if ((recoef || reseed) && (rc = build_start_tables(P, P->obs))) return rc;
  }
  std::vector<double> ftop(L + 1, 1.0);
  for (int i = 0; i < H.H; ++i) {
    PixLevel& lev = H.pix[i];
    lev.nside_h = specs[i].nside_h;
    lev.lmax_h = specs[i].lmax_h;
    lev.n_rec = specs[i].n_rec;
    lev.fl = specs[i].fl;
    lev.k = 8;
    lev.grid = new Grid();
    healpix_rings(*lev.grid, lev.nside_h);
    if ((rc = grid_upload(*lev.grid, lev.lmax_h, P->stream))) return rc;
    if ((rc = build_start_tables(P, *lev.grid))) return rc;
    if ((rc = ensure_workspace(P, *lev.grid, lev.lmax_h))) return rc;
    max_npix_h = std::max(max_npix_h, lev.grid->npix);
  }
  H.fb = specs.empty() ? ftop : specs.back().fl;
  for (int l = H.ld + 1; l <= L; ++l) H.fb[l] = 0.0;
  if ((rc = upload_level_arrays(P))) return rc;
  // restriction ratios f^{h+1} / f^h for l <= lmax_{h+1}
  for (int h = 0; h <= H.H; ++h) {
    const std::vector<double>& fh = (h == 0) ? ftop : H.pix[h - 1].fl;
    const std::vector<double>& fH = (h == H.H) ? H.fb : H.pix[h].fl;
    const int LH = (h == H.H) ? H.ld : H.pix[h].lmax_h;
    std::vector<double> ratio(LH + 1);
    for (int l = 0; l <= LH; ++l) ratio[l] = (fh[l] != 0.0) ? fH[l] / fh[l] : 0.0;
    if ((rc = hops->ops[h].ratio.upload(ratio))) return rc;
  }
  for (int i = 0; i < H.H; ++i)
    if (use_gl[i] && (rc = build_gl_level(P, H.pix[i]))) return rc;
  // work vectors
  if ((rc = alloc_work(H, 0, L))) return rc;
  for (int h = 1; h <= H.H; ++h)
    if ((rc = alloc_work(H, h, H.pix[h - 1].lmax_h))) return rc;
  if ((rc = alloc_work(H, H.H + 1, H.ld))) return rc;
  CR_CUDA(cudaMalloc(&H.map_work, max_npix_h * sizeof(double)));
  CR_CUDA(cudaMalloc(&H.map_work2, max_npix_h * sizeof(double)));
  CR_CUDA(cudaMalloc(&P->hier_tile_work, max_npix_h * sizeof(float)));
  CR_CUDA(cudaMalloc(&H.d_dot, 4 * sizeof(double)));
  CR_CUDA(cudaMalloc(&H.d_sweep_flag, (max_npix_h / 64 + 1) * sizeof(int)));
  CR_CUDA(cudaMalloc(&H.d_sweep_status, sizeof(int)));
  CR_CUDA(cudaMemset(H.d_sweep_flag, 0, (max_npix_h / 64 + 1) * sizeof(int)));
  CR_CUDA(cudaMalloc(&H.d_sweep_epoch, 2 * sizeof(unsigned int)));
  CR_CUDA(cudaMemset(H.d_sweep_epoch, 0, 2 * sizeof(unsigned int)));
  CR_CUDA(cudaMemset(H.d_sweep_status, 0, sizeof(int)));
  for (int i = 0; i < 5; ++i) CR_CUDA(cudaMalloc(&H.krylov[i], n_lm(L) * sizeof(double2)));
  // settings of the C_l-dependent precompute
  H.ridge_factor = rf;
  H.bisections = nbis;
  H.lam_target = p->ridge_lambda_target == 0.0 ? 1.5 : p->ridge_lambda_target;
  if (p->ridge_alpha && p->nlevels > 0) H.ridge_fixed.assign(p->ridge_alpha, p->ridge_alpha + H.H);
  // smoother structure (geometry only)
  for (int i = 0; i < H.H; ++i)
    if ((rc = smoother_structure(P, H.pix[i]))) return rc;
  if (p->defer_precompute) {
    CR_CUDA(cudaStreamSynchronize(P->stream));
    return CR_OK;
  }
  return build_numeric(P);
}

// The C_l-dependent part of the precompute (Section 5: recomputed whenever
// the prior changes): level arrays, the pixel smoothers' assembly, ridge
// search and factorisation, the top-level diagonal smoother and the bottom
// dense inverse.  Device arrays are updated in place where their sizes allow.
int build_numeric(cr_plan* P) {
  Hierarchy& H = *P->hier;
  const int L = P->lmax;
  H.numeric_ready = false;
  int rc = upload_level_arrays(P);
  if (rc) return rc;
  // pixel smoothers: the paper's ridge search, then (unless the ridges are
  // given) the ridge is raised until the smoother cannot over-correct:
  // lambda_max(S_h A_h) <= target (power-iteration estimate)
  const bool fixed_given = !H.ridge_fixed.empty();
  const double lam_target = H.lam_target;
  for (int i = 0; i < H.H; ++i) {
    PixLevel& lev = H.pix[i];
    if ((rc = smoother_numeric(P, lev, H.ridge_factor, H.bisections, fixed_given ? H.ridge_fixed[i] : -1.0)))
      return rc;
    lev.lambda_max = 0.0;
    if (fixed_given || lam_target < 0.0) continue;
    for (int trial = 0; trial < 24; ++trial) {
      double lam = 0.0;
      if ((rc = smoother_lambda_max(P, i + 1, 12, &lam))) return rc;
      lev.lambda_max = lam;
      if (lam <= lam_target) break;
      double a = lev.alpha > 0.0 ? lev.alpha : 1e-6 * lev.amax;
      a *= std::max(2.0, lam / lam_target);
      bool ok = false;
      if ((rc = factorise(P, lev, (float)a, &ok))) return rc;
      if (!ok) return fail(CR_EICC, "smoother: ICC(0) failed while raising the ridge");
      lev.alpha = a;
    }
  }
  // top-level diagonal smoother and bottom dense level
  std::vector<double> f1 = H.H ? H.pix[0].fl : std::vector<double>(L + 1, 0.0);
  if ((rc = build_top_diag(P, H, f1))) return rc;
  // the same bound for the top-level diagonal smoother: scale the high-pass
  // by target / lambda_max when the estimate exceeds the target
  H.top_scale = 1.0;
  H.top_lambda = 0.0;
  if (lam_target > 0.0 && !fixed_given) {
    double lam = 0.0;
    if ((rc = smoother_lambda_max(P, 0, 12, &lam))) return rc;
    H.top_lambda = lam;
    if (lam > lam_target) {
      H.top_scale = lam_target / lam;
      const int64_t n = n_lm(L);
      std::vector<double> hv(n);
      CR_CUDA(cudaMemcpy(hv.data(), H.inv_diag_hp.d, n * sizeof(double), cudaMemcpyDeviceToHost));
      for (auto& v : hv) v *= H.top_scale;
      if ((rc = H.inv_diag_hp.assign(hv))) return rc;
    }
  }
  if ((rc = build_bottom(P, H))) return rc;
  CR_CUDA(cudaStreamSynchronize(P->stream));
  H.numeric_ready = true;
  return CR_OK;
}

void free_hierarchy(cr_plan* P) {
  if (!P->hier) return;
  Hierarchy& H = *P->hier;
  for (auto& lev : H.pix) {
    free_smoother(lev);
    if (lev.grid) {
      grid_free(*lev.grid);
      delete lev.grid;
    }
    if (lev.gl) {
      grid_free(*lev.gl);
      delete lev.gl;
    }
    if (lev.d_nt) cudaFree(lev.d_nt);
    if (lev.d_nt32) cudaFree(lev.d_nt32);
  }
  if (H.ops_store) {
    HierOps* hops = reinterpret_cast<HierOps*>(H.ops_store);
    for (auto& o : hops->ops) {
      o.b.release();
      o.d.release();
      o.ratio.release();
      o.act.release();
    }
    delete hops;
  }
  for (auto& w : H.work) {
    if (w.x) cudaFree(w.x);
    if (w.b) cudaFree(w.b);
    if (w.r) cudaFree(w.r);
  }
  H.inv_diag_hp.release();
  for (int i = 0; i < 5; ++i)
    if (H.krylov[i]) cudaFree(H.krylov[i]);
  for (auto& w : H.tcw) {
    void* q[] = {w.x, w.b, w.r};
    for (void* p : q)
      if (p) cudaFree(p);
  }
  void* ptrs[] = {H.d_Ainv, H.d_Abottom, H.d_dof_lm, H.map_work, H.map_work2, H.d_dot, P->hier_tile_work,
                  H.d_mr_y, H.d_mr_m1, H.d_mr_m2,
                  H.d_sweep_flag, H.d_sweep_epoch, H.d_sweep_status};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  P->hier_tile_work = nullptr;
  delete P->hier;
  P->hier = nullptr;
}

// relative S^-1-weighted residual sqrt(r^T S^-1 r / b^T S^-1 b) (FP64 vectors)
static int weighted_norm2(cr_plan* P, const void* v, double* out) {
  int rc = launch_dot<double>(v, v, P->d_sinv, P->lmax, P->hier->d_dot, P->d_dotpart, P->stream);
  if (rc) return rc;
  CR_CUDA(cudaMemcpyAsync(out, P->hier->d_dot, sizeof(double), cudaMemcpyDeviceToHost, P->stream));
  CR_CUDA(cudaStreamSynchronize(P->stream));
  return CR_OK;
}

__global__ void nonfinite_kernel(const double* v, int64_t n, int* flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(v[i])) *flag = 1;
}

// Flexible preconditioned CG with one CR-Cycle (from zero) as the
// preconditioner (the use of CR-Cycle inside CG mentioned with Fig. code:mg):
// z = C(r), beta = <z, r - r_old> / <z_old, r_old> (Polak-Ribiere form, so
// that an FP32 cycle -- a slightly nonlinear preconditioner -- stays safe),
// p = z + beta p, alpha = <z, r> / <p, A p>.  Residual and A in FP64.
static int pcg_solve(cr_plan* P, void* x, const void* b, double eps, int max_cycles, bool mixed, bool fixed,
                     double bsb, int* cycles_out, double* relres_out, double* history) {
  Hierarchy& H = *P->hier;
  const int L = P->lmax;
  const int64_t nlm = n_lm(L);
  const size_t bytes = nlm * sizeof(double2);
  // the cycle uses work[0].r internally, so the Krylov residual has its own vector
  void *r = H.krylov[4], *z = H.krylov[0], *rold = H.krylov[1], *pv = H.krylov[2], *q = H.krylov[3];
  void* c32 = H.work[0].x;
  void* r32 = H.work[0].b;
  int rc;
  CR_CUDA(cudaMemsetAsync(x, 0, bytes, P->stream));
  CR_CUDA(cudaMemcpyAsync(r, b, bytes, cudaMemcpyDeviceToDevice, P->stream));
  double zr_old = 0.0, rel = 1.0;
  int k;
  for (k = 1; k <= max_cycles; ++k) {
    // z = C r
    if (!mixed) {
      if ((rc = cycle<double>(P, 0, z, r, true, nullptr))) return rc;
    } else {
      if ((rc = launch_convert_d2f((const double*)r, (float*)r32, 2 * nlm, P->stream))) return rc;
      if ((rc = cycle<float>(P, 0, c32, r32, true, nullptr))) return rc;
      CR_CUDA(cudaMemsetAsync(z, 0, bytes, P->stream));
      if ((rc = launch_add_f2d((double*)z, (const float*)c32, 2 * nlm, P->stream))) return rc;
    }
    double d[3];
    if ((rc = launch_dot<double>(z, r, nullptr, L, H.d_dot, P->d_dotpart, P->stream))) return rc;
    if (k > 1 && (rc = launch_dot<double>(z, rold, nullptr, L, H.d_dot + 1, P->d_dotpart, P->stream))) return rc;
    CR_CUDA(cudaMemcpyAsync(d, H.d_dot, 2 * sizeof(double), cudaMemcpyDeviceToHost, P->stream));
    CR_CUDA(cudaStreamSynchronize(P->stream));
    const double zr = d[0];
    if (k == 1) {
      CR_CUDA(cudaMemcpyAsync(pv, z, bytes, cudaMemcpyDeviceToDevice, P->stream));
    } else {
      const double beta = (zr - d[1]) / zr_old;
      if ((rc = launch_axpby(pv, 1.0, z, beta, nlm, P->stream))) return rc;  // p = z + beta p
    }
    zr_old = zr;
    // q = A p (FP64)
    {
      TimerScope ts(P->timing, P->stream, "outer_residual");
      if ((rc = level_apply<double>(P, 0, pv, q))) return rc;
    }
    if ((rc = launch_dot<double>(pv, q, nullptr, L, H.d_dot + 2, P->d_dotpart, P->stream))) return rc;
    CR_CUDA(cudaMemcpyAsync(d + 2, H.d_dot + 2, sizeof(double), cudaMemcpyDeviceToHost, P->stream));
    CR_CUDA(cudaStreamSynchronize(P->stream));
    if (!(d[2] > 0.0)) return fail(CR_ENONFINITE, "pcg: non-positive curvature p^T A p");
    const double alpha = zr / d[2];
    CR_CUDA(cudaMemcpyAsync(rold, r, bytes, cudaMemcpyDeviceToDevice, P->stream));
    if ((rc = launch_axpby(x, alpha, pv, 1.0, nlm, P->stream))) return rc;   // x += alpha p
    if ((rc = launch_axpby(r, -alpha, q, 1.0, nlm, P->stream))) return rc;   // r -= alpha q
    double rsr = 0.0;
    if ((rc = weighted_norm2(P, r, &rsr))) return rc;
    rel = std::sqrt(std::max(rsr, 0.0) / bsb);
    if (history) history[k - 1] = rel;
    if (!std::isfinite(rel)) {
      if (cycles_out) *cycles_out = k;
      if (relres_out) *relres_out = rel;
      return fail(CR_ENONFINITE, "pcg: non-finite residual");
    }
    if (!fixed && rel * rel < eps) break;
  }
  if (cycles_out) *cycles_out = std::min(k, max_cycles);
  if (relres_out) *relres_out = rel;
  if (k > max_cycles && !fixed) return fail(CR_EMAXITER, "pcg: cycle cap reached before the tolerance");
  return CR_OK;
}

int solve(cr_plan* P, void* x, const void* b, double eps, int max_cycles, int mode, int* cycles_out,
          double* relres_out, double* history) {
  Hierarchy& H = *P->hier;
  const int L = P->lmax;
  const int64_t nlm = n_lm(L);
  double bsb = 1.0, rsr = 0.0;
  int rc = CR_OK;
  // under graph capture (fixed-count stationary solves only) no norm is read
  // back: the stop test and the residual history are skipped
  if (P->capturing && (!(mode & CR_FIXED) || (mode & CR_PCG)))
    return fail(CR_EINVAL, "solve: graph capture needs a fixed-count stationary solve");
  if (!P->capturing && (rc = weighted_norm2(P, b, &bsb))) return rc;
  if (!(bsb > 0.0)) {
    CR_CUDA(cudaMemsetAsync(x, 0, nlm * sizeof(double2), P->stream));
    if (cycles_out) *cycles_out = 0;
    if (relres_out) *relres_out = 0.0;
    return CR_OK;
  }
  if (mode & CR_PCG)
    return pcg_solve(P, x, b, eps, max_cycles, (mode & 3) == CR_MIXED, (mode & CR_FIXED) != 0, bsb, cycles_out,
                     relres_out, history);
  void* r = H.work[0].r;   // FP64 residual
  void* c32 = H.work[0].x; // FP32 correction (mixed mode)
  void* r32 = H.work[0].b; // FP32 residual (mixed mode)
  CR_CUDA(cudaMemsetAsync(x, 0, nlm * sizeof(double2), P->stream));
  CR_CUDA(cudaMemcpyAsync(r, b, nlm * sizeof(double2), cudaMemcpyDeviceToDevice, P->stream));
  double prev = 1.0;
  int grow = 0;
  int k = 0;
  double rel = 1.0;
  for (k = 1; k <= max_cycles; ++k) {
    if ((mode & 3) == CR_F64) {
      if ((rc = cycle<double>(P, 0, x, b, false, r))) return rc;
    } else {
      if ((rc = launch_convert_d2f((const double*)r, (float*)r32, 2 * nlm, P->stream))) return rc;
      if ((rc = cycle<float>(P, 0, c32, r32, true, nullptr))) return rc;
      if ((rc = launch_add_f2d((double*)x, (const float*)c32, 2 * nlm, P->stream))) return rc;
    }
    if ((mode & CR_FIXED) && k == max_cycles) {
      // fixed cycle count: the last residual would only feed the stop test
      if (history) history[k - 1] = std::nan("");
      if (cycles_out) *cycles_out = k;
      if (relres_out) *relres_out = rel;
      return CR_OK;
    }
    // r = b - A x in FP64
    {
      TimerScope ts(P->timing, P->stream, "outer_residual");
      if ((rc = residual<double>(P, 0, x, b, r))) return rc;
    }
    if (P->capturing) {
      rel = std::nan("");
      continue;
    }
    if ((rc = weighted_norm2(P, r, &rsr))) return rc;
    rel = std::sqrt(std::max(rsr, 0.0) / bsb);
    if (history) history[k - 1] = rel;
    if (!std::isfinite(rel)) {
      if (cycles_out) *cycles_out = k;
      if (relres_out) *relres_out = rel;
      return fail(CR_ENONFINITE, "solve: non-finite residual");
    }
    if (mode & CR_FIXED) continue;
    if (rel * rel < eps) break;
    grow = (rel > prev) ? grow + 1 : 0;
    if (grow >= 2) {
      if (cycles_out) *cycles_out = k;
      if (relres_out) *relres_out = rel;
      return fail(CR_EDIVERGED, "solve: residual grew over two consecutive cycles");
    }
    prev = rel;
  }
  if (cycles_out) *cycles_out = std::min(k, max_cycles);
  if (relres_out) *relres_out = rel;
  if (k > max_cycles && !(mode & CR_FIXED)) return fail(CR_EMAXITER, "solve: cycle cap reached before the tolerance");
  return CR_OK;
}

// tensor-core buffers sized for every grid the batched cycle visits, so
// that nothing is allocated once a capture has begun
static int tc_prepare_all(cr_plan* P) {
  Hierarchy& H = *P->hier;
  int rc = ensure_tc_work(P);
  if (!rc) rc = ensure_mr_workspace(P, P->obs, P->lmax);
  if (!rc) rc = tc_begin(P, P->obs, P->lmax, true, true);
  for (int h = 1; h <= H.H && !rc; ++h) {
    const float* pix = nullptr;
    const Grid& g = noise_grid<float>(P, h, &pix);
    rc = tc_begin(P, g, H.pix[h - 1].lmax_h, true, false);
    if (!rc) rc = tc_begin(P, *H.pix[h - 1].grid, H.pix[h - 1].lmax_h, true, false);
  }
  return rc;
}

// Batched mixed-precision CR-Solve: the stationary refinement of solve() for
// nrhs right-hand sides, 16 at a time -- FP64 residual r = b - A x per
// right-hand side, then one batched FP32 cycle (cycle_tc) of the group on
// the FP32 residuals, x += c.  Without `fixed` a group stops when every
// right-hand side meets r^T S^-1 r < eps b^T S^-1 b.
int solve_tc(cr_plan* P, void* x, const void* b, int nrhs, double eps, int max_cycles, bool fixed, int* cycles_out,
             double* relres_out, double* history) {
  Hierarchy& H = *P->hier;
  const int L = P->lmax;
  const int64_t nlm = n_lm(L);
  int rc = CR_OK;
  if (!P->capturing && (rc = tc_prepare_all(P))) return rc;
  if ((int)H.tcw.size() != H.H + 2 || !P->d_tc_status)
    return fail(CR_ESTATE, "solve: batched cycle buffers missing (run the solve once outside a capture)");
  CR_CUDA(cudaMemsetAsync(P->d_tc_status, 0, sizeof(int), P->stream));
  Hierarchy::TcWork& w0 = H.tcw[0];
  void* r64 = H.work[0].r;  // (a batch's FP64 residuals are in P->d_tc_r64)
  bool capped = false;
  for (int r0 = 0; r0 < nrhs; r0 += 16) {
    const int nr = std::min(16, nrhs - r0);
    double2* X = reinterpret_cast<double2*>(x) + r0 * nlm;
    const double2* B = reinterpret_cast<const double2*>(b) + r0 * nlm;
    std::vector<double> bsb(nr, 1.0), rel(nr, 1.0);
    if (!P->capturing)
      for (int j = 0; j < nr; ++j)
        if ((rc = weighted_norm2(P, B + j * nlm, &bsb[j]))) return rc;
    CR_CUDA(cudaMemsetAsync(X, 0, nr * nlm * sizeof(double2), P->stream));
    for (int j = 0; j < nr; ++j)
      if ((rc = launch_convert_d2f((const double*)(B + j * nlm), (float*)(w0.b + j * nlm), 2 * nlm, P->stream)))
        return rc;
    int k;
    bool done = false;
    for (k = 1; k <= max_cycles && !done; ++k) {
      if ((rc = cycle_tc(P, 0, nr, true))) return rc;
      for (int j = 0; j < nr; ++j)
        if ((rc = launch_add_f2d((double*)(X + j * nlm), (const float*)(w0.x + j * nlm), 2 * nlm, P->stream)))
          return rc;
      if (fixed && k == max_cycles) {
        if (history)
          for (int j = 0; j < nr; ++j) history[(int64_t)(r0 + j) * max_cycles + k - 1] = std::nan("");
        break;
      }
      bool all = true;
      // FP64 residuals: up to 8 right-hand sides per pass of the batched
      // FP64 stages (one evaluation of the recurrence for all of them)
      const bool batched = nr > 1 && !P->fp64_df && P->d_tc_r64;
      if (batched) {
        TimerScope ts(P->timing, P->stream, "outer_residual");
        LevelOps& o = ops_of(P).ops[0];
        const double* pix = nullptr;
        const Grid& g0 = noise_grid<double>(P, 0, &pix);
        for (int j0 = 0; j0 < nr && !rc; j0 += 8)
          rc = do_sandwich_mr(P, g0, L, std::min(8, nr - j0), X + j0 * nlm, P->d_tc_r64 + j0 * nlm,
                              o.b.get<double>(), pix, o.b.get<double>(), o.d.get<double>(), B + j0 * nlm);
        if (rc) return rc;
      }
      for (int j = 0; j < nr; ++j) {
        if (batched) {
          r64 = P->d_tc_r64 + j * nlm;
        } else {
          TimerScope ts(P->timing, P->stream, "outer_residual");
          if ((rc = residual<double>(P, 0, X + j * nlm, B + j * nlm, r64))) return rc;
        }
        if (!P->capturing) {
          double rsr = 0.0;
          if ((rc = weighted_norm2(P, r64, &rsr))) return rc;
          rel[j] = bsb[j] > 0.0 ? std::sqrt(std::max(rsr, 0.0) / bsb[j]) : 0.0;
          if (history) history[(int64_t)(r0 + j) * max_cycles + k - 1] = rel[j];
          if (!std::isfinite(rel[j])) return fail(CR_ENONFINITE, "solve: non-finite residual");
          if (!(rel[j] * rel[j] < eps)) all = false;
        }
        if ((rc = launch_convert_d2f((const double*)r64, (float*)(w0.b + j * nlm), 2 * nlm, P->stream))) return rc;
      }
      if (!fixed && !P->capturing && all) done = true;
    }
    const int kk = std::min(done ? k - 1 : k, max_cycles);
    for (int j = 0; j < nr; ++j) {
      if (cycles_out) cycles_out[r0 + j] = kk;
      if (relres_out) relres_out[r0 + j] = fixed ? std::nan("") : rel[j];
    }
    if (!fixed && !done) capped = true;
  }
  if (!P->capturing && (rc = tc_end(P, "batched cycle: a tensor-core completion wait gave up"))) return rc;
  if (capped) return fail(CR_EMAXITER, "solve: cycle cap reached before the tolerance");
  return CR_OK;
}

template <typename T>
int wcycle(cr_plan* P, void* x, const void* b) {
  return cycle<T>(P, 0, x, b, false, nullptr);
}
template int wcycle<double>(cr_plan*, void*, const void*);
template int wcycle<float>(cr_plan*, void*, const void*);

template <typename T>
int level_apply(cr_plan* P, int h, const void* x, void* y) {
  LevelOps& o = ops_of(P).ops[h];
  const T* pix = nullptr;
  const Grid& g = noise_grid<T>(P, h, &pix);
  return do_sandwich<T>(P, g, lmax_of(P, h), x, y, o.b.get<T>(), pix, o.b.get<T>(), o.d.get<T>(), nullptr,
                        nullptr);
}
template <typename T>
int level_restrict(cr_plan* P, int h, const void* in, void* out) {
  return launch_restrict<T>(in, lmax_of(P, h), out, lmax_of(P, h + 1), ops_of(P).ops[h].ratio.get<T>(), P->stream);
}
template <typename T>
int level_prolong(cr_plan* P, int h, const void* c, void* x) {
  return launch_prolong_add<T>(x, lmax_of(P, h), c, lmax_of(P, h + 1), ops_of(P).ops[h].ratio.get<T>(), P->stream);
}
template <typename T>
int level_smooth(cr_plan* P, int h, const void* r, void* c) {
  CR_CUDA(cudaMemsetAsync(c, 0, n_lm(lmax_of(P, h)) * sizeof(typename Tr<T>::C), P->stream));
  return smooth_add<T>(P, h, c, r);
}

}  // namespace cr

using namespace cr;

extern "C" {

static int check_dtype(int dtype, const char* who) {
  if (dtype != CR_F64 && dtype != CR_F32) return fail(CR_EINVAL, std::string(who) + ": dtype must be CR_F64 or CR_F32");
  return CR_OK;
}

static int check_hier(cr_plan* plan, const char* who, bool numeric = false) {
  if (!plan) return fail(CR_EINVAL, std::string(who) + ": null plan");
  if (!plan->hier) return fail(CR_ESTATE, std::string(who) + ": plan was created without levels");
  if (numeric && !plan->hier->numeric_ready)
    return fail(CR_ESTATE, std::string(who) + ": the C_l-dependent precompute was deferred (cr_load or cr_plan_update_cl first)");
  return CR_OK;
}

int cr_plan_level(cr_plan* plan, int h, int* nside_h, int* lmax_h, int* n_rec, double* fl, double* ridge,
                  double* lambda_max) {
  int rc = check_hier(plan, "cr_plan_level");
  if (rc) return rc;
  Hierarchy& H = *plan->hier;
  if (h < 0 || h > H.H + 1) return fail(CR_EINVAL, "cr_plan_level: level out of range");
  const std::vector<double>* f = nullptr;
  std::vector<double> ones(plan->lmax + 1, 1.0);
  if (lambda_max) *lambda_max = 0.0;
  if (h == 0) {
    if (nside_h) *nside_h = 0;
    if (n_rec) *n_rec = H.n_rec_top;
    if (ridge) *ridge = H.top_scale;
    if (lambda_max) *lambda_max = H.top_lambda;
    f = &ones;
  } else if (h <= H.H) {
    const PixLevel& lev = H.pix[h - 1];
    if (nside_h) *nside_h = lev.nside_h;
    if (n_rec) *n_rec = lev.n_rec;
    if (ridge) *ridge = lev.alpha;
    if (lambda_max) *lambda_max = lev.lambda_max;
    f = &lev.fl;
  } else {
    if (nside_h) *nside_h = 0;
    if (n_rec) *n_rec = 0;
    if (ridge) *ridge = 0.0;
    f = &H.fb;
  }
  if (lmax_h) *lmax_h = lmax_of(plan, h);
  if (fl) std::memcpy(fl, f->data(), (plan->lmax + 1) * sizeof(double));
  return CR_OK;
}

int cr_plan_nlevels(cr_plan* plan, int* H) {
  int rc = check_hier(plan, "cr_plan_nlevels");
  if (rc) return rc;
  if (H) *H = plan->hier->H;
  return CR_OK;
}

int cr_plan_level_grid(const cr_plan* cplan, int h, int* kind, int* nring, int64_t* npix) {
  cr_plan* plan = const_cast<cr_plan*>(cplan);
  int rc = check_hier(plan, "cr_plan_level_grid");
  if (rc) return rc;
  if (h < 1 || h > plan->hier->H) return fail(CR_EINVAL, "cr_plan_level_grid: h must be a pixel level");
  const PixLevel& lev = plan->hier->pix[h - 1];
  const Grid& g = lev.gl ? *lev.gl : plan->obs;
  if (kind) *kind = g.kind;
  if (nring) *nring = g.nring;
  if (npix) *npix = g.npix;
  return CR_OK;
}

int cr_level_apply(cr_plan* plan, int h, const void* x, void* y, int dtype) {
  int rc = check_hier(plan, "cr_level_apply");
  if (!rc) rc = check_dtype(dtype, "cr_level_apply");
  if (rc) return rc;
  if (h < 0 || h > plan->hier->H + 1) return fail(CR_EINVAL, "cr_level_apply: level out of range");
  return dtype == CR_F64 ? level_apply<double>(plan, h, x, y) : level_apply<float>(plan, h, x, y);
}

int cr_restrict(cr_plan* plan, int h, const void* r_h, void* r_H, int dtype) {
  int rc = check_hier(plan, "cr_restrict");
  if (!rc) rc = check_dtype(dtype, "cr_restrict");
  if (rc) return rc;
  if (h < 0 || h > plan->hier->H) return fail(CR_EINVAL, "cr_restrict: level out of range");
  return dtype == CR_F64 ? level_restrict<double>(plan, h, r_h, r_H) : level_restrict<float>(plan, h, r_h, r_H);
}

int cr_prolong_add(cr_plan* plan, int h, const void* c_H, void* x_h, int dtype) {
  int rc = check_hier(plan, "cr_prolong_add");
  if (!rc) rc = check_dtype(dtype, "cr_prolong_add");
  if (rc) return rc;
  if (h < 0 || h > plan->hier->H) return fail(CR_EINVAL, "cr_prolong_add: level out of range");
  return dtype == CR_F64 ? level_prolong<double>(plan, h, c_H, x_h) : level_prolong<float>(plan, h, c_H, x_h);
}

int cr_pixel_smoother(cr_plan* plan, int h, const void* map_in, void* map_out, int nrhs, int dtype) {
  int rc = check_hier(plan, "cr_pixel_smoother", true);
  if (!rc) rc = check_dtype(dtype, "cr_pixel_smoother");
  if (rc) return rc;
  if (h < 1 || h > plan->hier->H) return fail(CR_EINVAL, "cr_pixel_smoother: level out of range");
  if (nrhs < 1 || nrhs > 16) return fail(CR_EINVAL, "cr_pixel_smoother: 1 to 16 maps");
  if (!map_in || !map_out) return fail(CR_EINVAL, "cr_pixel_smoother: null map");
  if ((rc = ensure_smoother_batch(plan))) return rc;
  PixLevel& lev = plan->hier->pix[h - 1];
  const int64_t np = lev.grid->npix;
  rc = dtype == CR_F64 ? apply_smoother_mr<double>(plan, lev, nrhs, (const double*)map_in, (double*)map_out, np)
                       : apply_smoother_mr<float>(plan, lev, nrhs, (const float*)map_in, (float*)map_out, np);
  return rc ? rc : sweep_status(plan);
}

int cr_smooth(cr_plan* plan, int h, const void* r, void* c, int dtype) {
  int rc = check_hier(plan, "cr_smooth", true);
  if (!rc) rc = check_dtype(dtype, "cr_smooth");
  if (rc) return rc;
  if (h < 0 || h > plan->hier->H) return fail(CR_EINVAL, "cr_smooth: level out of range");
  rc = dtype == CR_F64 ? level_smooth<double>(plan, h, r, c) : level_smooth<float>(plan, h, r, c);
  return rc ? rc : sweep_status(plan);
}

int cr_bottom_solve(cr_plan* plan, const void* b, void* x, int dtype) {
  int rc = check_hier(plan, "cr_bottom_solve", true);
  if (!rc) rc = check_dtype(dtype, "cr_bottom_solve");
  if (rc) return rc;
  return dtype == CR_F64 ? bottom_solve<double>(plan, *plan->hier, b, x)
                         : bottom_solve<float>(plan, *plan->hier, b, x);
}

int cr_bottom_matrix(cr_plan* plan, double* host, int* nd) {
  int rc = check_hier(plan, "cr_bottom_matrix", true);
  if (rc) return rc;
  return bottom_matrix(plan, host, nd);
}

int cr_wcycle(cr_plan* plan, void* x, const void* b, int nrhs, int dtype) {
  int rc = check_hier(plan, "cr_wcycle", true);
  if (!rc) rc = check_dtype(dtype, "cr_wcycle");
  if (rc) return rc;
  if (nrhs < 0) return fail(CR_EINVAL, "cr_wcycle: nrhs must be >= 0");
  const int64_t nlm = n_lm(plan->lmax);
  const size_t es = dtype == CR_F64 ? sizeof(double2) : sizeof(float2);
  for (int i = 0; i < nrhs; ++i) {
    rc = dtype == CR_F64 ? wcycle<double>(plan, (char*)x + i * nlm * es, (const char*)b + i * nlm * es)
                         : wcycle<float>(plan, (char*)x + i * nlm * es, (const char*)b + i * nlm * es);
    if (rc) return rc;
  }
  return sweep_status(plan);
}

int cr_solve(cr_plan* plan, void* x, const void* b, int nrhs, double eps, int max_cycles, int mode, int* cycles_out,
             double* relres_out, double* history) {
  if (plan && (mode & CR_CG)) {
    if (!plan->has_op) return fail(CR_EINVAL, "cr_solve: CG needs a plan created with C_l");
    if ((mode & 3) != CR_F64) return fail(CR_EINVAL, "cr_solve: CG runs in FP64 (CR_F64)");
    if (max_cycles < 1 || !(eps >= 0.0)) return fail(CR_EINVAL, "cr_solve: eps / max_cycles");
    const int64_t nlm = n_lm(plan->lmax);
    for (int i = 0; i < nrhs; ++i) {
      int rc = cg_solve(plan, (char*)x + i * nlm * sizeof(double2), (const char*)b + i * nlm * sizeof(double2), eps,
                        max_cycles, cycles_out ? cycles_out + i : nullptr, relres_out ? relres_out + i : nullptr,
                        history ? history + (int64_t)i * max_cycles : nullptr);
      if (rc) return rc;
    }
    return CR_OK;
  }
  int rc = check_hier(plan, "cr_solve", true);
  if (rc) return rc;
  if (mode & CR_TC_CYCLES) {
    if ((mode & 3) != CR_MIXED || (mode & CR_PCG))
      return fail(CR_EINVAL, "cr_solve: CR_TC_CYCLES is a stationary CR_MIXED solve");
    if (max_cycles < 1 || !(eps >= 0.0) || nrhs < 0) return fail(CR_EINVAL, "cr_solve: eps / max_cycles / nrhs");
    if (nrhs == 0) return CR_OK;
    plan->tc_top_f32 = (mode & CR_TC_TOP_F32) != 0;
    plan->tc_split = (mode & CR_TC_SPLIT) ? 1 : plan->tc_split_param;
    rc = solve_tc(plan, x, b, nrhs, eps, max_cycles, (mode & CR_FIXED) != 0, cycles_out, relres_out, history);
    plan->tc_split = plan->tc_split_param;
    return rc ? rc : sweep_status(plan);
  }
  if ((mode & 3) != CR_F64 && (mode & 3) != CR_MIXED) return fail(CR_EINVAL, "cr_solve: mode precision must be CR_F64 or CR_MIXED");
  if (max_cycles < 1 || !(eps >= 0.0)) return fail(CR_EINVAL, "cr_solve: eps / max_cycles");
  const int64_t nlm = n_lm(plan->lmax);
  for (int i = 0; i < nrhs; ++i) {
    rc = solve(plan, (char*)x + i * nlm * sizeof(double2), (const char*)b + i * nlm * sizeof(double2), eps,
               max_cycles, mode, cycles_out ? cycles_out + i : nullptr, relres_out ? relres_out + i : nullptr,
               history ? history + (int64_t)i * max_cycles : nullptr);
    if (rc) return rc;
  }
  return sweep_status(plan);
}

}  // extern "C"
