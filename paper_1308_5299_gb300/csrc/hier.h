// Multi-level hierarchy of the CR solver (Sections 3.2-3.5, Fig. code:mg):
// level 0 is the spherical-harmonic top level (band limit lmax, filter 1,
// diagonal error smoother); levels 1..H are spherical-harmonic levels with a
// sibling HEALPix pixel grid and a block incomplete-Cholesky error smoother;
// the bottom level is a dense solve over l <= lmax_dense.
#pragma once
#include <vector>

#include "common.cuh"
#include "plan.h"

namespace cr {

// Per-precision device copies of an l-indexed array.
struct LArr {
  double* d = nullptr;
  float* f = nullptr;
  int n = 0;
  int upload(const std::vector<double>& h);
  // copy into the existing arrays when the size is unchanged (device
  // pointers stay valid, e.g. inside captured CUDA graphs), else upload
  int assign(const std::vector<double>& h);
  void release();
  template <typename T> const T* get() const;
};
template <> inline const double* LArr::get<double>() const { return d; }
template <> inline const float* LArr::get<float>() const { return f; }

// Block-sparse lower-triangular storage over tiles in elimination order.
// Row p holds blocks (p, q) for neighbouring q < p (ascending q), then the
// diagonal block (p, p).  Blocks are kk x kk, stored column-major.
struct BlockPattern {
  int ntile = 0;
  int kk = 0;
  std::vector<int> order;         // position -> NESTED tile index
  std::vector<int> pos;           // NESTED tile index -> position
  std::vector<int> colour_start;  // positions of colour c: [cs[c], cs[c+1])
  std::vector<int64_t> row_ptr;   // [ntile + 1]
  std::vector<int> row_col;       // column position of each block
  std::vector<std::vector<int>> nb;  // NESTED neighbour lists (incl. self)
  int64_t nblocks = 0;
  int64_t block_of(int p, int q) const;  // -1 if (p, q) is not stored
};

struct SmootherBuild;

struct PixLevel {
  int nside_h = 0, lmax_h = 0, n_rec = 1, k = 8, nside_t = 0;
  std::vector<double> fl;  // cumulative filter, [lmax + 1], 0 above lmax_h
  Grid* grid = nullptr;    // pixel grid (RING order) at lmax_h
  // Gauss-Legendre grid of the level's inverse-noise term (Section 3.4), or
  // null (the observation grid); d_nt = quadrature-weighted band-limited
  // inverse-noise map on it
  Grid* gl = nullptr;
  double* d_nt = nullptr;
  float* d_nt32 = nullptr;
  LArr bh, dh;             // B_h = f b p, D_h = f^2 / C  (0 where C_l = 0), [lmax_h + 1]
  BlockPattern pat;
  double alpha = 0.0;      // ridge used for the factorisation
  double amax = 0.0;       // max |A_hat| entry
  double lambda_max = 0.0; // power-iteration estimate of lambda_max(S_h A_h) after the ridge
  // device
  float* d_A = nullptr;    // A_hat blocks
  float* d_L = nullptr;    // factor blocks (diagonal blocks hold inv(L_pp))
  float* d_LT = nullptr;   // backward-sweep copy: per position p, column p's blocks transposed, then inv(L_pp)^T
  bool lt_valid = false;
  int* d_perm = nullptr;   // tile-ordered level pixel -> RING index
  int* d_colour_start = nullptr;  // device copy of pat.colour_start
  int coop_grid = 0;       // CTAs of the one-launch cooperative sweeps (0: one launch per colour)
  void* d_flow_task = nullptr;  // their per-CTA task lists (smoother.cu)
  int* d_flow_off = nullptr;
  int64_t* d_row_ptr = nullptr;
  int* d_row_col = nullptr;
  // column lists for the backward solve: blocks (u, p), u > p
  int64_t* d_col_ptr = nullptr;
  int* d_col_row = nullptr;
  int64_t* d_col_blk = nullptr;
  // ICC update lists per position p: for each later neighbour u (and the
  // diagonal), the pairs of blocks (L_uk, L_pk), k < p coupled to both
  int64_t* d_upd_ptr = nullptr;     // [ntile + 1] into targets
  int64_t* d_tgt_blk = nullptr;     // target block (u, p) or (p, p)
  int* d_tgt_u = nullptr;           // u (== p for the diagonal)
  int64_t* d_tgt_ptr = nullptr;     // [ntargets + 1] into pair lists
  int64_t* d_pair_a = nullptr;      // block (u, k)
  int64_t* d_pair_b = nullptr;      // block (p, k)
  int* d_fail = nullptr;            // factorisation failure flag
  SmootherBuild* sb = nullptr;      // assembly inputs (smoother.cu)
};

struct Hierarchy {
  int H = 0;                  // number of pixel levels
  int k = 8;
  std::vector<PixLevel> pix;  // levels 1..H -> pix[0..H-1]
  int n_rec_top = 1;
  // top-level diagonal smoother: x += H_l r / diag(A)
  LArr inv_diag_hp;           // [n_lm(lmax)] (highpass / diag(A)), complex-storage index
  double top_lambda = 0.0;    // lambda_max estimate of the top smoother (before scaling)
  double top_scale = 1.0;     // damping applied to the top smoother
  // bottom dense level
  int ld = 0;
  std::vector<double> fb;     // bottom filter [lmax + 1]
  int nd = 0;                 // active real dofs of the bottom block
  int nd_alloc = 0;           // dofs the bottom arrays are allocated for
  double* d_Ainv = nullptr;   // [nd][nd] inverse of the bottom A (FP64)
  double* d_Abottom = nullptr; // [nd][nd] the assembled bottom A (FP64)
  int* d_dof_lm = nullptr;    // real dof -> (lm index * 2 + part)
  LArr bd;                    // B at the bottom, used by the ring formula
  // per-level work vectors (complex, sized for double2)
  struct Work {
    void *x = nullptr, *b = nullptr, *r = nullptr;
  };
  std::vector<Work> work;     // [H + 2]: 0 = top, 1..H, H+1 = bottom
  void* map_work = nullptr;   // largest level pixel map (double)
  void* map_work2 = nullptr;
  double* d_dot = nullptr;    // dot-product scratch
  int* d_sweep_flag = nullptr;          // per-tile progress flags of the cooperative smoother sweeps
  unsigned int* d_sweep_epoch = nullptr;  // their launch epoch and exit count [2]
  int* d_sweep_status = nullptr;        // set when a wait of those sweeps gave up
  double* d_dot_host = nullptr;
  void* ops_store = nullptr;  // per-level operator arrays (solver.cu)
  void* krylov[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // PCG vectors (FP64, top level)
  // FP32 work vectors of the batched cycles (16 right-hand sides each,
  // [16][n_lm(lmax_h)] complex64), allocated on first use
  struct TcWork {
    float2 *x = nullptr, *b = nullptr, *r = nullptr;
  };
  std::vector<TcWork> tcw;  // [H + 2]
  // settings of the C_l-dependent precompute, kept for cr_plan_update_cl
  double ridge_factor = 1.5;
  int bisections = 30;
  double lam_target = 1.5;
  std::vector<double> ridge_fixed;  // given ridges per pixel level, or empty
  bool numeric_ready = false;       // smoothers, top diagonal and bottom built
  int smoother_kind = 0;            // 0 multicolour block ICC(0), 1 additive Schwarz (block Jacobi)
  // batch buffers of the many-map pixel smoother (smoother.cu): tile work
  // vectors and two map panels of 16 x the largest level, made on first use
  float* d_mr_y = nullptr;
  float* d_mr_m1 = nullptr;
  float* d_mr_m2 = nullptr;
  int64_t mr_y_len = 0;
  int sweep_mode = 0;               // ICC(0) sweeps: 0 auto, 1 one launch per colour, 2 cooperative
};

}  // namespace cr
