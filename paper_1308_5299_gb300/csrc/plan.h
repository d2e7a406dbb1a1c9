// Internal plan and grid structures of the CR solver library.
#pragma once
#include <map>
#include <string>
#include <vector>

#include "common.cuh"

namespace cr {

// Per-ring FFT description.  A ring of n pixels (n even) is transformed as a
// complex sequence of nh = n/2 values (real-data packing).  If nh is a power
// of two the FFT has size M = nh; otherwise Bluestein's chirp-z algorithm is
// used with a power-of-two convolution of size M >= 2 nh - 1.
struct RingFFT {
  int n;         // pixels on the ring
  int nh;        // n / 2
  int M;         // power-of-two FFT size
  int logM;      // log2(M)
  int bluestein; // 1 if nh is not a power of two
  int shift;     // azimuth of pixel j is pi (2 j + shift) / n, shift in {0, 1}
  int64_t off;   // first pixel of the ring in the map
  int64_t tab;   // offset of this ring length's e^{i pi u / n}, u < 2n, table
  int64_t vhat;  // offset of the Bluestein kernel spectrum (bit-reversed, /M)
};

// A ring grid with its transform tables.
struct Grid {
  int kind = CR_GRID_HEALPIX;
  int nside = 0;
  int nring = 0;
  int npairs = 0;  // north/south ring pairs (the middle ring pairs with itself)
  int64_t npix = 0;
  int Lseed = -1;  // seeds exist for m <= Lseed
  int Mmax = 1;    // largest FFT size
  std::vector<double> z, sth;
  std::vector<RingFFT> fft;
  std::vector<int> cls_M, cls_start;  // FFT-size classes over d_rings
  int* d_rings = nullptr;             // ring indices ordered by FFT size
  // device tables
  double* d_z = nullptr;      // [nring]
  float* d_z32 = nullptr;     // [nring]
  float* d_w32 = nullptr;     // [nring] 1 - z (FP32 polar recurrence form)
  int npolar32 = 0;           // FP32: pairs [0, npolar32) use the polar form
  double* d_sth = nullptr;    // [nring]
  RingFFT* d_fft = nullptr;   // [nring]
  double2* d_tab = nullptr;   // concatenated e^{i pi u/n}
  float2* d_tab32 = nullptr;
  double2* d_vhat = nullptr;  // concatenated Bluestein spectra
  float2* d_vhat32 = nullptr;
  double2* d_tw = nullptr;    // e^{-2 pi i j / Mmax}, j < Mmax/2
  float2* d_tw32 = nullptr;
  int64_t tab_len = 0, vhat_len = 0;
  // Legendre seeds P~_mm(z_pair) in scaled form, [m][pair]
  double* d_seed = nullptr;
  int* d_lev = nullptr;
  float* d_seed32 = nullptr;
  int* d_lev32 = nullptr;
  // Legendre start tables, [m][pair] for m <= Lseed: the first l with
  // |P~_lm| >= tau (FP64 2^-100, FP32 2^-60; Lseed + 1 if none) and the
  // recurrence state there: (Q_{l-1}, Q_{l-2}), or (Q_{l-1}, D_{l-1}) on the
  // FP32 polar pairs; built from the plan's recurrence tables
  int* d_ls64 = nullptr;
  double2* d_st64 = nullptr;
  int* d_ls32 = nullptr;
  float2* d_st32 = nullptr;
  double2* d_st64b = nullptr;  // FP64 state at the FP32 start (double-float kernels)
  // number of (ring pair, l, m) terms the Legendre kernels evaluate at band
  // limit L -- those at or past the 2^-60 start of each (m, pair) -- filled
  // on demand from the start table (per-stage timing only)
  std::map<int, double> exec_terms;
};

// Scratch sizes for transforms at band limit L on a grid (ws_mr: the FP64
// stages of several right-hand sides, [8][...] of each).
struct Workspace {
  void* phase = nullptr;   // [nring][ldp] complex (sized for double2)
  void* partial = nullptr; // [nblk][n_lm] complex (sized for double2)
  int64_t phase_bytes = 0, partial_bytes = 0;
};

// Optional per-stage CUDA-event timing (enabled with cr_plan_set_timing).
struct Timing {
  bool enabled = false;
  struct Rec {
    std::string name;
    cudaEvent_t a, b;
    double work;
    double work_exec;
  };
  struct Acc {
    double ms = 0.0;
    long n = 0;
    double work = 0.0;       // algorithmic flops (or bytes) of the recorded launches
    double work_exec = 0.0;  // Legendre stages: flops of the terms actually evaluated
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  std::map<std::string, Acc> acc;
  cudaEvent_t get();
  void flush();
  ~Timing();
};

class TimerScope {
 public:
  TimerScope(Timing& t, cudaStream_t st, const char* name, double work = 0.0, double work_exec = 0.0);
  TimerScope(Timing& t, cudaStream_t st, const std::string& name, double work = 0.0, double work_exec = 0.0);
  ~TimerScope();

 private:
  Timing* t_;
  cudaStream_t st_;
  int idx_;
};

struct Level {
  int nside_h = 0;
  int lmax_h = 0;
};

}  // namespace cr

namespace cr {
struct Hierarchy;
}

struct cr_plan {
  cr_params p{};
  cudaStream_t stream = nullptr;
  int lmax = 0;
  int Lcoef = -1;
  cr::Grid obs;
  std::vector<cr::Grid*> level_grids;  // pixel grids of levels 1..H
  std::vector<cr::Level> levels;       // levels[0] = top
  // Legendre recurrence tables, layout off_m(Lcoef) + l - m
  double* d_c = nullptr;
  double* d_s = nullptr;
  float* d_c32 = nullptr;
  float* d_c2_32 = nullptr;  // c - 2, FP32 (polar difference form)
  float* d_s32 = nullptr;
  // operator diagonals (l-indexed, [lmax+1])
  bool has_op = false;
  double* d_bl = nullptr;    // b_l p_l, 0 where C_l = 0
  double* d_sinv = nullptr;  // 1/C_l, 0 where C_l = 0
  float* d_bl32 = nullptr;
  float* d_sinv32 = nullptr;
  double* d_ninv = nullptr;  // [npix] obs grid
  float* d_ninv32 = nullptr;
  cr::Workspace ws;
  cr::Workspace ws_mr;
  double2* d_tc_r64 = nullptr;  // FP64 residuals of a batch of 16 right-hand sides
  cr::Timing timing;
  int fp64_df = 0;  // FP64 Legendre stages in double-float arithmetic
  bool capturing = false;  // inside a CUDA-graph capture: no host synchronisation
  void* tc_phase = nullptr;  // batched tensor-core synthesis: [16][nring][L+1] complex64
  int64_t tc_phase_bytes = 0;
  int* d_tc_status = nullptr;
  bool tc_top_f32 = false;   // batched cycles: top-level residuals on the FP32 CUDA-core kernels
  int tc_split = 0;          // tensor-core contractions with hi + lo BF16 operands (in effect)
  int tc_split_param = 0;    // the plan option (CR_TC_SPLIT turns it on for one solve or batch)
  void* tc_partial = nullptr;  // batched tensor-core adjoint: [16][nblk][n_lm] complex64
  int64_t tc_partial_bytes = 0;
  cr::Hierarchy* hier = nullptr;      // multi-level data (plans created with levels)
  void* hier_tile_work = nullptr;     // FP32 tile-ordered smoother work vector
  // diagonal-preconditioned CG (created on first use)
  double* d_dotpart = nullptr;        // [lmax + 1] per-m partial sums of inner products
  double* d_pcinv = nullptr;          // [n_lm] 1 / diag(A), 0 where C_l = 0
  void* cgv[4] = {nullptr, nullptr, nullptr, nullptr};
  double* d_cgdot = nullptr;
  std::vector<double> h_cl, h_bl;
};
