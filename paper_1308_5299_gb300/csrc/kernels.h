// Kernel argument blocks and launcher declarations shared between the
// translation units of the CR solver library.
#pragma once
#include <algorithm>

#include "common.cuh"
#include "plan.h"

namespace cr {

template <typename T>
struct LegArgs {
  const typename Tr<T>::C* alm = nullptr;  // synthesis input, layout off_m(L)
  typename Tr<T>::C* phase = nullptr;      // [nring][ldp]
  int64_t ldp = 0;
  int L = 0;       // band limit of the coefficient vector
  int Lc = 0;      // band limit of the recurrence-table layout
  const T* c = nullptr;
  const T* c2 = nullptr;   // c - 2 (polar difference form)
  const T* s = nullptr;
  const T* dl = nullptr;   // synthesis: per-l multiplier of a_lm (may be null)
  const T* z = nullptr;    // cos(colatitude) per ring (north ring of each pair)
  const T* w = nullptr;    // 1 - z per ring (used by the polar form)
  int npolar = 0;          // pairs [0, npolar) use the polar form z Q = Q - w Q
  const int* ls = nullptr;                 // [m][pair] start l (start tables)
  const typename Tr<T>::C* st = nullptr;   // [m][pair] recurrence state at the start
  int df = 0;                              // FP64 stages in double-float arithmetic (legendre_df.cu)
  int npolar_df = 0;                       // double-float: pairs [0, npolar_df) use the polar form
  const int* ls_df = nullptr;              // double-float start l (FP32 threshold) and FP64 state there
  const double2* st_df = nullptr;
  int ld_seed = 0;
  int npairs = 0, nring = 0;
  typename Tr<T>::C* partial = nullptr;    // adjoint: [nblk][n_lm(L)]
  const T* ringval = nullptr;              // SQ variant: per-ring value
  int rp_synth = 4, rp_adj = 4;            // ring pairs per thread (2, 4, 8) of the two stages
  int mt_synth = 1, mt_adj = 1;            // m tile: 1 (one m per CTA) or 2 (m and L - m per CTA)
  int tc_variant = 0;                      // tensor-core kernels: stage shape (legendre_tc.cu)
  int tc_split = 0;                        // tensor-core kernels: hi + lo BF16 operands
};

template <typename T>
struct FinalizeArgs {
  const typename Tr<T>::C* partial = nullptr;
  int nblk = 1;
  int L = 0;
  const T* dl_out = nullptr;               // per-l multiplier (may be null = 1)
  const T* dadd = nullptr;                 // per-l multiplier of xadd (may be null)
  const typename Tr<T>::C* xadd = nullptr;
  int accumulate = 0;                      // out += result instead of out = result
  const typename Tr<T>::C* bsub = nullptr; // if set: out = bsub - result (residual)
  typename Tr<T>::C* out = nullptr;
};

// Ring FFT stage: mode 0 = synthesis (phase -> map), 1 = adjoint
// (map -> phase), 2 = both with a pixel diagonal in between (phase -> phase).
template <typename T>
struct RingArgs {
  const RingFFT* fft = nullptr;
  const typename Tr<T>::C* tab = nullptr;
  const typename Tr<T>::C* vhat = nullptr;
  const typename Tr<T>::C* tw = nullptr;
  int Mmax = 1;
  typename Tr<T>::C* phase = nullptr;
  int64_t ldp = 0;
  int L = 0;
  T* map_out = nullptr;        // mode 0 output; mode 2 optional copy of Y x
  const T* map_in = nullptr;   // mode 1 input
  const T* pixdiag = nullptr;  // mode 2 diagonal
  int nring = 0;
  const int* rings = nullptr;  // ring indices ordered by FFT size (device)
  int rbase = 0;               // first entry of this launch's class
  int nclass = 0;              // host: FFT-size classes
  const int* cls_M = nullptr;
  const int* cls_start = nullptr;
};

template <typename T> int launch_leg_synth(const LegArgs<T>& a, cudaStream_t st);
template <typename T> int launch_leg_adjoint(const LegArgs<T>& a, const FinalizeArgs<T>& f, cudaStream_t st);
int leg_partial_blocks(int npairs);
int df_pair_blocks(int npairs);
int launch_tc_synth(const LegArgs<float>& la, const float2* alm, int64_t ld_alm, int nrhs, float2* phase,
                    int* status, cudaStream_t st);
int launch_tc_adjoint(const LegArgs<float>& la, const float2* phase, int nrhs, float2* partial, int* nblk,
                      int* status, cudaStream_t st);
int tc_adjoint_blocks(int npolar, int npairs);

// batched tensor-core stages of a plan (plan.cu): phase slots and partial
// rows for 16 right-hand sides, the Legendre stages and the finalisation
struct TcTail {
  const float* dl_out = nullptr;
  const float* dadd = nullptr;
  const float2* xadd = nullptr;
  const float2* bsub = nullptr;
  float2* out = nullptr;
  int accumulate = 0;
};
int tc_begin(cr_plan* P, const Grid& g, int L, bool adjoint, bool reset_status);
int tc_end(cr_plan* P, const char* what);
float2* tc_slot(cr_plan* P, const Grid& g, int L, int r);
int tc_synth_stage(cr_plan* P, const Grid& g, int L, const float2* x, int nr, const float* dl);
int tc_adjoint_tail(cr_plan* P, const Grid& g, int L, int nr, const TcTail& t);
int tc_ring(cr_plan* P, const Grid& g, int L, int r, int mode, const float* map_in, float* map_out);
int tc_sandwich(cr_plan* P, const Grid& g, int L, int nr, const float2* x, const float* dl_in, const float* pix,
                const TcTail& t);
template <typename T> int launch_leg_finalize(const FinalizeArgs<T>& f, cudaStream_t st);
int launch_leg_synth_df(const LegArgs<double>& a, cudaStream_t st);
int launch_leg_adjoint_df(const LegArgs<double>& a, int* nblk, cudaStream_t st);
// FP64 stages of up to 8 right-hand sides at once (legendre_mr.cu)
int mr_blocks(int npairs);
int launch_leg_synth_mr(const LegArgs<double>& a, const double2* alm, int64_t ld_alm, int nr, double2* phase,
                        int64_t ld_phase, cudaStream_t st);
int launch_leg_adjoint_mr(const LegArgs<double>& a, const double2* phase, int64_t ld_phase, int nr, double2* partial,
                          int* nblk, cudaStream_t st);
// y_r = dl_out Y^T diag(pix) Y (dl_in x_r) + dadd x_r, or bsub_r - that, in
// FP64 for nr <= 8 right-hand sides at stride n_lm(L) (plan.cu)
int do_sandwich_mr(cr_plan* P, const Grid& g, int L, int nr, const double2* x, double2* y, const double* dl_in,
                   const double* pix, const double* dl_out, const double* dadd, const double2* bsub);
int ensure_mr_workspace(cr_plan* P, const Grid& g, int L);
int launch_leg_diag(cr_plan* P, const double* ringval, double2* out);
template <typename T> int launch_ring_fft(const RingArgs<T>& a, int mode, cudaStream_t st);

// transform drivers (plan.cu)
template <typename T> int do_synth(cr_plan* P, const Grid& g, int L, const void* alm, void* map, const T* dl);
template <typename T>
int do_adjoint(cr_plan* P, const Grid& g, int L, const void* map, void* alm, const T* dl_out, const T* dadd,
               const void* xadd, int accumulate);
template <typename T>
int do_sandwich(cr_plan* P, const Grid& g, int L, const void* x, void* y, const T* dl_in, const T* pix,
                const T* dl_out, const T* dadd, T* map_copy, const void* bsub);

// grids and workspace (plan.cu)
void healpix_rings(Grid& g, int N);
void gl_rings(Grid& g, int ntheta, int nphi, std::vector<double>* weights);
int grid_reseed(Grid& g, int Lseed, cudaStream_t st);
int rebuild_coef(cr_plan* P, int Lc);
int grid_upload(Grid& g, int Lseed, cudaStream_t st);
void grid_free(Grid& g);
int ensure_workspace(cr_plan* P, const Grid& g, int L);

// plan-time table builders (ringfft.cu)
int build_fft_tables(Grid& g, cudaStream_t st);
int build_seeds(Grid& g, int Lseed, cudaStream_t st);
int build_start_tables(cr_plan* P, Grid& g);

}  // namespace cr
