// Declarations shared by the multi-level translation units.
#pragma once
#include <vector>

#include "common.cuh"
#include "healpix.cuh"
#include "hier.h"

namespace cr {

struct LevelSpec {
  int nside_h = 0, lmax_h = 0, n_rec = 2;
  std::vector<double> fl;
};

std::vector<double> q_filter(int lmax, double ell_star, double value);
std::vector<double> gauss_filter(int lmax, int nside_h);
int first_level_nside(int nside, int lmax, int k);
void default_levels(int nside, int lmax, int k, std::vector<LevelSpec>& out, int* lmax_dense);
void tile_pattern(int nside_t, BlockPattern& P);


template <typename T> int launch_restrict(const void* in, int Lh, void* out, int LH, const T* ratio, cudaStream_t st);
template <typename T> int launch_prolong_add(void* x, int Lh, const void* c, int LH, const T* ratio, cudaStream_t st);
template <typename T> int launch_diag_axpy(void* x, const void* r, const T* d, int64_t n, cudaStream_t st);
int launch_fill_random(void* v, int L, uint32_t seed, cudaStream_t st);
int launch_axpby(void* y, double a, const void* x, double b, int64_t n, cudaStream_t st);
int launch_scale_copy(const void* in, void* out, float s, int64_t n, cudaStream_t st);
// out = weighted real inner product (FP64); part: scratch of >= L + 1 doubles
template <typename T>
int launch_dot(const void* a, const void* b, const double* wl, int L, double* out, double* part, cudaStream_t st);
int launch_convert_d2f(const double* in, float* out, int64_t n, cudaStream_t st);
int launch_add_f2d(double* x, const float* y, int64_t n, cudaStream_t st);

// smoother.cu
int smoother_structure(cr_plan* P, PixLevel& lev);
int smoother_numeric(cr_plan* P, PixLevel& lev, double ridge_factor, int bisections, double fixed_alpha);
int factorise(cr_plan* P, PixLevel& lev, float alpha, bool* ok);
template <typename T> int apply_smoother(cr_plan* P, PixLevel& lev, T* map_in, T* map_out);
template <typename T>
int apply_smoother_mr(cr_plan* P, PixLevel& lev, int nr, const T* map_in, T* map_out, int64_t ld);
int ensure_smoother_batch(cr_plan* P);
int sweep_status(cr_plan* P);
void free_smoother(PixLevel& lev);

// dense.cu
int build_bottom(cr_plan* P, Hierarchy& Hh);
std::vector<int32_t> bottom_dof_map(const cr_plan* P, int Ld);
template <typename T> int bottom_solve(cr_plan* P, Hierarchy& Hh, const void* b, void* x);
int bottom_matrix(cr_plan* P, double* host, int* nd);
int bottom_upload(cr_plan* P, Hierarchy& Hh, int nd, const double* a, const double* ainv, const int32_t* dofs);
int build_top_diag(cr_plan* P, Hierarchy& Hh, const std::vector<double>& f1);
int inv_diag_A(cr_plan* P, const std::vector<double>& hpl, double* out);
int cg_solve(cr_plan* P, void* x, const void* b, double eps, int maxit, int* it_out, double* relres_out,
             double* history);

// solver.cu
int build_hierarchy(cr_plan* P, const cr_params* p);
int build_numeric(cr_plan* P);
void free_hierarchy(cr_plan* P);

}  // namespace cr
