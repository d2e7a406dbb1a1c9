// Shared device/host helpers of the CR solver library (complex arithmetic on
// double2/float2, real-type traits, error plumbing).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "cr.h"

namespace cr {

// ---- real-type traits ------------------------------------------------------
template <typename T> struct Tr;
template <> struct Tr<double> {
  using C = double2;
  // Underflow-safe Legendre recurrence: values are carried as v * 2^(S*lev)
  // with lev <= 0; while lev < 0 they are renormalised by 2^-S whenever
  // |v| > 2^THR, so lev < 0 means |true value| <= 2^(THR-S) (negligible).
  static constexpr int S = 600;
  static constexpr int THR = 300;
};
template <> struct Tr<float> {
  using C = float2;
  static constexpr int S = 96;
  static constexpr int THR = 24;
};

__host__ __device__ inline double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ inline float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ inline float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__host__ __device__ inline float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// i * a
__host__ __device__ inline double2 cmuli(double2 a) { return make_double2(-a.y, a.x); }
__host__ __device__ inline float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }

__host__ __device__ inline int64_t lm_off(int L, int m) {
  return (int64_t)m * (L + 1) - (int64_t)m * (m - 1) / 2;
}
__host__ __device__ inline int64_t n_lm(int L) { return (int64_t)(L + 1) * (L + 2) / 2; }

// ---- launch accounting (kernels launched by the library, process-wide) ----
void count_launch(long n = 1);
long launch_count();

// ---- error plumbing ----------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

}  // namespace cr

#define CR_CUDA(call)                                          \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return ::cr::cuda_fail(e_, #call);  \
  } while (0)

#define CR_CHECK_LAUNCH(what)                                  \
  do {                                                         \
    cudaError_t e_ = cudaGetLastError();                       \
    if (e_ != cudaSuccess) return ::cr::cuda_fail(e_, what);   \
  } while (0)
