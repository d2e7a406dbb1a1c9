// Arithmetic peak probes for the roofline denominators: sustained FMA rate of
// the FP32 pipe (scalar FFMA and packed f32x2 FMA) and of the FP64 pipe,
// measured with CUDA events on the device the library runs on.  Measurement
// tooling with no counterpart in the paper; the Legendre stages are bound by
// these pipes, not by a dense contraction or by HBM.
//
// Each thread runs NCH independent FMA chains (enough to cover the pipe's
// latency at a few warps per scheduler), unrolled, for `iters` rounds; the
// grid fills every SM several times over.  The chains' values are folded into
// one store per thread behind a data-dependent branch the compiler cannot
// remove, so no FMA is dead code.
#include "common.cuh"

namespace cr {

constexpr int PROBE_NT = 256;
constexpr int PROBE_NCH = 8;

__global__ void __launch_bounds__(PROBE_NT) probe_f32_kernel(float* out, int iters, float a, float b) {
  float v[PROBE_NCH];
#pragma unroll
  for (int c = 0; c < PROBE_NCH; ++c) v[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < PROBE_NCH; ++c) v[c] = fmaf(v[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < PROBE_NCH; ++c) s += v[c];
  if (s == 1234.5f) out[blockIdx.x * PROBE_NT + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_NT) probe_f32x2_kernel(float* out, int iters, float a, float b) {
  unsigned long long v[PROBE_NCH], A, B;
  asm("mov.b64 %0, {%1, %1};" : "=l"(A) : "f"(a));
  asm("mov.b64 %0, {%1, %1};" : "=l"(B) : "f"(b));
#pragma unroll
  for (int c = 0; c < PROBE_NCH; ++c) {
    const float x = (float)(threadIdx.x + c) * 1e-3f;
    asm("mov.b64 %0, {%1, %2};" : "=l"(v[c]) : "f"(x), "f"(x + 1.f));
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < PROBE_NCH; ++c) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(v[c]) : "l"(A), "l"(B));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < PROBE_NCH; ++c) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v[c]));
    s += lo + hi;
  }
  if (s == 1234.5f) out[blockIdx.x * PROBE_NT + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PROBE_NT) probe_f64_kernel(float* out, int iters, double a, double b) {
  double v[PROBE_NCH];
#pragma unroll
  for (int c = 0; c < PROBE_NCH; ++c) v[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < PROBE_NCH; ++c) v[c] = fma(v[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PROBE_NCH; ++c) s += v[c];
  if (s == 1234.5) out[blockIdx.x * PROBE_NT + threadIdx.x] = (float)s;
}

}  // namespace cr

using namespace cr;

extern "C" int cr_probe_fma_peak(int kind, double* tflops) {
  if (!tflops || kind < 0 || kind > 2) return fail(CR_EINVAL, "cr_probe_fma_peak: kind 0 (FP32), 1 (FP32x2), 2 (FP64)");
  int dev = 0, nsm = 0;
  CR_CUDA(cudaGetDevice(&dev));
  CR_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = nsm * 8;
  // FP64 runs at a small fraction of the FP32 rate: fewer rounds
  const int iters = kind == 2 ? 64 : 2048;
  float* out = nullptr;
  CR_CUDA(cudaMalloc(&out, (size_t)blocks * PROBE_NT * sizeof(float)));
  cudaEvent_t e0, e1;
  CR_CUDA(cudaEventCreate(&e0));
  CR_CUDA(cudaEventCreate(&e1));
  auto launch = [&]() {
    if (kind == 0) probe_f32_kernel<<<blocks, PROBE_NT>>>(out, iters, 0.999f, 1e-4f);
    else if (kind == 1) probe_f32x2_kernel<<<blocks, PROBE_NT>>>(out, iters, 0.999f, 1e-4f);
    else probe_f64_kernel<<<blocks, PROBE_NT>>>(out, iters, 0.999, 1e-4);
    count_launch();
  };
  launch();  // warm-up
  float best = 1e30f;
  cudaError_t err = cudaSuccess;
  for (int r = 0; r < 5 && err == cudaSuccess; ++r) {
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess) best = fminf(best, ms);
  }
  if (err == cudaSuccess) err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (err != cudaSuccess) return cuda_fail(err, "cr_probe_fma_peak");
  const double lanes = kind == 1 ? 2.0 : 1.0;  // FMAs per thread instruction
  const double fmas = (double)blocks * PROBE_NT * iters * 16.0 * PROBE_NCH * lanes;
  *tflops = 2.0 * fmas / (best * 1e-3) / 1e12;
  return CR_OK;
}
