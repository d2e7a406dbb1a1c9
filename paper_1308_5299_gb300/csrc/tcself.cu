// Tensor-core self-test: one 128 x 32 x K BF16 GEMM tile (tcgen05.mma,
// FP32 accumulation in tensor memory) against the same product on the CUDA
// cores.  Inputs are small integers (exact in BF16, exact FP32 sums), so a
// correct tile reproduces the reference exactly.
#include "common.cuh"
#include "tc.cuh"

namespace cr {

constexpr int TC_M = 128, TC_N = 32, TC_KMAX = 64;

__global__ void __launch_bounds__(128) tc_selftest_kernel(int K, float* D, float* Dref, int* status) {
  __shared__ __align__(1024) uint8_t smA[TC_M * TC_KMAX * 2];
  __shared__ __align__(1024) uint8_t smB[TC_N * TC_KMAX * 2];
  __shared__ uint64_t mbar;
  __shared__ uint32_t taddr_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto aval = [](int r, int k) { return (float)(((r * 7 + k * 3) % 9) - 4); };
  auto bval = [](int n, int k) { return (float)(((n * 5 + k * 11) % 7) - 3); };
  // operands into the K-major no-swizzle layout
  for (int e = tid; e < TC_M * K; e += 128) {
    const int r = e / K, k = e % K;
    *reinterpret_cast<__nv_bfloat16*>(smA + tc::kmajor_offset(r, k, K)) = __float2bfloat16(aval(r, k));
  }
  for (int e = tid; e < TC_N * K; e += 128) {
    const int n = e / K, k = e % K;
    *reinterpret_cast<__nv_bfloat16*>(smB + tc::kmajor_offset(n, k, K)) = __float2bfloat16(bval(n, k));
  }
  if (warp == 0) tc::tmem_alloc(&taddr_s, 32);
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::mbar_fence_init();
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = taddr_s;
  if (tid == 0) {
    const uint32_t idesc = tc::idesc_bf16_f32(TC_M, TC_N);
    const uint32_t a0 = tc::smem_addr(smA), b0 = tc::smem_addr(smB);
    for (int kk = 0; kk < K / 16; ++kk) {
      const uint64_t ad = tc::smem_desc(a0 + kk * 256, 128, (K / 8) * 128);
      const uint64_t bd = tc::smem_desc(b0 + kk * 256, 128, (K / 8) * 128);
      tc::mma_bf16(taddr, ad, bd, idesc, kk > 0);
    }
    tc::mma_commit(&mbar);
  }
  const bool ok = tc::mbar_wait_block(&mbar, 0, 1u << 24);
  if (!ok) {
    // a second bounded wait before tensor memory is freed below
    tc::mbar_wait_block(&mbar, 0, 1u << 24);
    if (tid == 0) atomicExch(status, 2);
  }
  tc::fence_after_sync();
  if (ok) {
    float v[32];
    tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16), v);
    const int r = warp * 32 + lane;
    for (int n = 0; n < TC_N; ++n) D[r * TC_N + n] = v[n];
  }
  // reference on the CUDA cores
  for (int e = tid; e < TC_M * TC_N; e += 128) {
    const int r = e / TC_N, n = e % TC_N;
    float s = 0.f;
    for (int k = 0; k < K; ++k) s += aval(r, k) * bval(n, k);
    Dref[e] = s;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(taddr, 32);
}

// The same tile with both operands in the MN-major ("transposed") layout
// without swizzle: core matrix (i, j) holds MN rows 8 i .. 8 i + 7 and K
// columns 8 j .. 8 j + 7 as 8 rows of 16 bytes, one per K index, each row
// 8 consecutive MN elements; core matrices adjacent in MN are 128 bytes
// apart, those adjacent in K (MN / 8) * 128 bytes apart.  `swap` exchanges
// which of the two descriptor offsets carries which stride.  The operand
// buffers are sized so that either reading of the offsets stays inside
// them (a wrong reading gives wrong numbers, never an out-of-range access).
constexpr int TCM_ABUF = 2 * TC_M * TC_KMAX * 2;  // twice the A operand
constexpr int TCM_BBUF = 2 * TC_N * TC_KMAX * 2 + 8 * 2048;

__device__ __forceinline__ uint32_t mn_offset(int mn, int k, int MN) {
  return (uint32_t)(((mn >> 3) * 128) + ((k >> 3) * (MN / 8) * 128) + ((k & 7) << 4) + ((mn & 7) << 1));
}

__global__ void __launch_bounds__(128) tc_selftest_mn_kernel(int K, int swap, float* D, float* Dref, int* status) {
  extern __shared__ __align__(1024) uint8_t tcm[];
  uint8_t* smA = tcm;
  uint8_t* smB = tcm + TCM_ABUF;
  __shared__ uint64_t mbar;
  __shared__ uint32_t taddr_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto aval = [](int r, int k) { return (float)(((r * 7 + k * 3) % 9) - 4); };
  auto bval = [](int n, int k) { return (float)(((n * 5 + k * 11) % 7) - 3); };
  for (int e = tid; e < TCM_ABUF / 2; e += 128) reinterpret_cast<__nv_bfloat16*>(smA)[e] = __float2bfloat16(0.f);
  for (int e = tid; e < TCM_BBUF / 2; e += 128) reinterpret_cast<__nv_bfloat16*>(smB)[e] = __float2bfloat16(0.f);
  __syncthreads();
  for (int e = tid; e < TC_M * K; e += 128) {
    const int r = e / K, k = e % K;
    *reinterpret_cast<__nv_bfloat16*>(smA + mn_offset(r, k, TC_M)) = __float2bfloat16(aval(r, k));
  }
  for (int e = tid; e < TC_N * K; e += 128) {
    const int n = e / K, k = e % K;
    *reinterpret_cast<__nv_bfloat16*>(smB + mn_offset(n, k, TC_N)) = __float2bfloat16(bval(n, k));
  }
  if (warp == 0) tc::tmem_alloc(&taddr_s, 32);
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::mbar_fence_init();
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = taddr_s;
  if (tid == 0) {
    // transpose A and B (bits 15 and 16 of the instruction descriptor)
    const uint32_t idesc = tc::idesc_bf16_f32(TC_M, TC_N) | (1u << 15) | (1u << 16);
    const uint32_t a0 = tc::smem_addr(smA), b0 = tc::smem_addr(smB);
    const uint32_t a_mn = 128, a_k = (TC_M / 8) * 128, b_mn = 128, b_k = (TC_N / 8) * 128;
    for (int kk = 0; kk < K / 16; ++kk) {
      // each K = 16 step starts two K core matrices further
      const uint64_t ad = swap ? tc::smem_desc(a0 + kk * 2 * a_k, a_k, a_mn) : tc::smem_desc(a0 + kk * 2 * a_k, a_mn, a_k);
      const uint64_t bd = swap ? tc::smem_desc(b0 + kk * 2 * b_k, b_k, b_mn) : tc::smem_desc(b0 + kk * 2 * b_k, b_mn, b_k);
      tc::mma_bf16(taddr, ad, bd, idesc, kk > 0);
    }
    tc::mma_commit(&mbar);
  }
  const bool ok = tc::mbar_wait_block(&mbar, 0, 1u << 24);
  if (!ok) {
    tc::mbar_wait_block(&mbar, 0, 1u << 24);
    if (tid == 0) atomicExch(status, 2);
  }
  tc::fence_after_sync();
  if (ok) {
    float v[32];
    tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16), v);
    const int r = warp * 32 + lane;
    for (int n = 0; n < TC_N; ++n) D[r * TC_N + n] = v[n];
  }
  for (int e = tid; e < TC_M * TC_N; e += 128) {
    const int r = e / TC_N, n = e % TC_N;
    float sum = 0.f;
    for (int k = 0; k < K; ++k) sum += aval(r, k) * bval(n, k);
    Dref[e] = sum;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(taddr, 32);
}

}  // namespace cr

using namespace cr;

extern "C" int cr_tc_selftest_mn(int K, int swap, float* max_abs_err) {
  if (K < 16 || K > TC_KMAX || (K % 16) || !max_abs_err)
    return fail(CR_EINVAL, "cr_tc_selftest_mn: K must be 16, 32, 48 or 64");
  float *D = nullptr, *R = nullptr;
  int* st = nullptr;
  const int smem = TCM_ABUF + TCM_BBUF;
  CR_CUDA(cudaFuncSetAttribute(tc_selftest_mn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  CR_CUDA(cudaMalloc(&D, TC_M * TC_N * sizeof(float)));
  CR_CUDA(cudaMalloc(&R, TC_M * TC_N * sizeof(float)));
  CR_CUDA(cudaMalloc(&st, sizeof(int)));
  CR_CUDA(cudaMemset(st, 0, sizeof(int)));
  CR_CUDA(cudaMemset(D, 0, TC_M * TC_N * sizeof(float)));
  { tc_selftest_mn_kernel<<<1, 128, smem>>>(K, swap ? 1 : 0, D, R, st); count_launch(); }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  float hD[TC_M * TC_N], hR[TC_M * TC_N];
  int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpy(hD, D, sizeof(hD), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hR, R, sizeof(hR), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&hs, st, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(D);
  cudaFree(R);
  cudaFree(st);
  if (e != cudaSuccess) return cuda_fail(e, "cr_tc_selftest_mn");
  if (hs) return fail(CR_ECUDA, "cr_tc_selftest_mn: mbarrier wait gave up");
  float m = 0.f;
  for (int i = 0; i < TC_M * TC_N; ++i) m = fmaxf(m, fabsf(hD[i] - hR[i]));
  *max_abs_err = m;
  return CR_OK;
}

extern "C" int cr_tc_selftest(int K, float* max_abs_err) {
  if (K < 16 || K > TC_KMAX || (K % 16)) return fail(CR_EINVAL, "cr_tc_selftest: K must be 16, 32, 48 or 64");
  float *D = nullptr, *R = nullptr;
  int* st = nullptr;
  CR_CUDA(cudaMalloc(&D, TC_M * TC_N * sizeof(float)));
  CR_CUDA(cudaMalloc(&R, TC_M * TC_N * sizeof(float)));
  CR_CUDA(cudaMalloc(&st, sizeof(int)));
  CR_CUDA(cudaMemset(st, 0, sizeof(int)));
  CR_CUDA(cudaMemset(D, 0, TC_M * TC_N * sizeof(float)));
  { tc_selftest_kernel<<<1, 128>>>(K, D, R, st); count_launch(); }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  float hD[TC_M * TC_N], hR[TC_M * TC_N];
  int hs = 0;
  if (e == cudaSuccess) e = cudaMemcpy(hD, D, sizeof(hD), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hR, R, sizeof(hR), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&hs, st, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(D);
  cudaFree(R);
  cudaFree(st);
  if (e != cudaSuccess) return cuda_fail(e, "cr_tc_selftest");
  if (hs) return fail(CR_ECUDA, "cr_tc_selftest: mbarrier wait gave up");
  float m = 0.f;
  for (int i = 0; i < TC_M * TC_N; ++i) m = fmaxf(m, fabsf(hD[i] - hR[i]));
  *max_abs_err = m;
  return CR_OK;
}
