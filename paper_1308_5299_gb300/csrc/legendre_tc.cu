// Batched Legendre synthesis on the fifth-generation tensor cores.
//
// For many right-hand sides the synthesis Legendre stage is, per m, a dense
// contraction F[pair, rhs] = sum_l P~_lm(z_pair) a_lm[rhs] (Section 2.1,
// Eq. sh-synthesis), split by the parity of l - m into E (even) and O (odd)
// sums so that F(z) = E + O and F(-z) = E - O.  One CTA per (m, 128 ring
// pairs): each thread runs its pair's FP32 recurrence Q_l (start tables,
// polar difference form near the poles as in legendre.cu) and writes Q of
// 64 even and 64 odd l per chunk as BF16 into the A operands (128 x 64,
// K-major); the B operands hold a_lm s_lm (times an optional per-l factor)
// of up to 16 right-hand sides, real and imaginary parts as 32 columns.
// One thread issues tcgen05.mma (M 128, N 32, K 16, FP32 accumulation in
// tensor memory) for both parities; stages are double-buffered on mbarriers
// so the recurrence of the next chunk overlaps the tensor cores.  The
// accumulators are read back with tcgen05.ld at the end.
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace cr {

constexpr int TS_M = 128;     // ring pairs per CTA
constexpr int TS_KC = 32;     // K per chunk and parity (64 l per chunk)
constexpr int TS_N = 32;      // 16 right-hand sides x (re, im)
constexpr int TS_RHS = 16;
constexpr int TS_A_BYTES = TS_M * TS_KC * 2;   // 8 KB
constexpr int TS_B_BYTES = TS_N * TS_KC * 2;   // 2 KB
constexpr int TS_STAGE = 2 * TS_A_BYTES + 2 * TS_B_BYTES;
constexpr uint32_t TS_WAIT = 1u << 26;

struct TsArgs {
  const float2* alm;     // [nrhs][ld_alm] complex64
  int64_t ld_alm;
  float2* phase;         // [nrhs][nring][ldp]
  int64_t ld_phase;      // nring * ldp
  int64_t ldp;
  int L, Lc, nrhs;
  const float *c, *c2, *s, *dl;
  const float *z, *w;
  int npolar;
  const int* ls;
  const float2* st;
  int ld_seed, npairs, nring;
  int* status;
};

template <bool POLAR>
__device__ __forceinline__ float tstep(float c, float c2, float zw, float& s1, float& s2) {
  if (POLAR) {
    const float e = fmaf(-c, zw, c2);
    const float d = fmaf(e, s1, s2);
    const float q = s1 + d;
    s1 = q;
    s2 = d;
    return q;
  }
  const float q = fmaf(c * zw, s1, -s2);
  s2 = s1;
  s1 = q;
  return q;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

template <bool POLAR>
__global__ void __launch_bounds__(TS_M) tc_synth_kernel(TsArgs a, int nbp, int yoff) {
  extern __shared__ __align__(1024) uint8_t tsmem[];
  __shared__ float sc[128], sc2[128], sfac[128];
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t taddr_s;
  __shared__ int s_min;
  // blockIdx.x runs over ring-pair blocks and blockIdx.y over m, so the
  // blocks sharing an m's coefficients run together and share them in L2
  const int m = blockIdx.y;
  const int L = a.L;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int yb = (int)blockIdx.x + yoff;
  const int base = POLAR ? yb * TS_M : a.npolar + (yb - nbp) * TS_M;
  const int pend = POLAR ? a.npolar : a.npairs;
  const int p = base + tid;
  int ls = L + 1;
  float P1 = 0.f, P2 = 0.f, zz = 0.f;
  if (p < pend) {
    const int64_t o = (int64_t)m * a.ld_seed + p;
    zz = POLAR ? a.w[p] : a.z[p];
    const int l = a.ls[o];
    if (l <= L) {
      const float2 s = a.st[o];
      ls = l;
      P1 = s.x;
      P2 = s.y;
    }
  }
  if (tid == 0) s_min = L + 1;
  __syncthreads();
  if (ls <= L) atomicMin(&s_min, ls);
  __syncthreads();
  const int cmin = s_min;
  if (cmin > L) {
    // no pair of the block reaches the threshold: F = 0
    if (p < pend)
      for (int r = 0; r < a.nrhs; ++r) {
        const int rn = p, rs = a.nring - 1 - p;
        a.phase[r * a.ld_phase + (int64_t)rn * a.ldp + m] = make_float2(0.f, 0.f);
        if (rs != rn) a.phase[r * a.ld_phase + (int64_t)rs * a.ldp + m] = make_float2(0.f, 0.f);
      }
    return;
  }
  const int lbeg = m + ((cmin - m) & ~1);
  const int nch = (L + 1 - lbeg + 2 * TS_KC - 1) / (2 * TS_KC);
  const int64_t offa = lm_off(L, m), offc = lm_off(a.Lc, m);
  if (warp == 0) tc::tmem_alloc(&taddr_s, 64);
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_fence_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = taddr_s;
  const uint32_t idesc = tc::idesc_bf16_f32(TS_M, TS_N);
  bool ok = true;
  for (int ch = 0; ch < nch && ok; ++ch) {
    const int stg = ch & 1;
    uint8_t* AE = tsmem + stg * TS_STAGE;
    uint8_t* AO = AE + TS_A_BYTES;
    uint8_t* BE = AO + TS_A_BYTES;
    uint8_t* BO = BE + TS_B_BYTES;
    const int l0 = lbeg + ch * 2 * TS_KC;
    // the MMAs that read this stage two chunks ago must be done
    if (ch >= 2) ok = tc::mbar_wait(&mbar[stg], ((ch - 2) >> 1) & 1, TS_WAIT);
    if (!ok) break;
    {
      const int l = l0 + tid;
      const bool in = l <= L;
      sc[tid] = in ? a.c[offc + (l - m)] : 0.f;
      if (POLAR) sc2[tid] = in ? a.c2[offc + (l - m)] : 0.f;
      sfac[tid] = in ? a.s[offc + (l - m)] * (a.dl ? a.dl[l] : 1.f) : 0.f;
    }
    __syncthreads();
    // B operands: rows 2 r (re) and 2 r + 1 (im), K index k: l = l0 + 2 k
    // (+1 for odd); each task packs 8 K values of both rows of one
    // right-hand side and parity into two 16-byte stores
    for (int e = tid; e < TS_RHS * 2 * (TS_KC / 8); e += TS_M) {
      const int r = e / (2 * (TS_KC / 8)), rem = e % (2 * (TS_KC / 8));
      const int par = rem & 1, k8 = rem >> 1;
      float vr[8], vi[8];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const int j = 2 * (k8 * 8 + kk) + par;  // l - l0
        const int l = l0 + j;
        vr[kk] = 0.f;
        vi[kk] = 0.f;
        if (r < a.nrhs && l <= L) {
          const float2 av = a.alm[r * a.ld_alm + offa + (l - m)];
          vr[kk] = av.x * sfac[j];
          vi[kk] = (m == 0) ? 0.f : av.y * sfac[j];
        }
      }
      uint8_t* B = par ? BO : BE;
      *reinterpret_cast<uint4*>(B + tc::kmajor_offset(2 * r, k8 * 8, TS_KC)) =
          make_uint4(pack_bf16(vr[0], vr[1]), pack_bf16(vr[2], vr[3]), pack_bf16(vr[4], vr[5]), pack_bf16(vr[6], vr[7]));
      *reinterpret_cast<uint4*>(B + tc::kmajor_offset(2 * r + 1, k8 * 8, TS_KC)) =
          make_uint4(pack_bf16(vi[0], vi[1]), pack_bf16(vi[2], vi[3]), pack_bf16(vi[4], vi[5]), pack_bf16(vi[6], vi[7]));
    }
    // A operands: this thread's row, 8 K values (16 l) per 16-byte store;
    // chunks the pair covers entirely run without per-step checks
    const bool full = (ls <= l0) && (l0 + 2 * TS_KC - 1 <= L);
    for (int k8 = 0; k8 < TS_KC / 8; ++k8) {
      float ve[8], vo[8];
      if (full) {
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int j = (k8 * 8 + kk) * 2;
          ve[kk] = tstep<POLAR>(sc[j], POLAR ? sc2[j] : 0.f, zz, P1, P2);
          vo[kk] = tstep<POLAR>(sc[j + 1], POLAR ? sc2[j + 1] : 0.f, zz, P1, P2);
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int j = (k8 * 8 + kk) * 2;
          const int l = l0 + j;
          float q0 = 0.f, q1 = 0.f;
          if (l >= ls && l <= L) q0 = tstep<POLAR>(sc[j], POLAR ? sc2[j] : 0.f, zz, P1, P2);
          if (l + 1 >= ls && l + 1 <= L) q1 = tstep<POLAR>(sc[j + 1], POLAR ? sc2[j + 1] : 0.f, zz, P1, P2);
          ve[kk] = q0;
          vo[kk] = q1;
        }
      }
      const uint4 pe = make_uint4(pack_bf16(ve[0], ve[1]), pack_bf16(ve[2], ve[3]), pack_bf16(ve[4], ve[5]),
                                  pack_bf16(ve[6], ve[7]));
      const uint4 po = make_uint4(pack_bf16(vo[0], vo[1]), pack_bf16(vo[2], vo[3]), pack_bf16(vo[4], vo[5]),
                                  pack_bf16(vo[6], vo[7]));
      *reinterpret_cast<uint4*>(AE + tc::kmajor_offset(tid, k8 * 8, TS_KC)) = pe;
      *reinterpret_cast<uint4*>(AO + tc::kmajor_offset(tid, k8 * 8, TS_KC)) = po;
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t ae = tc::smem_addr(AE), ao = tc::smem_addr(AO), be = tc::smem_addr(BE), bo = tc::smem_addr(BO);
      const uint32_t sbo_a = (TS_KC / 8) * 128, sbo_b = (TS_KC / 8) * 128;
      for (int kk = 0; kk < TS_KC / 16; ++kk) {
        const uint32_t acc = (ch > 0 || kk > 0) ? 1u : 0u;
        tc::mma_bf16(taddr, tc::smem_desc(ae + kk * 256, 128, sbo_a), tc::smem_desc(be + kk * 256, 128, sbo_b), idesc,
                     acc);
        tc::mma_bf16(taddr + TS_N, tc::smem_desc(ao + kk * 256, 128, sbo_a), tc::smem_desc(bo + kk * 256, 128, sbo_b),
                     idesc, acc);
      }
      tc::mma_commit(&mbar[stg]);
    }
    __syncthreads();  // the staged tables are rewritten next chunk
  }
  if (ok) {
    const int cl = nch - 1;
    ok = tc::mbar_wait(&mbar[cl & 1], (cl >> 1) & 1, TS_WAIT);
  }
  tc::fence_after_sync();
  if (ok) {
    float ve[32], vo[32];
    tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16), ve);
    tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + TS_N, vo);
    if (p < pend) {
      const int rn = p, rs = a.nring - 1 - p;
#pragma unroll
      for (int r = 0; r < TS_RHS; ++r) {
        if (r < a.nrhs) {
          const float er = ve[2 * r], ei = ve[2 * r + 1], orr = vo[2 * r], oi = vo[2 * r + 1];
          a.phase[r * a.ld_phase + (int64_t)rn * a.ldp + m] = make_float2(er + orr, ei + oi);
          if (rs != rn) a.phase[r * a.ld_phase + (int64_t)rs * a.ldp + m] = make_float2(er - orr, ei - oi);
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(a.status, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(taddr, 64);
}

// F for nrhs <= 16 right-hand sides of FP32 coefficients into phase
// [nrhs][nring][L+1] (complex64); status: device int set to 1 if a
// completion wait gave up
int launch_tc_synth(const LegArgs<float>& la, const float2* alm, int64_t ld_alm, int nrhs, float2* phase,
                    int* status, cudaStream_t st) {
  if (la.L < 0 || nrhs <= 0) return CR_OK;
  if (nrhs > TS_RHS) return fail(CR_EINVAL, "tensor-core synthesis: at most 16 right-hand sides per launch");
  TsArgs a;
  a.alm = alm;
  a.ld_alm = ld_alm;
  a.phase = phase;
  a.ldp = la.L + 1;
  a.ld_phase = (int64_t)la.nring * a.ldp;
  a.L = la.L;
  a.Lc = la.Lc;
  a.nrhs = nrhs;
  a.c = la.c;
  a.c2 = la.c2;
  a.s = la.s;
  a.dl = la.dl;
  a.z = la.z;
  a.w = la.w;
  a.npolar = la.npolar;
  a.ls = la.ls;
  a.st = la.st;
  a.ld_seed = la.ld_seed;
  a.npairs = la.npairs;
  a.nring = la.nring;
  a.status = status;
  const int nbp = (la.npolar + TS_M - 1) / TS_M;
  const int nbe = (la.npairs - la.npolar + TS_M - 1) / TS_M;
  const size_t smem = 2 * (size_t)TS_STAGE;
  CR_CUDA(cudaFuncSetAttribute(tc_synth_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CR_CUDA(cudaFuncSetAttribute(tc_synth_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (la.L + 1 > 65535) return fail(CR_EINVAL, "tensor-core synthesis: lmax too large for the grid");
  if (nbp) { tc_synth_kernel<true><<<dim3(nbp, la.L + 1), TS_M, smem, st>>>(a, nbp, 0); count_launch(); }
  if (nbe) { tc_synth_kernel<false><<<dim3(nbe, la.L + 1), TS_M, smem, st>>>(a, nbp, nbp); count_launch(); }
  CR_CHECK_LAUNCH("tc_synth_kernel");
  return CR_OK;
}

}  // namespace cr
