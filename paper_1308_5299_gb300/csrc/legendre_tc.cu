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
__global__ void __launch_bounds__(TS_M, 4) tc_synth_kernel(TsArgs a, int nbp, int yoff) {
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
  // B operands: rows 2 r (re) and 2 r + 1 (im), K index k: l = l0 + 2 k
  // (+1 for odd).  Each thread owns one task -- right-hand side br, parity
  // bpar, K group bk8 (8 K values of both rows, two 16-byte stores) -- and
  // loads the next chunk's coefficients into registers before running the
  // current chunk's recurrence, so their latency hides behind it.
  static_assert(TS_RHS * 2 * (TS_KC / 8) == TS_M, "one B task per thread");
  const int br = tid / (2 * (TS_KC / 8)), brem = tid % (2 * (TS_KC / 8));
  const int bpar = brem & 1, bk8 = brem >> 1;
  float2 pa[8];
  float pc = 0.f, pc2 = 0.f, pf = 0.f;
  auto prefetch = [&](int l0n) {
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const int l = l0n + 2 * (bk8 * 8 + kk) + bpar;
      pa[kk] = (br < a.nrhs && l <= L) ? a.alm[br * a.ld_alm + offa + (l - m)] : make_float2(0.f, 0.f);
    }
    const int l = l0n + tid;
    const bool in = l <= L;
    pc = in ? a.c[offc + (l - m)] : 0.f;
    if (POLAR) pc2 = in ? a.c2[offc + (l - m)] : 0.f;
    pf = in ? a.s[offc + (l - m)] * (a.dl ? a.dl[l] : 1.f) : 0.f;
  };
  prefetch(lbeg);
  bool ok = true;  // block-uniform: every wait below is taken by the whole CTA
  int ncommit = 0;  // chunks whose MMAs have been committed
  for (int ch = 0; ch < nch; ++ch) {
    const int stg = ch & 1;
    uint8_t* AE = tsmem + stg * TS_STAGE;
    uint8_t* AO = AE + TS_A_BYTES;
    uint8_t* BE = AO + TS_A_BYTES;
    uint8_t* BO = BE + TS_B_BYTES;
    const int l0 = lbeg + ch * 2 * TS_KC;
    // the MMAs that read this stage two chunks ago must be done
    if (ch >= 2) ok = tc::mbar_wait_block(&mbar[stg], ((ch - 2) >> 1) & 1, TS_WAIT);
    if (!ok) break;
    sc[tid] = pc;
    if (POLAR) sc2[tid] = pc2;
    sfac[tid] = pf;
    __syncthreads();
    {
      float vr[8], vi[8];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const int j = 2 * (bk8 * 8 + kk) + bpar;  // l - l0
        vr[kk] = pa[kk].x * sfac[j];
        vi[kk] = (m == 0) ? 0.f : pa[kk].y * sfac[j];
      }
      uint8_t* B = bpar ? BO : BE;
      *reinterpret_cast<uint4*>(B + tc::kmajor_offset(2 * br, bk8 * 8, TS_KC)) =
          make_uint4(pack_bf16(vr[0], vr[1]), pack_bf16(vr[2], vr[3]), pack_bf16(vr[4], vr[5]), pack_bf16(vr[6], vr[7]));
      *reinterpret_cast<uint4*>(B + tc::kmajor_offset(2 * br + 1, bk8 * 8, TS_KC)) =
          make_uint4(pack_bf16(vi[0], vi[1]), pack_bf16(vi[2], vi[3]), pack_bf16(vi[4], vi[5]), pack_bf16(vi[6], vi[7]));
    }
    if (ch + 1 < nch) prefetch(l0 + 2 * TS_KC);
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
    ncommit = ch + 1;
    __syncthreads();  // the staged tables are rewritten next chunk
  }
  // Commits are cumulative, so the last committed chunk's phase covers every
  // MMA issued.  This wait also runs after a give-up, so that tensor memory
  // is not freed while an MMA may still write it.
  if (ncommit > 0) {
    const int cl = ncommit - 1;
    if (!tc::mbar_wait_block(&mbar[cl & 1], (cl >> 1) & 1, TS_WAIT)) ok = false;
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


// ---------------------------------------------------------------------------
// Batched adjoint Legendre stage on the tensor cores.
//
// For many right-hand sides the adjoint Legendre stage is, per m, the
// contraction a_lm[rhs] = s_lm sum_pairs Q_l(z_pair) G[pair, rhs] over ring
// pairs, with G = G_m(z) + G_m(-z) for even l - m and G_m(z) - G_m(-z) for
// odd (Section 2.1, Eq. sh-synthesis transposed).  One CTA per (m, 128 ring
// pairs); K runs over the CTA's pairs, so each chunk of 128 l is one
// complete product D[l, 64] = Q[l, pairs] G[pairs, 64] whose 64 columns hold
// the even-parity combination (16 right-hand sides x re, im) and the odd one:
// a row keeps the half of its own parity (the other half costs MMA work only,
// which is far from the bound).  Each thread runs its pair's FP32 recurrence
// (start tables, polar difference form as in legendre.cu); 8 consecutive l of
// 8 neighbouring pairs are transposed with warp shuffles so that every lane
// writes one 16-byte K-major row segment.  G is staged once per CTA the same
// way.  The product is read back from tensor memory after each chunk, scaled
// by s_lm and written as one partial row per ring-pair block; a second
// kernel sums the partial rows in a fixed order per right-hand side.

constexpr int TA_M = 128;    // l per chunk (rows of D)
constexpr int TA_K = 128;    // ring pairs per CTA
constexpr int TA_N = 64;     // 16 right-hand sides x (re, im) x parity
constexpr int TA_A_BYTES = TA_M * TA_K * 2;   // 32 KB
constexpr int TA_B_BYTES = TA_N * TA_K * 2;   // 16 KB

struct TaArgs {
  const float2* phase;   // [nrhs][nring][ldp]
  int64_t ld_phase, ldp;
  float2* partial;       // [nrhs][nblk][nlm]
  int64_t nlm;
  int nblk;
  int L, Lc, nrhs;
  const float *c, *c2, *s;
  const float *z, *w;
  int npolar;
  const int* ls;
  const float2* st;
  int ld_seed, npairs, nring;
  int* status;
};

// 8x8 transpose within each group of 8 lanes: on return lane 8 G + i holds,
// in v[j], the value that lane 8 G + j held in v[i] (three butterfly stages
// that exchange the off-diagonal blocks of halves, quarters and eighths)
__device__ __forceinline__ void transpose8(float v[8], int lane) {
#pragma unroll
  for (int b = 4; b >= 1; b >>= 1) {
    const bool hi = (lane & b) != 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (j & b) continue;
      const float send = hi ? v[j] : v[j | b];
      const float recv = __shfl_xor_sync(0xffffffffu, send, b);
      if (hi) v[j] = recv;
      else v[j | b] = recv;
    }
  }
}

// after transpose8: lane 8 G + i holds row (row0 + i) for the 8 pairs
// kbase + 8 G .. + 7; one 16-byte store of the K-major segment
__device__ __forceinline__ void store_rows8(uint8_t* buf, const float v[8], int row0, int kbase, int lane, int K) {
  *reinterpret_cast<uint4*>(buf + tc::kmajor_offset(row0 + (lane & 7), kbase + 8 * (lane >> 3), K)) =
      make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
}

template <bool POLAR>
__global__ void __launch_bounds__(TA_K) tc_adjoint_kernel(TaArgs a, int nbp, int yoff) {
  extern __shared__ __align__(1024) uint8_t tasmem[];
  uint8_t* A = tasmem;
  uint8_t* B = tasmem + TA_A_BYTES;
  __shared__ float sc[TA_M], sc2[TA_M];
  __shared__ uint64_t mbar;
  __shared__ uint32_t taddr_s;
  __shared__ int s_min;
  const int m = blockIdx.y;
  const int L = a.L;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int yb = (int)blockIdx.x + yoff;
  const int base = POLAR ? yb * TA_K : a.npolar + (yb - nbp) * TA_K;
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
  const int64_t offa = lm_off(L, m), offc = lm_off(a.Lc, m);
  const int64_t rstride = (int64_t)a.nblk * a.nlm;
  float2* part = a.partial + (int64_t)yb * a.nlm + offa;
  const int lbeg = (cmin <= L) ? m + ((cmin - m) & ~1) : L + 1;
  // rows before the block's earliest start are zero
  for (int r = 0; r < a.nrhs; ++r)
    for (int l = m + tid; l < lbeg; l += TA_K) part[r * rstride + (l - m)] = make_float2(0.f, 0.f);
  if (cmin > L) return;

  // B operand: row 2 r / 2 r + 1 = Re / Im of the even combination of
  // right-hand side r, rows 32 + 2 r / + 1 the odd one; K = this thread's pair
  {
    const bool live = p < pend && ls <= L;
    const int rn = p, rs = a.nring - 1 - p;
#pragma unroll 1
    for (int q = 0; q < TS_RHS / 4; ++q) {
      float ve[8], vo[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = 4 * q + i;
        float2 gn = make_float2(0.f, 0.f), gs = make_float2(0.f, 0.f);
        if (live && r < a.nrhs) {
          gn = a.phase[r * a.ld_phase + (int64_t)rn * a.ldp + m];
          if (rs != rn) gs = a.phase[r * a.ld_phase + (int64_t)rs * a.ldp + m];
        }
        ve[2 * i] = gn.x + gs.x;
        ve[2 * i + 1] = gn.y + gs.y;
        vo[2 * i] = gn.x - gs.x;
        vo[2 * i + 1] = gn.y - gs.y;
      }
      transpose8(ve, lane);
      transpose8(vo, lane);
      store_rows8(B, ve, 8 * q, warp * 32, lane, TA_K);
      store_rows8(B, vo, 32 + 8 * q, warp * 32, lane, TA_K);
    }
  }

  if (warp == 0) tc::tmem_alloc(&taddr_s, TA_N);
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::mbar_fence_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = taddr_s;
  const uint32_t idesc = tc::idesc_bf16_f32(TA_M, TA_N);
  const int nch = (L + 1 - lbeg + TA_M - 1) / TA_M;
  bool ok = true;
  for (int ch = 0; ch < nch; ++ch) {
    const int l0 = lbeg + ch * TA_M;
    {
      const int l = l0 + tid;
      const bool in = l <= L;
      sc[tid] = in ? a.c[offc + (l - m)] : 0.f;
      if (POLAR) sc2[tid] = in ? a.c2[offc + (l - m)] : 0.f;
    }
    __syncthreads();
    // A operand: row t = l - l0, K = this thread's pair; 8 l at a time,
    // transposed so that each lane stores 8 pairs of one row
    const bool full = (ls <= l0) && (l0 + TA_M - 1 <= L);
#pragma unroll 1
    for (int g = 0; g < TA_M / 8; ++g) {
      float v[8];
      if (full) {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = tstep<POLAR>(sc[8 * g + j], POLAR ? sc2[8 * g + j] : 0.f, zz, P1, P2);
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int l = l0 + 8 * g + j;
          v[j] = 0.f;
          if (l >= ls && l <= L) v[j] = tstep<POLAR>(sc[8 * g + j], POLAR ? sc2[8 * g + j] : 0.f, zz, P1, P2);
        }
      }
      transpose8(v, lane);
      store_rows8(A, v, 8 * g, warp * 32, lane, TA_K);
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (tid == 0) {
      const uint32_t aa = tc::smem_addr(A), bb = tc::smem_addr(B);
      const uint32_t sbo = (TA_K / 8) * 128;
#pragma unroll
      for (int kk = 0; kk < TA_K / 16; ++kk)
        tc::mma_bf16(taddr, tc::smem_desc(aa + kk * 256, 128, sbo), tc::smem_desc(bb + kk * 256, 128, sbo), idesc,
                     kk > 0 ? 1u : 0u);
      tc::mma_commit(&mbar);
    }
    ok = tc::mbar_wait_block(&mbar, ch & 1, TS_WAIT);
    tc::fence_after_sync();
    if (!ok) {
      // one more bounded wait for the MMAs in flight before tensor memory is
      // freed; the result is reported either way
      tc::mbar_wait_block(&mbar, ch & 1, TS_WAIT);
      if (tid == 0) atomicExch(a.status, 1);
      break;
    }
    {
      float ve[32], vo[32];
      tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16), ve);
      tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + 32, vo);
      const int l = l0 + tid;
      if (l <= L) {
        const float sl = a.s[offc + (l - m)];
        const bool odd = (tid & 1) != 0;  // l0 - m is even
#pragma unroll
        for (int r = 0; r < TS_RHS; ++r)
          if (r < a.nrhs)
            part[r * rstride + (l - m)] =
                make_float2((odd ? vo[2 * r] : ve[2 * r]) * sl, (odd ? vo[2 * r + 1] : ve[2 * r + 1]) * sl);
      }
    }
    // every thread's tensor-memory reads are done before the next MMA
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }
  if (warp == 0) tc::tmem_dealloc(taddr, TA_N);
}

// G of nrhs <= 16 right-hand sides (phase [nrhs][nring][L+1], complex64) ->
// partial rows [nrhs][nblk][n_lm(L)] (s_lm applied); *nblk receives the
// number of ring-pair blocks.  status: device int set to 1 if a completion
// wait gave up.
int tc_adjoint_blocks(int npolar, int npairs) {
  return (npolar + TA_K - 1) / TA_K + (npairs - npolar + TA_K - 1) / TA_K;
}

int launch_tc_adjoint(const LegArgs<float>& la, const float2* phase, int nrhs, float2* partial, int* nblk,
                      int* status, cudaStream_t st) {
  const int nbp = (la.npolar + TA_K - 1) / TA_K;
  const int nbe = (la.npairs - la.npolar + TA_K - 1) / TA_K;
  *nblk = nbp + nbe;
  if (la.L < 0 || nrhs <= 0) return CR_OK;
  if (nrhs > TS_RHS) return fail(CR_EINVAL, "tensor-core adjoint: at most 16 right-hand sides per launch");
  if (la.L + 1 > 65535) return fail(CR_EINVAL, "tensor-core adjoint: lmax too large for the grid");
  TaArgs a;
  a.phase = phase;
  a.ldp = la.L + 1;
  a.ld_phase = (int64_t)la.nring * a.ldp;
  a.partial = partial;
  a.nlm = n_lm(la.L);
  a.nblk = nbp + nbe;
  a.L = la.L;
  a.Lc = la.Lc;
  a.nrhs = nrhs;
  a.c = la.c;
  a.c2 = la.c2;
  a.s = la.s;
  a.z = la.z;
  a.w = la.w;
  a.npolar = la.npolar;
  a.ls = la.ls;
  a.st = la.st;
  a.ld_seed = la.ld_seed;
  a.npairs = la.npairs;
  a.nring = la.nring;
  a.status = status;
  const size_t smem = (size_t)TA_A_BYTES + TA_B_BYTES;
  CR_CUDA(cudaFuncSetAttribute(tc_adjoint_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CR_CUDA(cudaFuncSetAttribute(tc_adjoint_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (nbp) { tc_adjoint_kernel<true><<<dim3(nbp, la.L + 1), TA_K, smem, st>>>(a, nbp, 0); count_launch(); }
  if (nbe) { tc_adjoint_kernel<false><<<dim3(nbe, la.L + 1), TA_K, smem, st>>>(a, nbp, nbp); count_launch(); }
  CR_CHECK_LAUNCH("tc_adjoint_kernel");
  return CR_OK;
}

}  // namespace cr
