// Batched Legendre synthesis on the fifth-generation tensor cores.
//
// For many right-hand sides the synthesis Legendre stage is, per m, a dense
// contraction F[pair, rhs] = sum_l P~_lm(z_pair) a_lm[rhs] (Section 2.1,
// Eq. sh-synthesis), split by the parity of l - m into E (even) and O (odd)
// sums so that F(z) = E + O and F(-z) = E - O.  The CUDA cores generate the
// A operand -- Q_l of every ring pair by the FP32 recurrence (start tables,
// polar difference form near the poles as in legendre.cu), written as BF16
// K-major rows -- and the B operand, a_lm s_lm (times an optional per-l
// factor) of up to 16 right-hand sides, real and imaginary parts as 32
// columns; tcgen05.mma (M 128, N 32, FP32 accumulation in tensor memory)
// does the contraction, and the accumulators are read back with tcgen05.ld
// at the end.
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace cr {

constexpr int TS_RHS = 16;               // right-hand sides per launch (N = 32: Re, Im)
constexpr uint32_t TS_WAIT = 1u << 26;   // polls of a bounded mbarrier wait

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

// ---------------------------------------------------------------------------
// The work is split so that the CUDA cores never wait for each other:
//  - four producer warps generate the operands; every thread runs the FP32
//    recurrence of two ring pairs (one in each of two 128-row M tiles, two
//    independent dependency chains) and writes their Q rows (BF16, K-major)
//    and one task of the coefficient operand;
//  - a fifth warp issues the MMAs: it waits until all 128 producers have
//    arrived on the stage's "full" mbarrier, issues the stage's MMAs (two
//    tiles x two parities x K/16, D in tensor memory) and commits them to the
//    stage's "empty" mbarrier, which the producers wait on before they reuse
//    the stage NSTG chunks later;
//  - no block-wide barrier inside the chunk loop: the recurrence coefficients
//    are staged per warp.
// SPLIT: each operand value v is carried as hi = bf16(v) and lo = bf16(v - hi)
// and the product as A_hi B_hi + A_hi B_lo + A_lo B_hi (three MMAs on the same
// accumulator), which brings the contraction from the 2^-9 of one BF16
// rounding to about 2^-17 relative.
constexpr int T2_PW = 4;                   // producer warps
constexpr int T2_NT = 32 * (T2_PW + 1);    // + the MMA warp
constexpr int T2_TILES = 2;                // M tiles of 128 ring pairs

template <int KC, bool SPLIT>
struct T2Layout {
  static constexpr int NPART = SPLIT ? 2 : 1;
  static constexpr int A_BYTES = 128 * KC * 2;           // one tile, one parity, one part
  static constexpr int B_BYTES = 32 * KC * 2;            // one parity, one part
  static constexpr int STAGE = T2_TILES * 2 * NPART * A_BYTES + 2 * NPART * B_BYTES;
  __device__ static uint32_t a_off(int t, int q, int part) { return ((t * 2 + q) * NPART + part) * A_BYTES; }
  __device__ static uint32_t b_off(int q, int part) {
    return T2_TILES * 2 * NPART * A_BYTES + (q * NPART + part) * B_BYTES;
  }
};

__device__ __forceinline__ void mbar_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(mbar)) : "memory");
}

// 8 values -> 16 bytes of BF16 (hi part), and the residuals' BF16 (lo part)
__device__ __forceinline__ uint4 pack8_hi(const float v[8]) {
  return make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
}
__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ uint4 pack8_lo(const float v[8]) {
  float r[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) r[i] = v[i] - bf16_round(v[i]);
  return pack8_hi(r);
}

template <bool POLAR, int KC, int NSTG, bool SPLIT>
__global__ void __launch_bounds__(T2_NT) tc_synth2_kernel(TsArgs a, int nbp, int yoff) {
  using Lay = T2Layout<KC, SPLIT>;
  constexpr int CH = 2 * KC;  // l values per chunk
  extern __shared__ __align__(1024) uint8_t t2smem[];
  __shared__ float s_c[T2_PW][CH], s_c2[POLAR ? T2_PW : 1][CH], s_f[T2_PW][CH];
  __shared__ uint64_t full[NSTG], empty[NSTG];
  __shared__ uint32_t taddr_s;
  __shared__ int s_min;
  __shared__ volatile int s_abort;
  const int m = blockIdx.y;
  const int L = a.L;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool producer = warp < T2_PW;
  const int yb = (int)blockIdx.x + yoff;
  const int base = POLAR ? yb * (128 * T2_TILES) : a.npolar + (yb - nbp) * (128 * T2_TILES);
  const int pend = POLAR ? a.npolar : a.npairs;
  // this thread's two ring pairs (tile 0 row tid, tile 1 row tid)
  int pp[T2_TILES], ls[T2_TILES];
  float P1[T2_TILES], P2[T2_TILES], zz[T2_TILES];
#pragma unroll
  for (int t = 0; t < T2_TILES; ++t) {
    pp[t] = base + t * 128 + tid;
    ls[t] = L + 1;
    P1[t] = P2[t] = zz[t] = 0.f;
    if (producer && pp[t] < pend) {
      const int64_t o = (int64_t)m * a.ld_seed + pp[t];
      zz[t] = POLAR ? a.w[pp[t]] : a.z[pp[t]];
      const int l = a.ls[o];
      if (l <= L) {
        const float2 st = a.st[o];
        ls[t] = l;
        P1[t] = st.x;
        P2[t] = st.y;
      }
    }
  }
  if (tid == 0) {
    s_min = L + 1;
    s_abort = 0;
  }
  __syncthreads();
  if (producer) atomicMin(&s_min, min(ls[0], ls[1]));
  __syncthreads();
  const int cmin = s_min;
  if (cmin > L) {
    // no pair of the block reaches the threshold: F = 0
    if (producer)
      for (int t = 0; t < T2_TILES; ++t)
        if (pp[t] < pend)
          for (int r = 0; r < a.nrhs; ++r) {
            const int rn = pp[t], rs = a.nring - 1 - pp[t];
            a.phase[r * a.ld_phase + (int64_t)rn * a.ldp + m] = make_float2(0.f, 0.f);
            if (rs != rn) a.phase[r * a.ld_phase + (int64_t)rs * a.ldp + m] = make_float2(0.f, 0.f);
          }
    return;
  }
  const int lbeg = m + ((cmin - m) & ~1);
  const int nch = (L + 1 - lbeg + CH - 1) / CH;
  const int64_t offa = lm_off(L, m), offc = lm_off(a.Lc, m);
  if (warp == T2_PW) tc::tmem_alloc(&taddr_s, 32 * 2 * T2_TILES);
  if (tid == 0) {
    for (int i = 0; i < NSTG; ++i) {
      tc::mbar_init(&full[i], 32 * T2_PW);
      tc::mbar_init(&empty[i], 1);
    }
    tc::mbar_fence_init();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = taddr_s;
  bool ok = true;

  if (producer) {
    // coefficient-operand task of this thread: right-hand side br, parity
    // bpar, K group bk8 (8 K values of the Re and Im rows)
    constexpr int NTASK = 16 * 2 * (KC / 8);
    const bool btask = tid < NTASK;
    const int br = tid / (2 * (KC / 8)), brem = tid % (2 * (KC / 8));
    const int bpar = brem & 1, bk8 = brem >> 1;
    float2 pa[8];
    auto prefetch = [&](int l0n) {
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const int l = l0n + 2 * (bk8 * 8 + kk) + bpar;
        pa[kk] = (btask && br < a.nrhs && l <= L) ? a.alm[br * a.ld_alm + offa + (l - m)] : make_float2(0.f, 0.f);
      }
    };
    // the recurrence coefficients and factors of the next chunk, loaded into
    // registers one chunk ahead (CH / 32 values per lane and array), so
    // their latency hides behind the current chunk's recurrence
    constexpr int PER = CH / 32;
    float qc[PER], qc2[PER], qf[PER];
    auto prefetch_coef = [&](int l0n) {
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        const int l = l0n + lane + 32 * u;
        const bool in = l <= L;
        qc[u] = in ? a.c[offc + (l - m)] : 0.f;
        qc2[u] = (POLAR && in) ? a.c2[offc + (l - m)] : 0.f;
        qf[u] = in ? a.s[offc + (l - m)] * (a.dl ? a.dl[l] : 1.f) : 0.f;
      }
    };
    prefetch(lbeg);
    prefetch_coef(lbeg);
    float* sc = s_c[warp];
    float* sc2 = s_c2[POLAR ? warp : 0];
    float* sf = s_f[warp];
    for (int ch = 0; ch < nch; ++ch) {
      const int stg = ch % NSTG;
      const int l0 = lbeg + ch * CH;
      if (ch >= NSTG) {
        const bool w = tc::mbar_wait(&empty[stg], ((ch / NSTG) - 1) & 1, TS_WAIT);
        if (!__all_sync(0xffffffffu, w)) {
          if (lane == 0) s_abort = 1;
          ok = false;
          break;
        }
      }
      if (__any_sync(0xffffffffu, s_abort != 0)) {  // warp-uniform
        ok = false;
        break;
      }
      uint8_t* S = t2smem + stg * Lay::STAGE;
      // this warp's copy of the chunk's recurrence coefficients and factors
      __syncwarp();
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        sc[lane + 32 * u] = qc[u];
        if (POLAR) sc2[lane + 32 * u] = qc2[u];
        sf[lane + 32 * u] = qf[u];
      }
      __syncwarp();
      if (ch + 1 < nch) prefetch_coef(l0 + CH);
      if (btask) {
        float vr[8], vi[8];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const int j = 2 * (bk8 * 8 + kk) + bpar;
          vr[kk] = pa[kk].x * sf[j];
          vi[kk] = (m == 0) ? 0.f : pa[kk].y * sf[j];
        }
        const uint32_t orow = tc::kmajor_offset(2 * br, bk8 * 8, KC), irow = tc::kmajor_offset(2 * br + 1, bk8 * 8, KC);
        *reinterpret_cast<uint4*>(S + Lay::b_off(bpar, 0) + orow) = pack8_hi(vr);
        *reinterpret_cast<uint4*>(S + Lay::b_off(bpar, 0) + irow) = pack8_hi(vi);
        if (SPLIT) {
          *reinterpret_cast<uint4*>(S + Lay::b_off(bpar, 1) + orow) = pack8_lo(vr);
          *reinterpret_cast<uint4*>(S + Lay::b_off(bpar, 1) + irow) = pack8_lo(vi);
        }
      }
      if (ch + 1 < nch) prefetch(l0 + CH);
      // A operands: both pairs' recurrences in step (two chains), 8 K values
      // (16 l) per 16-byte store per tile and parity
      const bool full_chunk = (max(ls[0], ls[1]) <= l0) && (l0 + CH - 1 <= L);
#pragma unroll 1
      for (int k8 = 0; k8 < KC / 8; ++k8) {
        float ve[T2_TILES][8], vo[T2_TILES][8];
        if (full_chunk) {
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const int j = (k8 * 8 + kk) * 2;
            const float c0 = sc[j], c1 = sc[j + 1];
            const float d0 = POLAR ? sc2[j] : 0.f, d1 = POLAR ? sc2[j + 1] : 0.f;
#pragma unroll
            for (int t = 0; t < T2_TILES; ++t) {
              ve[t][kk] = tstep<POLAR>(c0, d0, zz[t], P1[t], P2[t]);
              vo[t][kk] = tstep<POLAR>(c1, d1, zz[t], P1[t], P2[t]);
            }
          }
        } else {
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const int j = (k8 * 8 + kk) * 2;
            const int l = l0 + j;
#pragma unroll
            for (int t = 0; t < T2_TILES; ++t) {
              float q0 = 0.f, q1 = 0.f;
              if (l >= ls[t] && l <= L) q0 = tstep<POLAR>(sc[j], POLAR ? sc2[j] : 0.f, zz[t], P1[t], P2[t]);
              if (l + 1 >= ls[t] && l + 1 <= L)
                q1 = tstep<POLAR>(sc[j + 1], POLAR ? sc2[j + 1] : 0.f, zz[t], P1[t], P2[t]);
              ve[t][kk] = q0;
              vo[t][kk] = q1;
            }
          }
        }
        const uint32_t row = tc::kmajor_offset(tid, k8 * 8, KC);
#pragma unroll
        for (int t = 0; t < T2_TILES; ++t) {
          *reinterpret_cast<uint4*>(S + Lay::a_off(t, 0, 0) + row) = pack8_hi(ve[t]);
          *reinterpret_cast<uint4*>(S + Lay::a_off(t, 1, 0) + row) = pack8_hi(vo[t]);
          if (SPLIT) {
            *reinterpret_cast<uint4*>(S + Lay::a_off(t, 0, 1) + row) = pack8_lo(ve[t]);
            *reinterpret_cast<uint4*>(S + Lay::a_off(t, 1, 1) + row) = pack8_lo(vo[t]);
          }
        }
      }
      tc::fence_proxy_async();
      mbar_arrive(&full[stg]);
    }
  } else {
    // the MMA warp: lane 0 issues, the warp waits together
    const uint32_t idesc = tc::idesc_bf16_f32(128, 32);
    const uint32_t sbo_a = (KC / 8) * 128, sbo_b = (KC / 8) * 128;
    int issued = 0;
    for (int ch = 0; ch < nch; ++ch) {
      const int stg = ch % NSTG;
      const bool w = tc::mbar_wait(&full[stg], (ch / NSTG) & 1, TS_WAIT);
      if (!__all_sync(0xffffffffu, w) || __any_sync(0xffffffffu, s_abort != 0)) {
        if (lane == 0) s_abort = 1;
        ok = false;
        break;
      }
      tc::fence_after_sync();
      if (lane == 0) {
        const uint32_t S = tc::smem_addr(t2smem + stg * Lay::STAGE);
#pragma unroll
        for (int t = 0; t < T2_TILES; ++t)
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const uint32_t d = taddr + (uint32_t)((t * 2 + q) * 32);
#pragma unroll
            for (int kk = 0; kk < KC / 16; ++kk) {
              const uint32_t acc = (ch > 0 || kk > 0) ? 1u : 0u;
              const uint64_t ah = tc::smem_desc(S + Lay::a_off(t, q, 0) + kk * 256, 128, sbo_a);
              const uint64_t bh = tc::smem_desc(S + Lay::b_off(q, 0) + kk * 256, 128, sbo_b);
              tc::mma_bf16(d, ah, bh, idesc, acc);
              if (SPLIT) {
                const uint64_t al = tc::smem_desc(S + Lay::a_off(t, q, 1) + kk * 256, 128, sbo_a);
                const uint64_t bl = tc::smem_desc(S + Lay::b_off(q, 1) + kk * 256, 128, sbo_b);
                tc::mma_bf16(d, ah, bl, idesc, 1u);
                tc::mma_bf16(d, al, bh, idesc, 1u);
              }
            }
          }
        tc::mma_commit(&empty[stg]);
      }
      __syncwarp();
      issued = ch + 1;
    }
    // every MMA is complete once the last committed chunk's phase is
    // (commits are cumulative); also after an abort, before tensor memory
    // is read or freed
    if (issued > 0) {
      const int cl = issued - 1;
      const bool w = tc::mbar_wait(&empty[cl % NSTG], (cl / NSTG) & 1, TS_WAIT);
      if (!__all_sync(0xffffffffu, w)) ok = false;
    }
  }
  tc::fence_before_sync();
  ok = __syncthreads_and(ok ? 1 : 0) != 0;
  tc::fence_after_sync();
  if (ok && producer) {
#pragma unroll
    for (int t = 0; t < T2_TILES; ++t) {
      float ve[32], vo[32];
      tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)((t * 2 + 0) * 32), ve);
      tc::tmem_ld32(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)((t * 2 + 1) * 32), vo);
      if (pp[t] < pend) {
        const int rn = pp[t], rs = a.nring - 1 - pp[t];
#pragma unroll
        for (int r = 0; r < TS_RHS; ++r) {
          if (r < a.nrhs) {
            const float er = ve[2 * r], ei = ve[2 * r + 1], orr = vo[2 * r], oi = vo[2 * r + 1];
            a.phase[r * a.ld_phase + (int64_t)rn * a.ldp + m] = make_float2(er + orr, ei + oi);
            if (rs != rn) a.phase[r * a.ld_phase + (int64_t)rs * a.ldp + m] = make_float2(er - orr, ei - oi);
          }
        }
      }
    }
  } else if (!ok && tid == 0) {
    atomicExch(a.status, 1);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == T2_PW) tc::tmem_dealloc(taddr, 32 * 2 * T2_TILES);
}

// F for nrhs <= 16 right-hand sides of FP32 coefficients into phase
// [nrhs][nring][L+1] (complex64); status: device int set to 1 if a
// completion wait gave up
// Shapes of the pipelined synthesis: K per parity per chunk, stages, split
// operands.  Variant 0: K 32, 2 stages (72 KB: three CTAs per SM); 1: K 32,
// 3 stages (108 KB: two CTAs per SM); 2: K 16, 3 stages (54 KB).  With split
// operands K 16 (the stage holds twice the operands).
template <bool POLAR, int KC, int NSTG, bool SPLIT>
static int t2_launch(const TsArgs& a, int nb, int nbp, int yoff, int L, cudaStream_t st) {
  const size_t smem = (size_t)NSTG * T2Layout<KC, SPLIT>::STAGE;
  CR_CUDA(cudaFuncSetAttribute(tc_synth2_kernel<POLAR, KC, NSTG, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem));
  if (nb) { tc_synth2_kernel<POLAR, KC, NSTG, SPLIT><<<dim3(nb, L + 1), T2_NT, smem, st>>>(a, nbp, yoff); count_launch(); }
  return CR_OK;
}

template <int KC, int NSTG, bool SPLIT>
static int t2_launch_both(const TsArgs& a, int nbp, int nbe, int L, cudaStream_t st) {
  int rc = t2_launch<true, KC, NSTG, SPLIT>(a, nbp, nbp, 0, L, st);
  if (!rc) rc = t2_launch<false, KC, NSTG, SPLIT>(a, nbe, nbp, nbp, L, st);
  return rc;
}

int launch_tc_synth(const LegArgs<float>& la, const float2* alm, int64_t ld_alm, int nrhs, float2* phase,
                    int* status, cudaStream_t st) {
  if (la.L < 0 || nrhs <= 0) return CR_OK;
  if (nrhs > TS_RHS) return fail(CR_EINVAL, "tensor-core synthesis: at most 16 right-hand sides per launch");
  if (la.L + 1 > 65535) return fail(CR_EINVAL, "tensor-core synthesis: lmax too large for the grid");
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
  const int per = 128 * T2_TILES;
  const int nbp = (la.npolar + per - 1) / per;
  const int nbe = (la.npairs - la.npolar + per - 1) / per;
  int rc;
  if (la.tc_split) {
    rc = t2_launch_both<16, 3, true>(a, nbp, nbe, la.L, st);
  } else if (la.tc_variant == 1) {
    rc = t2_launch_both<32, 3, false>(a, nbp, nbe, la.L, st);
  } else if (la.tc_variant == 2) {
    rc = t2_launch_both<16, 3, false>(a, nbp, nbe, la.L, st);
  } else {
    rc = t2_launch_both<32, 2, false>(a, nbp, nbe, la.L, st);
  }
  if (rc) return rc;
  CR_CHECK_LAUNCH("tc_synth2_kernel");
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
// which is far from the bound).  Each producer thread runs its pair's FP32
// recurrence (start tables, polar difference form as in legendre.cu).  The
// product is read back from tensor memory per chunk, scaled by s_lm and
// written as one partial row per ring-pair block; a second kernel sums the
// partial rows in a fixed order per right-hand side.

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

// ---------------------------------------------------------------------------
// Warp-specialised batched adjoint: D[l, 64] = Q[l, pairs] G[pairs, 64] per
// chunk of 128 l,
// with the operands in the MN-major layout (each 16-byte row of a core
// matrix is 8 consecutive MN elements of one K index), so that a thread --
// which owns one ring pair, i.e. one K index -- writes 8 consecutive l of
// its pair (A) or 8 consecutive columns of G (B) in one store and no
// shuffle transposition is needed.  Three roles:
//  - warps 0-3 (producers): every thread runs its pair's FP32 recurrence
//    and writes the chunk's A column; chunks go through two shared-memory
//    stages (full / empty mbarriers);
//  - warp 4 (MMA): waits until a stage is full and its accumulator buffer
//    is free, issues the chunk's K = 128 MMAs (M 128, N 64) into one of two
//    tensor-memory accumulators and commits to the stage's "empty" and the
//    accumulator's "full" mbarriers;
//  - warps 5-8 (epilogue): read a finished accumulator (each warp its lane
//    quarter: 32 l rows), release it, and write s_lm times the row's parity
//    half as the partial rows of 16 right-hand sides.
// The chunk loop has no block-wide barrier; every wait is bounded.
// SPLIT: both operands carried as hi = bf16(v) and lo = bf16(v - hi), each in
// its own copy of the layout, and every K step issues hi x hi, hi x lo and
// lo x hi into the same accumulator (the lo x lo term is below FP32 rounding
// of the sum), which brings the products to about 2^-16 relative.
constexpr int T3_M = 128;                  // l per chunk (rows of D)
constexpr int T3_K = 128;                  // ring pairs per CTA
constexpr int T3_N = 64;                   // 16 RHS x (Re, Im) x parity
constexpr int T3_NT = 32 * 9;
constexpr int T3_A_BYTES = T3_M * T3_K * 2;   // 32 KB
constexpr int T3_B_BYTES = T3_N * T3_K * 2;   // 16 KB
constexpr int T3_NSTG = 2;
template <bool SPLIT>
struct T3Layout {
  static constexpr int NPART = SPLIT ? 2 : 1;
  static constexpr int STAGE = NPART * T3_A_BYTES;            // A hi (+ lo) of one stage
  static constexpr int B0 = T3_NSTG * STAGE;                  // B hi (+ lo) after the stages
  static constexpr int BYTES = B0 + NPART * T3_B_BYTES;
};

// MN-major no-swizzle offset of element (mn, k) of an operand with MN rows:
// core matrices 128 bytes apart along MN, (MN / 8) * 128 apart along K (the
// tile self-test cr_tc_selftest_mn checks this layout and which descriptor
// offset carries which stride)
__device__ __forceinline__ uint32_t mn_off(int mn, int k, int MN) {
  return (uint32_t)(((mn >> 3) << 7) + (k >> 3) * (MN / 8) * 128 + ((k & 7) << 4) + ((mn & 7) << 1));
}

template <bool POLAR, bool SPLIT>
__global__ void __launch_bounds__(T3_NT) tc_adjoint2_kernel(TaArgs a, int nbp, int yoff) {
  using Lay = T3Layout<SPLIT>;
  extern __shared__ __align__(1024) uint8_t t3smem[];
  uint8_t* Bsm = t3smem + Lay::B0;
  __shared__ float s_c[4][T3_M], s_c2[POLAR ? 4 : 1][T3_M];
  __shared__ uint64_t a_full[T3_NSTG], a_empty[T3_NSTG], d_full[2], d_free[2];
  __shared__ uint32_t taddr_s;
  __shared__ int s_min;
  __shared__ volatile int s_abort;
  const int m = blockIdx.y;
  const int L = a.L;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int yb = (int)blockIdx.x + yoff;
  const int base = POLAR ? yb * T3_K : a.npolar + (yb - nbp) * T3_K;
  const int pend = POLAR ? a.npolar : a.npairs;
  const bool producer = warp < 4, mma_warp = warp == 4;  // warps 5-8: the epilogue
  const int p = base + tid;  // producers' ring pair
  int ls = L + 1;
  float P1 = 0.f, P2 = 0.f, zz = 0.f;
  if (producer && p < pend) {
    const int64_t o = (int64_t)m * a.ld_seed + p;
    zz = POLAR ? a.w[p] : a.z[p];
    const int l = a.ls[o];
    if (l <= L) {
      const float2 st = a.st[o];
      ls = l;
      P1 = st.x;
      P2 = st.y;
    }
  }
  if (tid == 0) {
    s_min = L + 1;
    s_abort = 0;
  }
  __syncthreads();
  if (producer && ls <= L) atomicMin(&s_min, ls);
  __syncthreads();
  const int cmin = s_min;
  const int64_t offa = lm_off(L, m), offc = lm_off(a.Lc, m);
  const int64_t rstride = (int64_t)a.nblk * a.nlm;
  float2* part = a.partial + (int64_t)yb * a.nlm + offa;
  const int lbeg = (cmin <= L) ? m + ((cmin - m) & ~1) : L + 1;
  // rows before the block's earliest start are zero
  for (int r = 0; r < a.nrhs; ++r)
    for (int l = m + tid; l < lbeg; l += T3_NT) part[r * rstride + (l - m)] = make_float2(0.f, 0.f);
  if (cmin > L) return;
  const int nch = (L + 1 - lbeg + T3_M - 1) / T3_M;

  // B operand (G of this CTA's pairs, all chunks): column n = 2 r (+1 Im)
  // of the even combination, 32 + 2 r (+1) of the odd one; K = the pair
  if (producer) {
    const bool live = p < pend && ls <= L;
    const int rn = p, rs = a.nring - 1 - p;
    float ve[32], vo[32];
#pragma unroll
    for (int r = 0; r < TS_RHS; ++r) {
      float2 gn = make_float2(0.f, 0.f), gs = make_float2(0.f, 0.f);
      if (live && r < a.nrhs) {
        gn = a.phase[r * a.ld_phase + (int64_t)rn * a.ldp + m];
        if (rs != rn) gs = a.phase[r * a.ld_phase + (int64_t)rs * a.ldp + m];
      }
      ve[2 * r] = gn.x + gs.x;
      ve[2 * r + 1] = gn.y + gs.y;
      vo[2 * r] = gn.x - gs.x;
      vo[2 * r + 1] = gn.y - gs.y;
    }
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      *reinterpret_cast<uint4*>(Bsm + mn_off(8 * g, tid, T3_N)) = pack8_hi(ve + 8 * g);
      *reinterpret_cast<uint4*>(Bsm + mn_off(32 + 8 * g, tid, T3_N)) = pack8_hi(vo + 8 * g);
      if (SPLIT) {
        *reinterpret_cast<uint4*>(Bsm + T3_B_BYTES + mn_off(8 * g, tid, T3_N)) = pack8_lo(ve + 8 * g);
        *reinterpret_cast<uint4*>(Bsm + T3_B_BYTES + mn_off(32 + 8 * g, tid, T3_N)) = pack8_lo(vo + 8 * g);
      }
    }
  }
  if (mma_warp) tc::tmem_alloc(&taddr_s, 2 * T3_N);
  if (tid == 0) {
    for (int i = 0; i < T3_NSTG; ++i) {
      tc::mbar_init(&a_full[i], 128);
      tc::mbar_init(&a_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&d_full[i], 1);
      tc::mbar_init(&d_free[i], 128);
    }
    tc::mbar_fence_init();
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = taddr_s;
  bool ok = true;

  if (producer) {
    float* sc = s_c[warp];
    float* sc2 = s_c2[POLAR ? warp : 0];
    float qc[T3_M / 32], qc2[T3_M / 32];
    auto prefetch_coef = [&](int l0n) {
#pragma unroll
      for (int u = 0; u < T3_M / 32; ++u) {
        const int l = l0n + lane + 32 * u;
        const bool in = l <= L;
        qc[u] = in ? a.c[offc + (l - m)] : 0.f;
        qc2[u] = (POLAR && in) ? a.c2[offc + (l - m)] : 0.f;
      }
    };
    prefetch_coef(lbeg);
    for (int ch = 0; ch < nch; ++ch) {
      const int stg = ch % T3_NSTG;
      const int l0 = lbeg + ch * T3_M;
      if (ch >= T3_NSTG) {
        const bool w = tc::mbar_wait(&a_empty[stg], ((ch / T3_NSTG) - 1) & 1, TS_WAIT);
        if (!__all_sync(0xffffffffu, w)) {
          if (lane == 0) s_abort = 1;
          ok = false;
          break;
        }
      }
      if (__any_sync(0xffffffffu, s_abort != 0)) {
        ok = false;
        break;
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < T3_M / 32; ++u) {
        sc[lane + 32 * u] = qc[u];
        if (POLAR) sc2[lane + 32 * u] = qc2[u];
      }
      __syncwarp();
      if (ch + 1 < nch) prefetch_coef(l0 + T3_M);
      uint8_t* A = t3smem + stg * Lay::STAGE;
      const bool full_chunk = (ls <= l0) && (l0 + T3_M - 1 <= L);
#pragma unroll 1
      for (int g = 0; g < T3_M / 8; ++g) {
        float v[8];
        if (full_chunk) {
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
        *reinterpret_cast<uint4*>(A + mn_off(8 * g, tid, T3_M)) = pack8_hi(v);
        if (SPLIT) *reinterpret_cast<uint4*>(A + T3_A_BYTES + mn_off(8 * g, tid, T3_M)) = pack8_lo(v);
      }
      tc::fence_proxy_async();
      mbar_arrive(&a_full[stg]);
    }
  } else if (mma_warp) {
    // D = A B^T with A (M x K) and B (N x K) both MN-major: transpose bits
    const uint32_t idesc = tc::idesc_bf16_f32(T3_M, T3_N) | (1u << 15) | (1u << 16);
    const uint32_t a_kstride = (T3_M / 8) * 128, b_kstride = (T3_N / 8) * 128;
    const uint32_t bb = tc::smem_addr(Bsm);
    int issued = 0;
    for (int ch = 0; ch < nch; ++ch) {
      const int stg = ch % T3_NSTG, db = ch & 1;
      bool w = tc::mbar_wait(&a_full[stg], (ch / T3_NSTG) & 1, TS_WAIT);
      if (w && ch >= 2) w = tc::mbar_wait(&d_free[db], ((ch >> 1) - 1) & 1, TS_WAIT);
      if (!__all_sync(0xffffffffu, w) || __any_sync(0xffffffffu, s_abort != 0)) {
        if (lane == 0) s_abort = 1;
        ok = false;
        break;
      }
      tc::fence_after_sync();
      if (lane == 0) {
        const uint32_t aa = tc::smem_addr(t3smem + stg * Lay::STAGE);
        const uint32_t dt = taddr + (uint32_t)(db * T3_N);
#pragma unroll
        for (int kk = 0; kk < T3_K / 16; ++kk) {
          // MN-major without swizzle: leading byte offset = the K-direction
          // core-matrix stride, stride byte offset = the MN-direction one
          const uint64_t ah = tc::smem_desc(aa + kk * 2 * a_kstride, a_kstride, 128);
          const uint64_t bh = tc::smem_desc(bb + kk * 2 * b_kstride, b_kstride, 128);
          tc::mma_bf16(dt, ah, bh, idesc, kk > 0 ? 1u : 0u);
          if (SPLIT) {
            tc::mma_bf16(dt, ah, tc::smem_desc(bb + T3_B_BYTES + kk * 2 * b_kstride, b_kstride, 128), idesc, 1u);
            tc::mma_bf16(dt, tc::smem_desc(aa + T3_A_BYTES + kk * 2 * a_kstride, a_kstride, 128), bh, idesc, 1u);
          }
        }
        tc::mma_commit(&a_empty[stg]);
        tc::mma_commit(&d_full[db]);
      }
      __syncwarp();
      issued = ch + 1;
    }
    if (issued > 0) {
      const int cl = issued - 1;
      const bool w = tc::mbar_wait(&a_empty[cl % T3_NSTG], (cl / T3_NSTG) & 1, TS_WAIT);
      if (!__all_sync(0xffffffffu, w)) ok = false;
    }
  } else {
    // epilogue: warp 5 + q reads TMEM lanes 32 ((5 + q) % 4) ...
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    for (int ch = 0; ch < nch; ++ch) {
      const int db = ch & 1;
      const bool w = tc::mbar_wait(&d_full[db], (ch >> 1) & 1, TS_WAIT);
      if (!__all_sync(0xffffffffu, w) || __any_sync(0xffffffffu, s_abort != 0)) {
        if (lane == 0) s_abort = 1;
        ok = false;
        break;
      }
      tc::fence_after_sync();
      float ve[32], vo[32];
      tc::tmem_ld32(taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(db * T3_N), ve);
      tc::tmem_ld32(taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(db * T3_N + 32), vo);
      tc::fence_before_sync();
      mbar_arrive(&d_free[db]);
      const int l = lbeg + ch * T3_M + row;
      if (l <= L) {
        const float sl = a.s[offc + (l - m)];
        const bool odd = ((l - m) & 1) != 0;
#pragma unroll
        for (int r = 0; r < TS_RHS; ++r)
          if (r < a.nrhs)
            part[r * rstride + (l - m)] =
                make_float2((odd ? vo[2 * r] : ve[2 * r]) * sl, (odd ? vo[2 * r + 1] : ve[2 * r + 1]) * sl);
      }
    }
  }
  tc::fence_before_sync();
  ok = __syncthreads_and(ok ? 1 : 0) != 0;
  tc::fence_after_sync();
  if (!ok && tid == 0) atomicExch(a.status, 1);
  if (mma_warp) tc::tmem_dealloc(taddr, 2 * T3_N);
}

template <bool SPLIT>
static int t3_launch_both(const TaArgs& a, int nbp, int nbe, int L, cudaStream_t st) {
  const size_t smem = (size_t)T3Layout<SPLIT>::BYTES;
  CR_CUDA(cudaFuncSetAttribute(tc_adjoint2_kernel<true, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CR_CUDA(cudaFuncSetAttribute(tc_adjoint2_kernel<false, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (nbp) { tc_adjoint2_kernel<true, SPLIT><<<dim3(nbp, L + 1), T3_NT, smem, st>>>(a, nbp, 0); count_launch(); }
  if (nbe) { tc_adjoint2_kernel<false, SPLIT><<<dim3(nbe, L + 1), T3_NT, smem, st>>>(a, nbp, nbp); count_launch(); }
  CR_CHECK_LAUNCH("tc_adjoint2_kernel");
  return CR_OK;
}

// G of nrhs <= 16 right-hand sides (phase [nrhs][nring][L+1], complex64) ->
// partial rows [nrhs][nblk][n_lm(L)] (s_lm applied); *nblk receives the
// number of ring-pair blocks.  status: device int set to 1 if a completion
// wait gave up.
int tc_adjoint_blocks(int npolar, int npairs) {
  return (npolar + T3_K - 1) / T3_K + (npairs - npolar + T3_K - 1) / T3_K;
}

int launch_tc_adjoint(const LegArgs<float>& la, const float2* phase, int nrhs, float2* partial, int* nblk,
                      int* status, cudaStream_t st) {
  const int nbp = (la.npolar + T3_K - 1) / T3_K;
  const int nbe = (la.npairs - la.npolar + T3_K - 1) / T3_K;
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
  if (la.tc_split) return t3_launch_both<true>(a, nbp, nbe, la.L, st);
  return t3_launch_both<false>(a, nbp, nbe, la.L, st);
}

}  // namespace cr
