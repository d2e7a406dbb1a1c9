// FP64 Legendre stages of several right-hand sides at once (Section 2.1,
// Eq. sh-synthesis and its transpose), for the batched solves' FP64 outer
// residual r = b - A x of each right-hand side (iterative refinement).
//
// On this GPU the FP64 pipe runs at 1/64 of the FP32 rate, so these stages
// are bound by FP64 fused multiply-adds and nothing else.  For one
// right-hand side a term (ring pair, l) costs 2 FMAs of recurrence and 2 of
// accumulation; for NR of them the recurrence is evaluated once:
// 2 + 2 NR FMAs, about 2.25 instead of 4 per right-hand side at NR = 8.
//
// Synthesis: one CTA per (m, MR_NT ring pairs), one pair per thread, the
// recurrence Q_l = c_lm z Q_{l-1} - Q_{l-2} of legendre.cu from the pair's
// start (start tables, FP64 state), accumulating the even- and odd-parity
// sums of every right-hand side in registers; the CTA stages s_lm dl_l a_lm
// of its m for all right-hand sides, MR_CH l at a time.
//
// Adjoint: a_lm[r] = s_lm sum_pairs Q_l(z) G_r(pair) as a small dense product
// per chunk of MR_LQ l: each thread first runs its pair's recurrence over the
// chunk into shared memory (zero before the pair's start), then owns one
// output (l, r) and sums over the CTA's MR_NT pairs in a fixed order -- no
// cross-lane reduction, a deterministic result.  One partial row per
// (right-hand side, block of pairs); the finalisation of legendre.cu sums the
// blocks per right-hand side.
#include "common.cuh"
#include "kernels.h"

namespace cr {

constexpr int MR_NT = 128;  // threads = ring pairs per CTA
constexpr int MR_NR = 8;    // right-hand sides per launch
constexpr int MR_CH = 32;   // l per staged chunk of the synthesis

template <int NR>
__global__ void __launch_bounds__(MR_NT) leg_synth_mr_kernel(LegArgs<double> a, const double2* __restrict__ alm,
                                                             int64_t ld_alm, int nr, double2* phase,
                                                             int64_t ld_phase) {
  const int m = blockIdx.y, L = a.L, tid = threadIdx.x;
  const int p = blockIdx.x * MR_NT + tid;
  __shared__ double2 sa[MR_CH][NR];
  __shared__ double sc[MR_CH];
  __shared__ int s_min;
  int ls = L + 1;
  double P1 = 0.0, P2 = 0.0, z = 0.0;
  if (p < a.npairs) {
    const int64_t o = (int64_t)m * a.ld_seed + p;
    z = a.z[p];
    const int l = a.ls[o];
    if (l <= L) {
      const double2 st = a.st[o];
      ls = l;
      P1 = st.x;
      P2 = st.y;
    }
  }
  if (tid == 0) s_min = L + 1;
  __syncthreads();
  if (ls <= L) atomicMin(&s_min, ls);
  __syncthreads();
  const int cmin = s_min;
  double ex[NR], ey[NR], ox[NR], oy[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) ex[r] = ey[r] = ox[r] = oy[r] = 0.0;
  const int64_t offa = lm_off(L, m), offc = lm_off(a.Lc, m);
  // chunks start an even number of l past m: l - m has the parity of i
  const int lbeg = cmin <= L ? m + ((cmin - m) & ~1) : L + 1;
  for (int l0 = lbeg; l0 <= L; l0 += MR_CH) {
    const int nl = min(MR_CH, L - l0 + 1);
    __syncthreads();  // the previous chunk is consumed
    for (int e = tid; e < nl * NR; e += MR_NT) {
      const int i = e / NR, r = e % NR, l = l0 + i;
      double2 v = make_double2(0.0, 0.0);
      if (r < nr) {
        v = alm[r * ld_alm + offa + (l - m)];
        if (m == 0) v.y = 0.0;
        const double f = a.s[offc + (l - m)] * (a.dl ? a.dl[l] : 1.0);
        v.x *= f;
        v.y *= f;
      }
      sa[i][r] = v;
    }
    for (int i = tid; i < nl; i += MR_NT) sc[i] = a.c[offc + (l0 + i - m)];
    __syncthreads();
    for (int i = 0; i < nl; ++i) {
      if (l0 + i < ls) continue;  // before this pair's start
      const double q = fma(sc[i] * z, P1, -P2);
      P2 = P1;
      P1 = q;
      if (i & 1) {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          ox[r] = fma(q, sa[i][r].x, ox[r]);
          oy[r] = fma(q, sa[i][r].y, oy[r]);
        }
      } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          ex[r] = fma(q, sa[i][r].x, ex[r]);
          ey[r] = fma(q, sa[i][r].y, ey[r]);
        }
      }
    }
  }
  if (p < a.npairs) {
    const int rn = p, rs = a.nring - 1 - p;
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nr) {
        phase[r * ld_phase + (int64_t)rn * a.ldp + m] = make_double2(ex[r] + ox[r], ey[r] + oy[r]);
        if (rs != rn) phase[r * ld_phase + (int64_t)rs * a.ldp + m] = make_double2(ex[r] - ox[r], ey[r] - oy[r]);
      }
  }
}

// shared memory of the adjoint: Q [MR_NT][LQ + 1] (rows padded against
// bank conflicts of the recurrence's row-wise writes), G [MR_NT][2][NR]
template <int NR>
__host__ __device__ constexpr int mr_lq() { return MR_NT / NR; }  // l per chunk: one output per thread
template <int NR>
constexpr size_t mr_adj_smem() {
  return (size_t)MR_NT * (mr_lq<NR>() + 1) * sizeof(double) + (size_t)MR_NT * 2 * NR * sizeof(double2);
}

template <int NR>
__global__ void __launch_bounds__(MR_NT) leg_adjoint_mr_kernel(LegArgs<double> a, const double2* __restrict__ phase,
                                                               int64_t ld_phase, int nr, double2* partial, int nblk) {
  constexpr int LQ = mr_lq<NR>();
  extern __shared__ __align__(16) double mr_dyn[];
  double* Qs = mr_dyn;                                                          // [MR_NT][LQ + 1]
  double2* Gs = reinterpret_cast<double2*>(mr_dyn + MR_NT * (LQ + 1));          // [MR_NT][2][NR]
  __shared__ int s_min;
  const int m = blockIdx.y, L = a.L, tid = threadIdx.x, blk = blockIdx.x;
  const int p = blk * MR_NT + tid;
  int ls = L + 1;
  double P1 = 0.0, P2 = 0.0, z = 0.0;
  if (p < a.npairs) {
    const int64_t o = (int64_t)m * a.ld_seed + p;
    z = a.z[p];
    const int l = a.ls[o];
    if (l <= L) {
      const double2 st = a.st[o];
      ls = l;
      P1 = st.x;
      P2 = st.y;
    }
  }
  // this pair's ring phases: even and odd combinations per right-hand side
  {
    const int rn = p, rs = a.nring - 1 - p;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      double2 ge = make_double2(0.0, 0.0), go = ge;
      if (r < nr && p < a.npairs && ls <= L) {
        const double2 gn = phase[r * ld_phase + (int64_t)rn * a.ldp + m];
        const double2 gs = (rs != rn) ? phase[r * ld_phase + (int64_t)rs * a.ldp + m] : make_double2(0.0, 0.0);
        ge = make_double2(gn.x + gs.x, gn.y + gs.y);
        go = make_double2(gn.x - gs.x, gn.y - gs.y);
      }
      Gs[(tid * 2 + 0) * NR + r] = ge;
      Gs[(tid * 2 + 1) * NR + r] = go;
    }
  }
  if (tid == 0) s_min = L + 1;
  __syncthreads();
  if (ls <= L) atomicMin(&s_min, ls);
  __syncthreads();
  const int cmin = s_min;
  const int64_t nlm = n_lm(L);
  const int64_t offa = lm_off(L, m), offc = lm_off(a.Lc, m);
  const int lbeg = cmin <= L ? m + ((cmin - m) & ~1) : L + 1;
  // rows before the block's earliest start are zero
  for (int r = 0; r < nr; ++r)
    for (int l = m + tid; l < lbeg && l <= L; l += MR_NT)
      partial[(int64_t)(r * nblk + blk) * nlm + offa + (l - m)] = make_double2(0.0, 0.0);
  const int oi = tid / NR, orr = tid % NR;  // this thread's output in a chunk: (l0 + oi, right-hand side orr)
  for (int l0 = lbeg; l0 <= L; l0 += LQ) {
    const int nl = min(LQ, L - l0 + 1);
    __syncthreads();  // the previous chunk's Q is consumed
    for (int i = 0; i < nl; ++i) {
      const int l = l0 + i;
      double q = 0.0;
      if (l >= ls) {
        q = fma(a.c[offc + (l - m)] * z, P1, -P2);
        P2 = P1;
        P1 = q;
      }
      Qs[tid * (LQ + 1) + i] = q;
    }
    __syncthreads();
    if (oi < nl && orr < nr) {
      const int par = oi & 1;  // l0 - m is even
      double ax = 0.0, ay = 0.0;
#pragma unroll 4
      for (int k = 0; k < MR_NT; ++k) {
        const double q = Qs[k * (LQ + 1) + oi];
        const double2 g = Gs[(k * 2 + par) * NR + orr];
        ax = fma(q, g.x, ax);
        ay = fma(q, g.y, ay);
      }
      const int l = l0 + oi;
      const double s = a.s[offc + (l - m)];
      partial[(int64_t)(orr * nblk + blk) * nlm + offa + (l - m)] = make_double2(ax * s, ay * s);
    }
  }
}

int mr_blocks(int npairs) { return (npairs + MR_NT - 1) / MR_NT; }

int launch_leg_synth_mr(const LegArgs<double>& a, const double2* alm, int64_t ld_alm, int nr, double2* phase,
                        int64_t ld_phase, cudaStream_t st) {
  if (a.L < 0 || nr <= 0) return CR_OK;
  if (nr > MR_NR) return fail(CR_EINVAL, "FP64 many-RHS synthesis: at most 8 right-hand sides per launch");
  if (a.L + 1 > 65535) return fail(CR_EINVAL, "FP64 many-RHS synthesis: lmax too large for the grid");
  const dim3 grid(mr_blocks(a.npairs), a.L + 1);
  if (nr <= 4) { leg_synth_mr_kernel<4><<<grid, MR_NT, 0, st>>>(a, alm, ld_alm, nr, phase, ld_phase); count_launch(); }
  else { leg_synth_mr_kernel<8><<<grid, MR_NT, 0, st>>>(a, alm, ld_alm, nr, phase, ld_phase); count_launch(); }
  CR_CHECK_LAUNCH("leg_synth_mr_kernel");
  return CR_OK;
}

int launch_leg_adjoint_mr(const LegArgs<double>& a, const double2* phase, int64_t ld_phase, int nr, double2* partial,
                          int* nblk, cudaStream_t st) {
  *nblk = mr_blocks(a.npairs);
  if (a.L < 0 || nr <= 0) return CR_OK;
  if (nr > MR_NR) return fail(CR_EINVAL, "FP64 many-RHS adjoint: at most 8 right-hand sides per launch");
  if (a.L + 1 > 65535) return fail(CR_EINVAL, "FP64 many-RHS adjoint: lmax too large for the grid");
  const dim3 grid(*nblk, a.L + 1);
  if (nr <= 4) {
    CR_CUDA(cudaFuncSetAttribute(leg_adjoint_mr_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)mr_adj_smem<4>()));
    { leg_adjoint_mr_kernel<4><<<grid, MR_NT, mr_adj_smem<4>(), st>>>(a, phase, ld_phase, nr, partial, *nblk); count_launch(); }
  } else {
    CR_CUDA(cudaFuncSetAttribute(leg_adjoint_mr_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)mr_adj_smem<8>()));
    { leg_adjoint_mr_kernel<8><<<grid, MR_NT, mr_adj_smem<8>(), st>>>(a, phase, ld_phase, nr, partial, *nblk); count_launch(); }
  }
  CR_CHECK_LAUNCH("leg_adjoint_mr_kernel");
  return CR_OK;
}

}  // namespace cr
