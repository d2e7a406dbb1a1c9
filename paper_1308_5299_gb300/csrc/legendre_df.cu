// FP64 Legendre stages evaluated in double-float arithmetic on the FP32 pipes.
//
// GB300 executes FP64 FMAs at 1/64 of the FP32 rate, so the FP64 synthesis
// and adjoint (used by the outer residual of the mixed-precision solve) can
// instead carry every value as an unevaluated sum hi + lo of two floats.
// Sums use Knuth's error-free TwoSum, products Dekker's exact product through
// a fused multiply-add, so each operation is accurate to about 2^-44 relative
// (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2).  Inputs and outputs stay FP64
// (a_lm, the phase array, the adjoint's partial rows); only the arithmetic of
// the recurrence and the accumulation changes.  Each (m, ring pair) starts at
// the FP32 start point (|P~_lm| >= 2^-60) from its FP64 recurrence state, so
// both halves of every value stay normal floats.  Pairs with z > 1/2 use the
// difference form of the recurrence (as the FP32 kernels do): near the poles
// Q changes slowly in l and the standard form would lose the second
// difference to cancellation; c - 2 and w = 1 - z are exact in FP64 there.
// The same work decomposition and reductions as the FP64 kernels
// (legendre.cu), over a polar and an equatorial range of ring pairs.
#include "common.cuh"
#include "kernels.h"

namespace cr {

struct df {
  float hi, lo;
};
struct dfc {
  df x, y;
};

__device__ __forceinline__ df mkdf(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double todbl(df a) { return (double)a.hi + (double)a.lo; }
// |a| >= |b| or a == 0
__device__ __forceinline__ df quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v))};
}
__device__ __forceinline__ df dmul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df dadd(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df dsub(df a, df b) { return dadd(a, {-b.hi, -b.lo}); }
__device__ __forceinline__ dfc cadd(dfc a, dfc b) { return {dadd(a.x, b.x), dadd(a.y, b.y)}; }
// acc += q * a (a complex)
__device__ __forceinline__ dfc cfma(df q, dfc a, dfc acc) { return {dadd(acc.x, dmul(q, a.x)), dadd(acc.y, dmul(q, a.y))}; }

constexpr int DF_NT = 128;
constexpr int DF_RP = 2;  // ring pairs per thread
constexpr int DF_CH = 128;
constexpr int DF_NW = DF_NT / 32;

// standard form Q_l = c z Q_{l-1} - Q_{l-2} on state (Q_{l-1}, Q_{l-2});
// polar form on state (Q_{l-1}, D_{l-1}): D_l = ((c - 2) - c w) Q_{l-1} + D_{l-1},
// Q_l = Q_{l-1} + D_l, with zw = w = 1 - z
template <bool POLAR>
__device__ __forceinline__ df dstep(df c, df c2, df zw, df& s1, df& s2) {
  if (POLAR) {
    const df e = dsub(c2, dmul(c, zw));
    const df d = dadd(dmul(e, s1), s2);
    const df q = dadd(s1, d);
    s1 = q;
    s2 = d;
    return q;
  }
  const df q = dsub(dmul(dmul(c, zw), s1), s2);
  s2 = s1;
  s1 = q;
  return q;
}

// block row yb < nbp covers polar pairs [0, npolar), the rest equatorial pairs
template <bool POLAR>
__device__ __forceinline__ bool df_load_pairs(const LegArgs<double>& a, int m, int yb, int nbp, int warp, int lane,
                                              int p[DF_RP], int ls[DF_RP], df P1[DF_RP], df P2[DF_RP],
                                              df zz[DF_RP], int* wmin, int* wmax) {
  int lo = a.L + 1, hi = m;
  const int base = POLAR ? yb * (DF_NT * DF_RP) : a.npolar_df + (yb - nbp) * (DF_NT * DF_RP);
  const int pend = POLAR ? a.npolar_df : a.npairs;
#pragma unroll
  for (int j = 0; j < DF_RP; ++j) {
    p[j] = base + warp * (32 * DF_RP) + j * 32 + lane;
    ls[j] = a.L + 1;
    P1[j] = {0.f, 0.f};
    P2[j] = {0.f, 0.f};
    zz[j] = {0.f, 0.f};
    if (p[j] < pend) {
      const int64_t o = (int64_t)m * a.ld_seed + p[j];
      const int l = a.ls_df[o];
      const double z = a.z[p[j]];
      zz[j] = POLAR ? mkdf(1.0 - z) : mkdf(z);  // 1 - z is exact for z >= 1/2
      if (l <= a.L) {
        const double2 st = a.st_df[o];
        ls[j] = l;
        P1[j] = mkdf(st.x);
        P2[j] = POLAR ? mkdf(st.x - st.y) : mkdf(st.y);
        lo = min(lo, l);
        hi = max(hi, l);
      }
    }
  }
  *wmin = __reduce_min_sync(0xffffffffu, lo);
  *wmax = __reduce_max_sync(0xffffffffu, hi);
  return *wmin <= a.L;
}

template <bool POLAR>
__global__ void __launch_bounds__(DF_NT) leg_synth_df_kernel(LegArgs<double> a, int nbp, int yoff) {
  const int m = blockIdx.x;
  const int L = a.L;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ dfc sa[DF_CH];
  __shared__ df sc[DF_CH];
  __shared__ df sc2[DF_CH];
  __shared__ int s_min;
  df P1[DF_RP], P2[DF_RP], zz[DF_RP];
  int ls[DF_RP], p[DF_RP];
  dfc accE[DF_RP], accO[DF_RP];
  const int yb = (int)blockIdx.y + yoff;
#pragma unroll
  for (int j = 0; j < DF_RP; ++j) {
    accE[j] = {{0.f, 0.f}, {0.f, 0.f}};
    accO[j] = accE[j];
  }
  int wmin, wmax;
  const bool live = df_load_pairs<POLAR>(a, m, yb, nbp, warp, lane, p, ls, P1, P2, zz, &wmin, &wmax);
  if (tid == 0) s_min = L + 1;
  __syncthreads();
  if (lane == 0 && live) atomicMin(&s_min, wmin);
  __syncthreads();
  const int cmin = s_min;
  const int64_t offa = lm_off(L, m);
  const int64_t offc = lm_off(a.Lc, m);
  const int lbeg = (cmin <= L) ? m + ((cmin - m) & ~7) : L + 1;
  for (int l0 = lbeg; l0 <= L; l0 += DF_CH) {
    const int nl = min(DF_CH, L - l0 + 1);
    __syncthreads();
    for (int i = tid; i < nl; i += DF_NT) {
      const int l = l0 + i;
      double2 v = a.alm[offa + (l - m)];
      if (m == 0) v.y = 0.0;
      double f = a.s[offc + (l - m)];
      if (a.dl) f *= a.dl[l];
      sa[i] = {mkdf(v.x * f), mkdf(v.y * f)};
      const double cc = a.c[offc + (l - m)];
      sc[i] = mkdf(cc);
      if (POLAR) sc2[i] = mkdf(cc - 2.0);  // exact for c in [1, 4]
    }
    __syncthreads();
    if (!live || wmin >= l0 + nl) continue;
    for (int i8 = 0; i8 < nl; i8 += 8) {
      const int lg = l0 + i8;
      const int ng = min(8, nl - i8);
      if (wmin >= lg + ng) continue;
      const bool full = (wmax <= lg && ng == 8);
      for (int u = 0; u < ng; ++u) {
        const int l = lg + u;
        const df c0 = sc[i8 + u];
        const df d0 = POLAR ? sc2[i8 + u] : df{0.f, 0.f};
        const dfc a0 = sa[i8 + u];
#pragma unroll
        for (int j = 0; j < DF_RP; ++j) {
          if (full || l >= ls[j]) {
            const df q = dstep<POLAR>(c0, d0, zz[j], P1[j], P2[j]);
            if (u & 1) accO[j] = cfma(q, a0, accO[j]);
            else accE[j] = cfma(q, a0, accE[j]);
          }
        }
      }
    }
  }
  const int pend = POLAR ? a.npolar_df : a.npairs;
#pragma unroll
  for (int j = 0; j < DF_RP; ++j) {
    if (p[j] < pend) {
      const int rn = p[j], rs = a.nring - 1 - p[j];
      const dfc sN = cadd(accE[j], accO[j]);
      a.phase[(int64_t)rn * a.ldp + m] = make_double2(todbl(sN.x), todbl(sN.y));
      if (rs != rn) {
        const dfc sS = {dsub(accE[j].x, accO[j].x), dsub(accE[j].y, accO[j].y)};
        a.phase[(int64_t)rs * a.ldp + m] = make_double2(todbl(sS.x), todbl(sS.y));
      }
    }
  }
}

__device__ __forceinline__ df shfl_df(df v, int mask) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, mask), __shfl_xor_sync(0xffffffffu, v.lo, mask)};
}
__device__ __forceinline__ dfc shfl_dfc(dfc v, int mask) { return {shfl_df(v.x, mask), shfl_df(v.y, mask)}; }

// transpose reduction of 8 values over the warp: lane l ends with the sum of
// value l >> 2 in v[0]
__device__ __forceinline__ void warp_reduce8_df(dfc v[8]) {
  const int lane = threadIdx.x & 31;
  {
    const bool hi = lane & 16;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const dfc send = hi ? v[i] : v[i + 4];
      const dfc keep = hi ? v[i + 4] : v[i];
      v[i] = cadd(keep, shfl_dfc(send, 16));
    }
  }
  {
    const bool hi = lane & 8;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const dfc send = hi ? v[i] : v[i + 2];
      const dfc keep = hi ? v[i + 2] : v[i];
      v[i] = cadd(keep, shfl_dfc(send, 8));
    }
  }
  {
    const bool hi = lane & 4;
    const dfc send = hi ? v[0] : v[1];
    const dfc keep = hi ? v[1] : v[0];
    v[0] = cadd(keep, shfl_dfc(send, 4));
  }
  v[0] = cadd(v[0], shfl_dfc(v[0], 2));
  v[0] = cadd(v[0], shfl_dfc(v[0], 1));
}

template <bool POLAR>
__global__ void __launch_bounds__(DF_NT) leg_adjoint_df_kernel(LegArgs<double> a, int nbp, int yoff) {
  const int m = blockIdx.x;
  const int L = a.L;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ df sc[DF_CH];
  __shared__ df sc2[DF_CH];
  __shared__ dfc red[DF_NW][DF_CH];  // per-warp sums of the chunk's l
  __shared__ int s_min;
  df P1[DF_RP], P2[DF_RP], zz[DF_RP];
  int ls[DF_RP], p[DF_RP];
  dfc GE[DF_RP], GO[DF_RP];
  const int yb = (int)blockIdx.y + yoff;
  int wmin, wmax;
  const bool live = df_load_pairs<POLAR>(a, m, yb, nbp, warp, lane, p, ls, P1, P2, zz, &wmin, &wmax);
  const int pend = POLAR ? a.npolar_df : a.npairs;
#pragma unroll
  for (int j = 0; j < DF_RP; ++j) {
    GE[j] = {{0.f, 0.f}, {0.f, 0.f}};
    GO[j] = GE[j];
    if (p[j] < pend && ls[j] <= L) {
      const int rn = p[j], rs = a.nring - 1 - p[j];
      const double2 gn = a.phase[(int64_t)rn * a.ldp + m];
      const double2 gs = (rs != rn) ? a.phase[(int64_t)rs * a.ldp + m] : make_double2(0.0, 0.0);
      GE[j] = {mkdf(gn.x + gs.x), mkdf(gn.y + gs.y)};
      GO[j] = {mkdf(gn.x - gs.x), mkdf(gn.y - gs.y)};
    }
  }
  if (tid == 0) s_min = L + 1;
  __syncthreads();
  if (lane == 0 && live) atomicMin(&s_min, wmin);
  __syncthreads();
  const int cmin = s_min;
  const int64_t offa = lm_off(L, m);
  const int64_t offc = lm_off(a.Lc, m);
  double2* part = a.partial + (int64_t)yb * n_lm(L);
  const int lbeg = (cmin <= L) ? m + ((cmin - m) & ~7) : L + 1;
  for (int l = m + tid; l < lbeg; l += DF_NT) part[offa + (l - m)] = make_double2(0.0, 0.0);
  for (int l0 = lbeg; l0 <= L; l0 += DF_CH) {
    const int nl = min(DF_CH, L - l0 + 1);
    __syncthreads();
    for (int i = tid; i < nl; i += DF_NT) {
      const double cc = a.c[offc + (l0 - m) + i];
      sc[i] = mkdf(cc);
      if (POLAR) sc2[i] = mkdf(cc - 2.0);
    }
    __syncthreads();
    for (int i8 = 0; i8 < nl; i8 += 8) {
      const int lg = l0 + i8;
      const int ng = min(8, nl - i8);
      if (!live || wmin >= lg + ng) {
        if (lane < 8) red[warp][i8 + lane] = {{0.f, 0.f}, {0.f, 0.f}};
      } else {
        dfc acc[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] = {{0.f, 0.f}, {0.f, 0.f}};
        const bool full = (wmax <= lg && ng == 8);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (u < ng) {
            const int l = lg + u;
            const df c0 = sc[i8 + u];
            const df d0 = POLAR ? sc2[i8 + u] : df{0.f, 0.f};
#pragma unroll
            for (int j = 0; j < DF_RP; ++j) {
              if (full || l >= ls[j]) {
                const df q = dstep<POLAR>(c0, d0, zz[j], P1[j], P2[j]);
                acc[u] = cfma(q, (u & 1) ? GO[j] : GE[j], acc[u]);
              }
            }
          }
        }
        warp_reduce8_df(acc);
        if ((lane & 3) == 0) red[warp][i8 + (lane >> 2)] = acc[0];
      }
    }
    // one barrier per chunk: the warps' sums in a fixed order
    __syncthreads();
    for (int i = tid; i < nl; i += DF_NT) {
      const int l = l0 + i;
      dfc sum = red[0][i];
#pragma unroll
      for (int w = 1; w < DF_NW; ++w) sum = cadd(sum, red[w][i]);
      const double sc_ = a.s[offc + (l - m)];
      part[offa + (l - m)] = make_double2(todbl(sum.x) * sc_, todbl(sum.y) * sc_);
    }
  }
}

static void df_blocks(int npolar, int npairs, int* nbp, int* nbe) {
  *nbp = (npolar + DF_NT * DF_RP - 1) / (DF_NT * DF_RP);
  *nbe = (npairs - npolar + DF_NT * DF_RP - 1) / (DF_NT * DF_RP);
}

// upper bound on the adjoint's partial rows over both ranges
int df_pair_blocks(int npairs) { return (npairs + DF_NT * DF_RP - 1) / (DF_NT * DF_RP) + 1; }

int launch_leg_synth_df(const LegArgs<double>& a, cudaStream_t st) {
  if (a.L < 0) return CR_OK;
  int nbp, nbe;
  df_blocks(a.npolar_df, a.npairs, &nbp, &nbe);
  if (nbp) { leg_synth_df_kernel<true><<<dim3(a.L + 1, nbp), DF_NT, 0, st>>>(a, nbp, 0); count_launch(); }
  if (nbe) { leg_synth_df_kernel<false><<<dim3(a.L + 1, nbe), DF_NT, 0, st>>>(a, nbp, nbp); count_launch(); }
  CR_CHECK_LAUNCH("leg_synth_df_kernel");
  return CR_OK;
}

int launch_leg_adjoint_df(const LegArgs<double>& a, int* nblk, cudaStream_t st) {
  if (a.L < 0) return CR_OK;
  int nbp, nbe;
  df_blocks(a.npolar_df, a.npairs, &nbp, &nbe);
  if (nbp) { leg_adjoint_df_kernel<true><<<dim3(a.L + 1, nbp), DF_NT, 0, st>>>(a, nbp, 0); count_launch(); }
  if (nbe) { leg_adjoint_df_kernel<false><<<dim3(a.L + 1, nbe), DF_NT, 0, st>>>(a, nbp, nbp); count_launch(); }
  CR_CHECK_LAUNCH("leg_adjoint_df_kernel");
  *nblk = nbp + nbe;
  return CR_OK;
}

}  // namespace cr
