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
// both halves of every value stay normal floats.  The same work
// decomposition and reductions as the FP64 kernels (legendre.cu).
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

// Q_l = c z Q_{l-1} - Q_{l-2}
__device__ __forceinline__ df dstep(df c, df z, df& s1, df& s2) {
  const df q = dsub(dmul(dmul(c, z), s1), s2);
  s2 = s1;
  s1 = q;
  return q;
}

__device__ __forceinline__ bool df_load_pairs(const LegArgs<double>& a, int m, int yb, int warp, int lane,
                                              int p[DF_RP], int ls[DF_RP], df P1[DF_RP], df P2[DF_RP],
                                              df zz[DF_RP], int* wmin, int* wmax) {
  int lo = a.L + 1, hi = m;
#pragma unroll
  for (int j = 0; j < DF_RP; ++j) {
    p[j] = yb * (DF_NT * DF_RP) + warp * (32 * DF_RP) + j * 32 + lane;
    ls[j] = a.L + 1;
    P1[j] = {0.f, 0.f};
    P2[j] = {0.f, 0.f};
    zz[j] = {0.f, 0.f};
    if (p[j] < a.npairs) {
      const int64_t o = (int64_t)m * a.ld_seed + p[j];
      const int l = a.ls_df[o];
      zz[j] = mkdf(a.z[p[j]]);
      if (l <= a.L) {
        const double2 st = a.st_df[o];
        ls[j] = l;
        P1[j] = mkdf(st.x);
        P2[j] = mkdf(st.y);
        lo = min(lo, l);
        hi = max(hi, l);
      }
    }
  }
  *wmin = __reduce_min_sync(0xffffffffu, lo);
  *wmax = __reduce_max_sync(0xffffffffu, hi);
  return *wmin <= a.L;
}

__global__ void __launch_bounds__(DF_NT) leg_synth_df_kernel(LegArgs<double> a) {
  const int m = blockIdx.x;
  const int L = a.L;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ dfc sa[DF_CH];
  __shared__ df sc[DF_CH];
  __shared__ int s_min;
  df P1[DF_RP], P2[DF_RP], zz[DF_RP];
  int ls[DF_RP], p[DF_RP];
  dfc accE[DF_RP], accO[DF_RP];
#pragma unroll
  for (int j = 0; j < DF_RP; ++j) {
    accE[j] = {{0.f, 0.f}, {0.f, 0.f}};
    accO[j] = accE[j];
  }
  int wmin, wmax;
  const bool live = df_load_pairs(a, m, blockIdx.y, warp, lane, p, ls, P1, P2, zz, &wmin, &wmax);
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
      sc[i] = mkdf(a.c[offc + (l - m)]);
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
        const dfc a0 = sa[i8 + u];
#pragma unroll
        for (int j = 0; j < DF_RP; ++j) {
          if (full || l >= ls[j]) {
            const df q = dstep(c0, zz[j], P1[j], P2[j]);
            if (u & 1) accO[j] = cfma(q, a0, accO[j]);
            else accE[j] = cfma(q, a0, accE[j]);
          }
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < DF_RP; ++j) {
    if (p[j] < a.npairs) {
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

__global__ void __launch_bounds__(DF_NT) leg_adjoint_df_kernel(LegArgs<double> a) {
  const int m = blockIdx.x;
  const int L = a.L;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ df sc[DF_CH];
  __shared__ dfc sacc[DF_CH];
  __shared__ dfc red[2][DF_NW][8];
  __shared__ int s_min;
  df P1[DF_RP], P2[DF_RP], zz[DF_RP];
  int ls[DF_RP], p[DF_RP];
  dfc GE[DF_RP], GO[DF_RP];
  const int yb = blockIdx.y;
  int wmin, wmax;
  const bool live = df_load_pairs(a, m, yb, warp, lane, p, ls, P1, P2, zz, &wmin, &wmax);
#pragma unroll
  for (int j = 0; j < DF_RP; ++j) {
    GE[j] = {{0.f, 0.f}, {0.f, 0.f}};
    GO[j] = GE[j];
    if (p[j] < a.npairs && ls[j] <= L) {
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
  int rb = 0;
  for (int l0 = lbeg; l0 <= L; l0 += DF_CH) {
    const int nl = min(DF_CH, L - l0 + 1);
    __syncthreads();
    for (int i = tid; i < nl; i += DF_NT) sc[i] = mkdf(a.c[offc + (l0 - m) + i]);
    __syncthreads();
    for (int i8 = 0; i8 < nl; i8 += 8) {
      const int lg = l0 + i8;
      const int ng = min(8, nl - i8);
      if (!live || wmin >= lg + ng) {
        if (lane < 8) red[rb][warp][lane] = {{0.f, 0.f}, {0.f, 0.f}};
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
#pragma unroll
            for (int j = 0; j < DF_RP; ++j) {
              if (full || l >= ls[j]) {
                const df q = dstep(c0, zz[j], P1[j], P2[j]);
                acc[u] = cfma(q, (u & 1) ? GO[j] : GE[j], acc[u]);
              }
            }
          }
        }
        warp_reduce8_df(acc);
        if ((lane & 3) == 0) red[rb][warp][lane >> 2] = acc[0];
      }
      __syncthreads();
      if (tid < 8) {
        dfc s = red[rb][0][tid];
#pragma unroll
        for (int w = 1; w < DF_NW; ++w) s = cadd(s, red[rb][w][tid]);
        sacc[i8 + tid] = s;
      }
      rb ^= 1;
    }
    __syncthreads();
    for (int i = tid; i < nl; i += DF_NT) {
      const int l = l0 + i;
      const double sc_ = a.s[offc + (l - m)];
      part[offa + (l - m)] = make_double2(todbl(sacc[i].x) * sc_, todbl(sacc[i].y) * sc_);
    }
  }
}

int df_pair_blocks(int npairs) { return (npairs + DF_NT * DF_RP - 1) / (DF_NT * DF_RP); }

int launch_leg_synth_df(const LegArgs<double>& a, cudaStream_t st) {
  if (a.L < 0) return CR_OK;
  const int nb = df_pair_blocks(a.npairs);
  { leg_synth_df_kernel<<<dim3(a.L + 1, nb), DF_NT, 0, st>>>(a); count_launch(); }
  CR_CHECK_LAUNCH("leg_synth_df_kernel");
  return CR_OK;
}

int launch_leg_adjoint_df(const LegArgs<double>& a, int* nblk, cudaStream_t st) {
  if (a.L < 0) return CR_OK;
  const int nb = df_pair_blocks(a.npairs);
  { leg_adjoint_df_kernel<<<dim3(a.L + 1, nb), DF_NT, 0, st>>>(a); count_launch(); }
  CR_CHECK_LAUNCH("leg_adjoint_df_kernel");
  *nblk = nb;
  return CR_OK;
}

}  // namespace cr
