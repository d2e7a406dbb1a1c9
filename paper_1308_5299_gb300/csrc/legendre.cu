// Legendre stages of spherical-harmonic synthesis Y and adjoint synthesis Y^T
// (Section 2.1, Eq. sh-synthesis; normalised P~_lm of Section 3.3).
//
// For one m and one north/south ring pair (z, -z):
//   synthesis  F_m(+-z) = sum_{l=m..L} a_lm P~_lm(+-z),
//   adjoint    a_lm    += P~_lm(z) G_m(z) + P~_lm(-z) G_m(-z),
// with P~_lm(-z) = (-1)^(l+m) P~_lm(z), so one recurrence serves both rings
// through even/odd (l-m) accumulators.
//
// P~_lm is generated on the fly in registers by the three-term recurrence in
// the rescaled form Q_l = P~_lm / s_lm,
//   Q_l = c_lm z Q_{l-1} - Q_{l-2},
// where s_lm and c_lm are plan-time tables (s_mm = s_{m+1,m} = 1).  Starting
// from (Q_{m-1}, Q_{m-2}) = (0, -P~_mm) makes the first step return the seed,
// so the loop is uniform from l = m.  a_lm is multiplied by s_lm when staged
// (synthesis) and the adjoint result by s_lm when written.
//
// Each (m, ring pair) starts where |P~_lm| first reaches a threshold tau
// (2^-60 for the transforms of both precisions, with the FP64 state there
// for the FP64 kernels; 2^-100 for the squared sums of the smoother's
// diagonal): the plan-time start tables hold
// that l and the recurrence state there, computed once from the seed
// P~_mm in scaled FP64 (build_start_tables).  Terms with |P~_lm| < tau are
// dropped: below FP32 rounding by ten orders of magnitude and below FP64
// rounding by two, and decaying geometrically away from the start, so their
// sum stays under the rounding of either sum.  Before its start a pair neither steps nor
// accumulates; pairs that never reach tau within the band limit hold a zero
// state.  Each warp classifies every group of 8 l as idle (no pair started
// yet), full (every live pair started: the unchecked loop) or ramp (per-pair
// start test), so the region below the turning point where the functions are
// negligible costs nothing.
//
// Work decomposition: one CTA per (m, block of LEG_NT*RP ring pairs) with
// the ring-pair blocks of one m adjacent in launch order (blockIdx.x) and m
// in blockIdx.y, so the longest CTAs (small m) are dispatched first, the
// short ones (m near L) last, and the CTAs of one m share its coefficients
// in L2; RP
// (2, 4 or 8 pairs per thread: the ring-block size) chosen per grid, band
// limit and precision by the plan's autotuner (default 4);
// each warp owns 32*RP consecutive pairs (lane + 32 j), so its pairs'
// start points are close.  The a_lm of the CTA's m (synthesis) and the
// recurrence coefficients are staged through shared memory in chunks of
// LEG_CH l-values from the CTA's earliest start.  The adjoint reduces over
// ring pairs with a warp-shuffle transpose reduction over 8 consecutive l
// (each lane ends with one l) into per-warp rows of shared memory, one
// fixed-order cross-warp sum per chunk of LEG_CH l (a single barrier per
// chunk), and one partial row per ring block summed in a second,
// deterministic kernel.
#include "common.cuh"
#include "kernels.h"

namespace cr {

constexpr int LEG_NT = 128;
constexpr int LEG_RP = 4;      // default ring pairs per thread
constexpr int LEG_RP_MIN = 2;  // smallest choice of the autotuner
constexpr int LEG_CH = 256;
constexpr int LEG_NW = LEG_NT / 32;
// The packed FP32 kernels run one warp per CTA: warps never wait for each
// other (no block barrier; the adjoint writes one partial row per warp), and
// a warp that finishes early frees its SM slot at once.
constexpr int L32_NT = 32;

// One recurrence step Q_l = c z Q_{l-1} - Q_{l-2}; returns Q_l and advances
// the state (s1, s2).
//  - standard form: state (Q_{l-1}, Q_{l-2});
//  - polar form (FP32 pairs with z > 1/2): state (Q_{l-1}, D_{l-1}) with the
//    difference D_l = Q_l - Q_{l-1} = ((c - 2) - c w) Q_{l-1} + D_{l-1},
//    w = 1 - z.  Near the poles Q changes slowly in l and the standard form
//    loses the small second difference to cancellation (in FP32 1 - z itself
//    rounds away); carrying D with c - 2 and w at full relative precision
//    keeps it.
template <typename T, bool POLAR>
__device__ __forceinline__ T rstep(T c, T c2, T zw, T& s1, T& s2) {
  if (POLAR) {
    const T e = fma(-c, zw, c2);
    const T d = fma(e, s1, s2);
    const T q = s1 + d;
    s1 = q;
    s2 = d;
    return q;
  }
  const T q = fma(c * zw, s1, -s2);
  s2 = s1;
  s1 = q;
  return q;
}

// Ring pairs are split into a polar range [0, npolar) and an equatorial
// range [npolar, npairs); each CTA covers LEG_NT*RP pairs of one range.
// Block row yb (= blockIdx.x + the launch's row offset) < nbp is polar.
template <int RP, int NT = LEG_NT>
__device__ __forceinline__ int pair_of(int npolar, int nbp, int yb, int warp, int lane, int j) {
  const int base = yb < nbp ? yb * (NT * RP) : npolar + (yb - nbp) * (NT * RP);
  return base + warp * (32 * RP) + j * 32 + lane;
}

// Per-thread pair setup shared by both kernels: start point, state, and the
// warp's earliest / latest start over its live pairs (a pair is live when it
// starts at or below L).  Returns false when the warp has no live pair.
template <typename T, bool POLAR, int RP, int NT = LEG_NT>
__device__ __forceinline__ bool load_pairs(const LegArgs<T>& a, int m, int yb, int nbp, int warp, int lane,
                                           int p[RP], int ls[RP], T P1[RP], T P2[RP], T zz[RP], int* wmin,
                                           int* wmax) {
  using C = typename Tr<T>::C;
  const int pend = POLAR ? a.npolar : a.npairs;
  int lo = a.L + 1, hi = m;
#pragma unroll
  for (int j = 0; j < RP; ++j) {
    p[j] = pair_of<RP, NT>(a.npolar, nbp, yb, warp, lane, j);
    ls[j] = a.L + 1;
    P1[j] = 0;
    P2[j] = 0;
    zz[j] = 0;
    if (p[j] < pend) {
      const int64_t o = (int64_t)m * a.ld_seed + p[j];
      const int l = a.ls[o];
      zz[j] = POLAR ? a.w[p[j]] : a.z[p[j]];
      if (l <= a.L) {
        const C st = a.st[o];
        ls[j] = l;
        P1[j] = st.x;
        P2[j] = st.y;
        lo = min(lo, l);
        hi = max(hi, l);
      }
    }
  }
  *wmin = __reduce_min_sync(0xffffffffu, lo);
  *wmax = __reduce_max_sync(0xffffffffu, hi);
  return *wmin <= a.L;
}

template <typename T, bool POLAR, int RP, int MT = 1>
__global__ void __launch_bounds__(LEG_NT) leg_synth_kernel(LegArgs<T> a, int nbp, int yoff) {
  using C = typename Tr<T>::C;
  // m tile: this CTA takes m = blockIdx.y and, with MT = 2, then
  // m = L - blockIdx.y, so that every CTA has about the same l range
#pragma unroll 1
  for (int mi = 0; mi < MT; ++mi) {
    const int m = mi == 0 ? (int)blockIdx.y : a.L - (int)blockIdx.y;
    if (mi > 0 && m <= (int)blockIdx.y) break;
    if (mi > 0) __syncthreads();  // the shared buffers of the previous m are free
    const int L = a.L;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    // each warp stages its own chunks (no block-wide barrier in the loop)
    __shared__ C sa_all[LEG_NW][LEG_CH];
    __shared__ T sc_all[LEG_NW][LEG_CH];
    __shared__ T sc2_all[POLAR ? LEG_NW : 1][LEG_CH];
    C* sa = sa_all[warp];
    T* sc = sc_all[warp];
    T* sc2 = sc2_all[POLAR ? warp : 0];

    T P1[RP], P2[RP], zz[RP];
    int ls[RP], p[RP];
    C accE[RP], accO[RP];
#pragma unroll
    for (int j = 0; j < RP; ++j) {
      accE[j] = mk((T)0, (T)0);
      accO[j] = mk((T)0, (T)0);
    }
    const int yb = (int)blockIdx.x + yoff;
    int wmin, wmax;
    const bool live = load_pairs<T, POLAR, RP>(a, m, yb, nbp, warp, lane, p, ls, P1, P2, zz, &wmin, &wmax);
    const int64_t offa = lm_off(L, m);
    const int64_t offc = lm_off(a.Lc, m);

    // chunks start at an offset from m that is a multiple of 8, so l - m and
    // the group index agree in parity; a warp starts at its earliest pair
    const int lbeg = live ? m + ((wmin - m) & ~7) : L + 1;
    for (int l0 = lbeg; l0 <= L; l0 += LEG_CH) {
      const int nl = min(LEG_CH, L - l0 + 1);
      __syncwarp();
      for (int i = lane; i < nl; i += 32) {
        const int l = l0 + i;
        C v = a.alm[offa + (l - m)];
        if (m == 0) v.y = 0;
        T f = a.s[offc + (l - m)];
        if (a.dl) f *= a.dl[l];
        sa[i] = cscale(v, f);
        sc[i] = a.c[offc + (l - m)];
        if (POLAR) sc2[i] = a.c2[offc + (l - m)];
      }
      __syncwarp();
      for (int i8 = 0; i8 < nl; i8 += 8) {
        const int lg = l0 + i8;
        const int ng = min(8, nl - i8);
        if (wmin >= lg + ng) continue;  // no pair of the warp has started
        if (wmax <= lg && ng == 8) {
#pragma unroll
          for (int u = 0; u < 8; u += 2) {
            const T c0 = sc[i8 + u], c1 = sc[i8 + u + 1];
            const T d0 = POLAR ? sc2[i8 + u] : (T)0, d1 = POLAR ? sc2[i8 + u + 1] : (T)0;
            const C a0 = sa[i8 + u], a1 = sa[i8 + u + 1];
#pragma unroll
            for (int j = 0; j < RP; ++j) {
              const T q0 = rstep<T, POLAR>(c0, d0, zz[j], P1[j], P2[j]);
              const T q1 = rstep<T, POLAR>(c1, d1, zz[j], P1[j], P2[j]);
              accE[j].x = fma(q0, a0.x, accE[j].x);
              accE[j].y = fma(q0, a0.y, accE[j].y);
              accO[j].x = fma(q1, a1.x, accO[j].x);
              accO[j].y = fma(q1, a1.y, accO[j].y);
            }
          }
        } else {
          for (int u = 0; u < ng; ++u) {
            const int l = lg + u;
            const T c0 = sc[i8 + u];
            const T d0 = POLAR ? sc2[i8 + u] : (T)0;
            const C a0 = sa[i8 + u];
#pragma unroll
            for (int j = 0; j < RP; ++j) {
              if (l >= ls[j]) {
                const T q0 = rstep<T, POLAR>(c0, d0, zz[j], P1[j], P2[j]);
                if (u & 1) {
                  accO[j].x = fma(q0, a0.x, accO[j].x);
                  accO[j].y = fma(q0, a0.y, accO[j].y);
                } else {
                  accE[j].x = fma(q0, a0.x, accE[j].x);
                  accE[j].y = fma(q0, a0.y, accE[j].y);
                }
              }
            }
          }
        }
      }
    }
    const int pend = POLAR ? a.npolar : a.npairs;
#pragma unroll
    for (int j = 0; j < RP; ++j) {
      if (p[j] < pend) {
        const int rn = p[j], rs = a.nring - 1 - p[j];
        a.phase[(int64_t)rn * a.ldp + m] = cadd(accE[j], accO[j]);
        if (rs != rn) a.phase[(int64_t)rs * a.ldp + m] = csub(accE[j], accO[j]);
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ T shfl_x(T v, int mask) {
  return __shfl_xor_sync(0xffffffffu, v, mask);
}

// Transpose reduction of 8 complex values over the 32 lanes of a warp: on
// return lane l holds in v[0] the warp sum of the value with index l >> 2.
template <typename C>
__device__ __forceinline__ void warp_reduce8(C v[8]) {
  const int lane = threadIdx.x & 31;
  {
    const bool hi = lane & 16;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      C send = hi ? v[i] : v[i + 4];
      C keep = hi ? v[i + 4] : v[i];
      send.x = shfl_x(send.x, 16);
      send.y = shfl_x(send.y, 16);
      v[i] = cadd(keep, send);
    }
  }
  {
    const bool hi = lane & 8;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      C send = hi ? v[i] : v[i + 2];
      C keep = hi ? v[i + 2] : v[i];
      send.x = shfl_x(send.x, 8);
      send.y = shfl_x(send.y, 8);
      v[i] = cadd(keep, send);
    }
  }
  {
    const bool hi = lane & 4;
    C send = hi ? v[0] : v[1];
    C keep = hi ? v[1] : v[0];
    send.x = shfl_x(send.x, 4);
    send.y = shfl_x(send.y, 4);
    v[0] = cadd(keep, send);
  }
  v[0].x += shfl_x(v[0].x, 2);
  v[0].y += shfl_x(v[0].y, 2);
  v[0].x += shfl_x(v[0].x, 1);
  v[0].y += shfl_x(v[0].y, 1);
}

// ---------------------------------------------------------------------------
// FP32 synthesis with packed pairs of FP32 lanes (f32x2 instructions of the
// sm_100 family: two FP32 operations per issued instruction).  Inside the
// unrolled 8-l group two ring pairs step together: one packed multiply and
// one packed FMA for the recurrence, two packed FMAs for the complex
// accumulators.  The minus sign of the three-term recurrence is folded into
// a fixed sign pattern: with V_l = sigma_l Q_l, sigma = (+, +, -, -) by
// (l - m) mod 4, the recurrence becomes V_l = alpha_l z V_{l-1} + V_{l-2},
// alpha_l = sigma_l sigma_{l-1} c_lm (-c, +c, -c, +c by (l - m) mod 4), and
// the staged coefficient carries sigma_l, so sum_l V_l (sigma_l a_lm) =
// sum_l Q_l a_lm.  The polar difference form needs no sign change.  Staged
// values are stored as (v, v) pairs so a 64-bit shared load yields the
// broadcast operand.
typedef unsigned long long u64;
__device__ __forceinline__ u64 pk2(float a, float b) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(u64 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 lds2(const float2* p) { return *reinterpret_cast<const u64*>(p); }

// The same reduction through shared memory, one warp's buffer of 8 rows.
// Each lane has stored its value u in buf[u][lane] as soon as it was complete
// (so no array of 8 sums stays live in registers); here lane l sums the
// entries k, k + 4, ..., k + 28 (k = l & 3) of row l >> 2 and two shuffle
// steps add the four residues.  Rows are SMEM_RS = 36 entries apart: a
// half-warp's 64-bit reads then fall on 16 distinct 8-byte bank pairs
// (4 u + k mod 16), and the row-wise writes are contiguous, so every access
// takes the two wavefronts of a 64-bit warp access.  The real and imaginary
// parts are added by one packed f32x2 add per entry.  About 30 instructions
// instead of the 64 of the shuffle transpose.
constexpr int SMEM_RS = 36;
__device__ __forceinline__ float2 smem_rows8_sum(float2 (*buf)[SMEM_RS]) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  const int u = lane >> 2, k = lane & 3;
  u64 acc = lds2(&buf[u][k]);
#pragma unroll
  for (int i = 1; i < 8; ++i) acc = add2(acc, lds2(&buf[u][k + 4 * i]));
  float2 s;
  upk2(acc, s.x, s.y);
  s.x += shfl_x(s.x, 1);
  s.y += shfl_x(s.y, 1);
  s.x += shfl_x(s.x, 2);
  s.y += shfl_x(s.y, 2);
  __syncwarp();  // the buffer is rewritten by the next group
  return s;
}

template <bool POLAR, int RP, int MT = 1>
__global__ void __launch_bounds__(L32_NT) leg_synth_f32x2_kernel(LegArgs<float> a, int nbp, int yoff) {
  static_assert(RP % 2 == 0, "pairs per thread must be even");
  constexpr int NP = RP / 2;
  // m tile: this CTA takes m = blockIdx.y and, with MT = 2, then
  // m = L - blockIdx.y, so that every CTA has about the same l range
#pragma unroll 1
  for (int mi = 0; mi < MT; ++mi) {
    const int m = mi == 0 ? (int)blockIdx.y : a.L - (int)blockIdx.y;
    if (mi > 0 && m <= (int)blockIdx.y) break;
    if (mi > 0) __syncwarp();  // the shared buffers of the previous m are free
    const int L = a.L;
    const int lane = threadIdx.x;
    const int warp = 0;
    __shared__ float2 sax[LEG_CH], say[LEG_CH], sk[LEG_CH];
    __shared__ float2 sk2[POLAR ? LEG_CH : 1];

    float P1[RP], P2[RP], zz[RP];
    int ls[RP], p[RP];
    float ex[RP], ey[RP], ox[RP], oy[RP];
#pragma unroll
    for (int j = 0; j < RP; ++j) ex[j] = ey[j] = ox[j] = oy[j] = 0.f;
    const int yb = (int)blockIdx.x + yoff;
    int wmin, wmax;
    const bool live = load_pairs<float, POLAR, RP, L32_NT>(a, m, yb, nbp, warp, lane, p, ls, P1, P2, zz, &wmin, &wmax);
    auto sgn = [&](int l) -> float { return ((l - m) & 2) ? -1.f : 1.f; };
    if (!POLAR) {
#pragma unroll
      for (int j = 0; j < RP; ++j)
        if (ls[j] <= L) {
          P1[j] *= sgn(ls[j] - 1);
          P2[j] *= sgn(ls[j] - 2);
        }
    }
    const int64_t offa = lm_off(L, m);
    const int64_t offc = lm_off(a.Lc, m);
    const int lbeg = live ? m + ((wmin - m) & ~7) : L + 1;
    for (int l0 = lbeg; l0 <= L; l0 += LEG_CH) {
      const int nl = min(LEG_CH, L - l0 + 1);
      __syncwarp();
      for (int i = lane; i < nl; i += 32) {
        const int l = l0 + i;
        float2 v = a.alm[offa + (l - m)];
        if (m == 0) v.y = 0.f;
        float f = a.s[offc + (l - m)];
        if (a.dl) f *= a.dl[l];
        const float c = a.c[offc + (l - m)];
        if (POLAR) {
          sax[i] = make_float2(v.x * f, v.x * f);
          say[i] = make_float2(v.y * f, v.y * f);
          sk[i] = make_float2(-c, -c);
          const float c2 = a.c2[offc + (l - m)];
          sk2[i] = make_float2(c2, c2);
        } else {
          const float g = f * sgn(l);
          const float al = ((l - m) & 1) ? c : -c;
          sax[i] = make_float2(v.x * g, v.x * g);
          say[i] = make_float2(v.y * g, v.y * g);
          sk[i] = make_float2(al, al);
        }
      }
      __syncwarp();
      for (int i8 = 0; i8 < nl; i8 += 8) {
        const int lg = l0 + i8;
        const int ng = min(8, nl - i8);
        if (wmin >= lg + ng) continue;  // no pair of the warp has started
        if (wmax <= lg && ng == 8) {
          u64 Z[NP], S1[NP], S2[NP], EX[NP], EY[NP], OX[NP], OY[NP];
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            Z[q] = pk2(zz[2 * q], zz[2 * q + 1]);
            S1[q] = pk2(P1[2 * q], P1[2 * q + 1]);
            S2[q] = pk2(P2[2 * q], P2[2 * q + 1]);
            EX[q] = pk2(ex[2 * q], ex[2 * q + 1]);
            EY[q] = pk2(ey[2 * q], ey[2 * q + 1]);
            OX[q] = pk2(ox[2 * q], ox[2 * q + 1]);
            OY[q] = pk2(oy[2 * q], oy[2 * q + 1]);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const u64 K = lds2(&sk[i8 + u]);
            const u64 K2 = POLAR ? lds2(&sk2[i8 + u]) : 0ull;
            const u64 AX = lds2(&sax[i8 + u]), AY = lds2(&say[i8 + u]);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
              u64 Q;
              if (POLAR) {
                const u64 E = fma2(K, Z[q], K2);
                const u64 D = fma2(E, S1[q], S2[q]);
                Q = add2(S1[q], D);
                S2[q] = D;
              } else {
                Q = fma2(mul2(K, Z[q]), S1[q], S2[q]);
                S2[q] = S1[q];
              }
              S1[q] = Q;
              if (u & 1) {
                OX[q] = fma2(Q, AX, OX[q]);
                OY[q] = fma2(Q, AY, OY[q]);
              } else {
                EX[q] = fma2(Q, AX, EX[q]);
                EY[q] = fma2(Q, AY, EY[q]);
              }
            }
          }
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            upk2(S1[q], P1[2 * q], P1[2 * q + 1]);
            upk2(S2[q], P2[2 * q], P2[2 * q + 1]);
            upk2(EX[q], ex[2 * q], ex[2 * q + 1]);
            upk2(EY[q], ey[2 * q], ey[2 * q + 1]);
            upk2(OX[q], ox[2 * q], ox[2 * q + 1]);
            upk2(OY[q], oy[2 * q], oy[2 * q + 1]);
          }
        } else {
          for (int u = 0; u < ng; ++u) {
            const int l = lg + u;
            const float K = sk[i8 + u].x;
            const float K2 = POLAR ? sk2[i8 + u].x : 0.f;
            const float ax = sax[i8 + u].x, ay = say[i8 + u].x;
#pragma unroll
            for (int j = 0; j < RP; ++j) {
              if (l >= ls[j]) {
                float q;
                if (POLAR) {
                  const float e = fmaf(K, zz[j], K2);
                  const float d = fmaf(e, P1[j], P2[j]);
                  q = P1[j] + d;
                  P2[j] = d;
                } else {
                  q = fmaf(K * zz[j], P1[j], P2[j]);
                  P2[j] = P1[j];
                }
                P1[j] = q;
                if (u & 1) {
                  ox[j] = fmaf(q, ax, ox[j]);
                  oy[j] = fmaf(q, ay, oy[j]);
                } else {
                  ex[j] = fmaf(q, ax, ex[j]);
                  ey[j] = fmaf(q, ay, ey[j]);
                }
              }
            }
          }
        }
      }
    }
    const int pend = POLAR ? a.npolar : a.npairs;
#pragma unroll
    for (int j = 0; j < RP; ++j) {
      if (p[j] < pend) {
        const int rn = p[j], rs = a.nring - 1 - p[j];
        a.phase[(int64_t)rn * a.ldp + m] = make_float2(ex[j] + ox[j], ey[j] + oy[j]);
        if (rs != rn) a.phase[(int64_t)rs * a.ldp + m] = make_float2(ex[j] - ox[j], ey[j] - oy[j]);
      }
    }
  }
}

// SQ: accumulate P~^2 times a per-ring value (ringval) instead of P~ times
// the ring's phase G_m: sum_k P~_lm(z_k)^2 v_k, used for the diagonal of
// Y^T N^-1 Y (the Delta m = 0 term of the ring formula).
template <typename T, bool POLAR, int RP, bool SQ = false, int MT = 1>
__global__ void __launch_bounds__(LEG_NT) leg_adjoint_kernel(LegArgs<T> a, int nbp, int yoff) {
  using C = typename Tr<T>::C;
  // m tile: this CTA takes m = blockIdx.y and, with MT = 2, then
  // m = L - blockIdx.y, so that every CTA has about the same l range
#pragma unroll 1
  for (int mi = 0; mi < MT; ++mi) {
    const int m = mi == 0 ? (int)blockIdx.y : a.L - (int)blockIdx.y;
    if (mi > 0 && m <= (int)blockIdx.y) break;
    if (mi > 0) __syncthreads();  // the shared buffers of the previous m are free
    const int L = a.L;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    // per-warp copies of the recurrence coefficients (staged by each warp),
    // and per-warp sums of the chunk's l, double-buffered by chunk parity in
    // FP32 so that one barrier per chunk suffices
    constexpr int NRB = sizeof(T) == 4 ? 2 : 1;
    __shared__ T sc_all[LEG_NW][LEG_CH];
    __shared__ T sc2_all[POLAR ? LEG_NW : 1][LEG_CH];
    __shared__ C red_all[NRB][LEG_NW][LEG_CH];
    __shared__ int s_min;
    T* sc = sc_all[warp];
    T* sc2 = sc2_all[POLAR ? warp : 0];

    T P1[RP], P2[RP], zz[RP];
    int ls[RP], p[RP];
    C GE[RP], GO[RP];
    const int yb = (int)blockIdx.x + yoff;
    int wmin, wmax;
    const bool live = load_pairs<T, POLAR, RP>(a, m, yb, nbp, warp, lane, p, ls, P1, P2, zz, &wmin, &wmax);
    const int pend = POLAR ? a.npolar : a.npairs;
#pragma unroll
    for (int j = 0; j < RP; ++j) {
      GE[j] = mk((T)0, (T)0);
      GO[j] = mk((T)0, (T)0);
      if (p[j] < pend && ls[j] <= L) {
        const int rn = p[j], rs = a.nring - 1 - p[j];
        if (SQ) {
          const T v = a.ringval[rn] + ((rs != rn) ? a.ringval[rs] : (T)0);
          GE[j] = mk(v, (T)0);
          GO[j] = GE[j];
        } else {
          const C gn = a.phase[(int64_t)rn * a.ldp + m];
          const C gs = (rs != rn) ? a.phase[(int64_t)rs * a.ldp + m] : mk((T)0, (T)0);
          GE[j] = cadd(gn, gs);
          GO[j] = csub(gn, gs);
        }
      }
    }
    if (tid == 0) s_min = L + 1;
    __syncthreads();
    if (lane == 0 && live) atomicMin(&s_min, wmin);
    __syncthreads();
    const int cmin = s_min;
    const int64_t offa = lm_off(L, m);
    const int64_t offc = lm_off(a.Lc, m);
    C* part = a.partial + (int64_t)yb * n_lm(L);
    const int lbeg = (cmin <= L) ? m + ((cmin - m) & ~7) : L + 1;
    // rows before the block's earliest start are zero
    for (int l = m + tid; l < lbeg; l += LEG_NT) part[offa + (l - m)] = mk((T)0, (T)0);

    int rb = 0;
    for (int l0 = lbeg; l0 <= L; l0 += LEG_CH) {
      const int nl = min(LEG_CH, L - l0 + 1);
      if (NRB == 1) __syncthreads();  // the previous chunk's sums are read
      C(*red)[LEG_CH] = red_all[rb];
      __syncwarp();
      for (int i = lane; i < nl; i += 32) {
        sc[i] = a.c[offc + (l0 - m) + i];
        if (POLAR) sc2[i] = a.c2[offc + (l0 - m) + i];
      }
      __syncwarp();
      for (int i8 = 0; i8 < nl; i8 += 8) {
        const int lg = l0 + i8;
        const int ng = min(8, nl - i8);
        if (!live || wmin >= lg + ng) {
          // no pair of this warp has started: its share of the sums is zero
          if (lane < 8) red[warp][i8 + lane] = mk((T)0, (T)0);
        } else {
          C acc[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) acc[u] = mk((T)0, (T)0);
          if (wmax <= lg && ng == 8) {
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
              const T c0 = sc[i8 + u], c1 = sc[i8 + u + 1];
              const T d0 = POLAR ? sc2[i8 + u] : (T)0, d1 = POLAR ? sc2[i8 + u + 1] : (T)0;
#pragma unroll
              for (int j = 0; j < RP; ++j) {
                T q0 = rstep<T, POLAR>(c0, d0, zz[j], P1[j], P2[j]);
                T q1 = rstep<T, POLAR>(c1, d1, zz[j], P1[j], P2[j]);
                if (SQ) {
                  q0 *= q0;
                  q1 *= q1;
                }
                acc[u].x = fma(q0, GE[j].x, acc[u].x);
                acc[u].y = fma(q0, GE[j].y, acc[u].y);
                acc[u + 1].x = fma(q1, GO[j].x, acc[u + 1].x);
                acc[u + 1].y = fma(q1, GO[j].y, acc[u + 1].y);
              }
            }
          } else {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              if (u < ng) {
                const int l = lg + u;
                const T c0 = sc[i8 + u];
                const T d0 = POLAR ? sc2[i8 + u] : (T)0;
#pragma unroll
                for (int j = 0; j < RP; ++j) {
                  if (l >= ls[j]) {
                    T q0 = rstep<T, POLAR>(c0, d0, zz[j], P1[j], P2[j]);
                    if (SQ) q0 *= q0;
                    const C g = (u & 1) ? GO[j] : GE[j];
                    acc[u].x = fma(q0, g.x, acc[u].x);
                    acc[u].y = fma(q0, g.y, acc[u].y);
                  }
                }
              }
            }
          }
          warp_reduce8(acc);
          if ((lane & 3) == 0) red[warp][i8 + (lane >> 2)] = acc[0];
        }
      }
      // one barrier per chunk: the warps' sums in a fixed order
      __syncthreads();
      for (int i = tid; i < nl; i += LEG_NT) {
        const int l = l0 + i;
        C sum = red[0][i];
#pragma unroll
        for (int w = 1; w < LEG_NW; ++w) sum = cadd(sum, red[w][i]);
        const T sc_ = a.s[offc + (l - m)];
        part[offa + (l - m)] = cscale(sum, SQ ? sc_ * sc_ : sc_);
      }
      rb = (rb + 1) % NRB;
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 adjoint with packed pairs of FP32 lanes.  Two ring pairs step together
// in one f32x2 instruction: the recurrence (sign-folded as in the packed
// synthesis: V_l = sigma_l Q_l, V_l = alpha_l z V_{l-1} + V_{l-2}, so the
// sums come out multiplied by sigma_l, which the partial-row write undoes;
// the polar difference form needs no sign change) and the accumulation
// A_l += V_l G, whose two halves hold the sums over the even and the odd
// members of the thread's pair list and are added once per 8-l group, each
// sum going straight to the warp's shared-memory transpose buffer.  Up to 16
// ring pairs per thread spread the reduction over more terms.  The chunk's
// recurrence coefficients and output scales s_lm (with the recurrence's sign)
// are staged in shared memory with their global loads issued four per lane
// at a time, so the per-group row write reads no global memory.
template <bool POLAR, int RP, int MT = 1>
__global__ void __launch_bounds__(L32_NT) leg_adjoint_f32x2_kernel(LegArgs<float> a, int nbp, int yoff) {
  static_assert(RP % 2 == 0, "pairs per thread must be even");
  constexpr int NP = RP / 2;
  // m tile: this CTA takes m = blockIdx.y and, with MT = 2, then
  // m = L - blockIdx.y, so that every CTA has about the same l range
#pragma unroll 1
  for (int mi = 0; mi < MT; ++mi) {
    const int m = mi == 0 ? (int)blockIdx.y : a.L - (int)blockIdx.y;
    if (mi > 0 && m <= (int)blockIdx.y) break;
    if (mi > 0) __syncwarp();  // the shared buffers of the previous m are free
    const int L = a.L;
    const int lane = threadIdx.x;
    __shared__ float2 sk[LEG_CH];
    __shared__ float2 sk2[POLAR ? LEG_CH : 1];
    __shared__ float sf[LEG_CH];
    __shared__ float2 rbuf[8][SMEM_RS];

    float P1[RP], P2[RP], zz[RP];
    int ls[RP], p[RP];
    float2 GE[RP], GO[RP];
    const int yb = (int)blockIdx.x + yoff;
    int wmin, wmax;
    const bool live = load_pairs<float, POLAR, RP, L32_NT>(a, m, yb, nbp, 0, lane, p, ls, P1, P2, zz, &wmin, &wmax);
    auto sgn = [&](int l) -> float { return ((l - m) & 2) ? -1.f : 1.f; };
    const int pend = POLAR ? a.npolar : a.npairs;
#pragma unroll
    for (int j = 0; j < RP; ++j) {
      GE[j] = make_float2(0.f, 0.f);
      GO[j] = make_float2(0.f, 0.f);
      if (p[j] < pend && ls[j] <= L) {
        const int rn = p[j], rs = a.nring - 1 - p[j];
        const float2 gn = a.phase[(int64_t)rn * a.ldp + m];
        const float2 gs = (rs != rn) ? a.phase[(int64_t)rs * a.ldp + m] : make_float2(0.f, 0.f);
        GE[j] = cadd(gn, gs);
        GO[j] = csub(gn, gs);
        if (!POLAR) {
          P1[j] *= sgn(ls[j] - 1);
          P2[j] *= sgn(ls[j] - 2);
        }
      }
    }
    const int64_t offa = lm_off(L, m);
    const int64_t offc = lm_off(a.Lc, m);
    // this warp's partial row: zero before its first group
    float2* part = a.partial + (int64_t)yb * n_lm(L);
    const int lbeg = live ? m + ((wmin - m) & ~7) : L + 1;
    for (int l = m + lane; l < lbeg; l += 32) part[offa + (l - m)] = make_float2(0.f, 0.f);

    for (int l0 = lbeg; l0 <= L; l0 += LEG_CH) {
      const int nl = min(LEG_CH, L - l0 + 1);
      __syncwarp();
      {
        const float* cg = a.c + offc + (l0 - m);
        const float* c2g = POLAR ? a.c2 + offc + (l0 - m) : nullptr;
        const float* sg = a.s + offc + (l0 - m);
        constexpr int SB = POLAR ? 2 : 4;  // loads in flight per array and lane
#pragma unroll
        for (int k0 = 0; k0 < LEG_CH / 32; k0 += SB) {
          float cv[SB], c2v[SB], sv[SB];
#pragma unroll
          for (int k = 0; k < SB; ++k) {
            const int i = lane + 32 * (k0 + k);
            cv[k] = c2v[k] = sv[k] = 0.f;
            if (i < nl) {
              cv[k] = cg[i];
              if (POLAR) c2v[k] = c2g[i];
              sv[k] = sg[i];
            }
          }
#pragma unroll
          for (int k = 0; k < SB; ++k) {
            const int i = lane + 32 * (k0 + k);
            if (i < nl) {
              const int l = l0 + i;
              if (POLAR) {
                sk[i] = make_float2(-cv[k], -cv[k]);
                sk2[i] = make_float2(c2v[k], c2v[k]);
                sf[i] = sv[k];
              } else {
                const float al = ((l - m) & 1) ? cv[k] : -cv[k];
                sk[i] = make_float2(al, al);
                sf[i] = sv[k] * sgn(l);
              }
            }
          }
        }
      }
      __syncwarp();
      for (int i8 = 0; i8 < nl; i8 += 8) {
        const int lg = l0 + i8;
        const int ng = min(8, nl - i8);
        if (wmax <= lg && ng == 8) {
          u64 Z[NP], S1[NP], S2[NP], EX[NP], EY[NP], OX[NP], OY[NP];
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            Z[q] = pk2(zz[2 * q], zz[2 * q + 1]);
            S1[q] = pk2(P1[2 * q], P1[2 * q + 1]);
            S2[q] = pk2(P2[2 * q], P2[2 * q + 1]);
            EX[q] = pk2(GE[2 * q].x, GE[2 * q + 1].x);
            EY[q] = pk2(GE[2 * q].y, GE[2 * q + 1].y);
            OX[q] = pk2(GO[2 * q].x, GO[2 * q + 1].x);
            OY[q] = pk2(GO[2 * q].y, GO[2 * q + 1].y);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const u64 K = lds2(&sk[i8 + u]);
            const u64 K2 = POLAR ? lds2(&sk2[i8 + u]) : 0ull;
            u64 AX = 0ull, AY = 0ull;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
              u64 Q;
              if (POLAR) {
                const u64 E = fma2(K, Z[q], K2);
                const u64 D = fma2(E, S1[q], S2[q]);
                Q = add2(S1[q], D);
                S2[q] = D;
              } else {
                Q = fma2(mul2(K, Z[q]), S1[q], S2[q]);
                S2[q] = S1[q];
              }
              S1[q] = Q;
              if (u & 1) {
                AX = q ? fma2(Q, OX[q], AX) : mul2(Q, OX[q]);
                AY = q ? fma2(Q, OY[q], AY) : mul2(Q, OY[q]);
              } else {
                AX = q ? fma2(Q, EX[q], AX) : mul2(Q, EX[q]);
                AY = q ? fma2(Q, EY[q], AY) : mul2(Q, EY[q]);
              }
            }
            float x0, x1, y0, y1;
            upk2(AX, x0, x1);
            upk2(AY, y0, y1);
            rbuf[u][lane] = make_float2(x0 + x1, y0 + y1);
          }
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            upk2(S1[q], P1[2 * q], P1[2 * q + 1]);
            upk2(S2[q], P2[2 * q], P2[2 * q + 1]);
          }
        } else {
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            float2 acc = make_float2(0.f, 0.f);
            if (u < ng) {
              const int l = lg + u;
              const float K = sk[i8 + u].x;
              const float K2 = POLAR ? sk2[i8 + u].x : 0.f;
#pragma unroll
              for (int j = 0; j < RP; ++j) {
                if (l >= ls[j]) {
                  float q;
                  if (POLAR) {
                    const float e = fmaf(K, zz[j], K2);
                    const float d = fmaf(e, P1[j], P2[j]);
                    q = P1[j] + d;
                    P2[j] = d;
                  } else {
                    q = fmaf(K * zz[j], P1[j], P2[j]);
                    P2[j] = P1[j];
                  }
                  P1[j] = q;
                  const float2 g = (u & 1) ? GO[j] : GE[j];
                  acc.x = fmaf(q, g.x, acc.x);
                  acc.y = fmaf(q, g.y, acc.y);
                }
              }
            }
            rbuf[u][lane] = acc;
          }
        }
        const float2 sum = smem_rows8_sum(rbuf);
        // lane 4 u holds the warp's sum for l = lg + u: scale by s_lm (and the
        // recurrence's sign) and write it to the row
        const int u = lane >> 2;
        if ((lane & 3) == 0 && u < ng) part[offa + (lg + u - m)] = cscale(sum, sf[i8 + u]);
      }
    }
  }
}

// y_lm = dl_out[l] * sum_blk partial[blk][lm] + dadd[l] * xadd_lm; zero at
// inactive l (dl_out = dadd = 0 there) and Im(a_l0) = 0.
template <typename T>
__global__ void leg_finalize_kernel(FinalizeArgs<T> a) {
  using C = typename Tr<T>::C;
  const int64_t nlm = n_lm(a.L);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nlm; i += (int64_t)gridDim.x * blockDim.x) {
    C s = a.partial[i];
    for (int b = 1; b < a.nblk; ++b) s = cadd(s, a.partial[(int64_t)b * nlm + i]);
    // recover l, m from the flat index (m-major layout)
    int m = (int)((2.0 * (a.L + 1) + 1.0 - sqrt((2.0 * (a.L + 1) + 1.0) * (2.0 * (a.L + 1) + 1.0) - 8.0 * (double)i)) * 0.5);
    while (m > 0 && lm_off(a.L, m) > i) --m;
    while (m < a.L && lm_off(a.L, m + 1) <= i) ++m;
    const int l = m + (int)(i - lm_off(a.L, m));
    T f = a.dl_out ? a.dl_out[l] : (T)1;
    C y = cscale(s, f);
    if (a.dadd) {
      C x = a.xadd[i];
      y.x = fma(a.dadd[l], x.x, y.x);
      y.y = fma(a.dadd[l], x.y, y.y);
    }
    if (a.bsub) {
      const C bb = a.bsub[i];
      y = mk(bb.x - y.x, (m == 0) ? (T)0 : bb.y - y.y);
    }
    if (m == 0) y.y = 0;
    if (a.accumulate) y = cadd(y, a.out[i]);
    a.out[i] = y;
  }
}

static inline void pair_blocks(int npolar, int npairs, int rp, int* nbp, int* nbe, int nt = LEG_NT) {
  *nbp = (npolar + nt * rp - 1) / (nt * rp);
  *nbe = (npairs - npolar + nt * rp - 1) / (nt * rp);
}

// ring pairs per thread of a launch: 2, 4 or 8, and 16 for the packed FP32
// adjoint (other values: the default)
static inline int legal_rp(int rp) { return (rp == 2 || rp == 4 || rp == 8) ? rp : LEG_RP; }
static inline int legal_rp_f32adj(int rp) { return (rp == 2 || rp == 4 || rp == 8 || rp == 16) ? rp : LEG_RP; }

// rows of m of a launch: L + 1, or (L + 2) / 2 when each CTA pairs m with L - m
static inline int m_rows(int L, int mt) { return mt == 2 ? (L + 2) / 2 : L + 1; }

template <typename T, int RP, int MT>
static void synth_launch_mt(const LegArgs<T>& a, int nbp, int nbe, cudaStream_t st) {
  const int MROWS = m_rows(a.L, MT);
  if constexpr (sizeof(T) == 4) {
    if (nbp) { leg_synth_f32x2_kernel<true, RP, MT><<<dim3(nbp, MROWS), L32_NT, 0, st>>>(a, nbp, 0); count_launch(); }
    if (nbe) { leg_synth_f32x2_kernel<false, RP, MT><<<dim3(nbe, MROWS), L32_NT, 0, st>>>(a, nbp, nbp); count_launch(); }
  } else {
    if (nbp) { leg_synth_kernel<T, true, RP, MT><<<dim3(nbp, MROWS), LEG_NT, 0, st>>>(a, nbp, 0); count_launch(); }
    if (nbe) { leg_synth_kernel<T, false, RP, MT><<<dim3(nbe, MROWS), LEG_NT, 0, st>>>(a, nbp, nbp); count_launch(); }
  }
}
template <typename T, int RP>
static void synth_launch(const LegArgs<T>& a, int nbp, int nbe, cudaStream_t st) {
  if (a.mt_synth == 2) synth_launch_mt<T, RP, 2>(a, nbp, nbe, st);
  else synth_launch_mt<T, RP, 1>(a, nbp, nbe, st);
}

template <typename T, int RP, int MT>
static void adjoint_launch_mt(const LegArgs<T>& a, int nbp, int nbe, cudaStream_t st) {
  const int MROWS = m_rows(a.L, MT);
  if constexpr (sizeof(T) == 4) {
    if (nbp) { leg_adjoint_f32x2_kernel<true, RP, MT><<<dim3(nbp, MROWS), L32_NT, 0, st>>>(a, nbp, 0); count_launch(); }
    if (nbe) { leg_adjoint_f32x2_kernel<false, RP, MT><<<dim3(nbe, MROWS), L32_NT, 0, st>>>(a, nbp, nbp); count_launch(); }
  } else {
    if (nbp) { leg_adjoint_kernel<T, true, RP, false, MT><<<dim3(nbp, MROWS), LEG_NT, 0, st>>>(a, nbp, 0); count_launch(); }
    if (nbe) { leg_adjoint_kernel<T, false, RP, false, MT><<<dim3(nbe, MROWS), LEG_NT, 0, st>>>(a, nbp, nbp); count_launch(); }
  }
}
template <typename T, int RP>
static void adjoint_launch(const LegArgs<T>& a, int nbp, int nbe, cudaStream_t st) {
  if (a.mt_adj == 2) adjoint_launch_mt<T, RP, 2>(a, nbp, nbe, st);
  else adjoint_launch_mt<T, RP, 1>(a, nbp, nbe, st);
}

template <typename T>
int launch_leg_synth(const LegArgs<T>& a, cudaStream_t st) {
  if (a.L < 0) return CR_OK;
  if constexpr (sizeof(T) == 8)
    if (a.df) return launch_leg_synth_df(a, st);
  int nbp, nbe;
  const int rp = legal_rp(a.rp_synth);
  pair_blocks(a.npolar, a.npairs, rp, &nbp, &nbe, sizeof(T) == 4 ? L32_NT : LEG_NT);
  if (rp == 2) synth_launch<T, 2>(a, nbp, nbe, st);
  else if (rp == 8) synth_launch<T, 8>(a, nbp, nbe, st);
  else synth_launch<T, 4>(a, nbp, nbe, st);
  CR_CHECK_LAUNCH("leg_synth_kernel");
  return CR_OK;
}

template <typename T>
int launch_leg_adjoint(const LegArgs<T>& a, const FinalizeArgs<T>& f, cudaStream_t st) {
  if (a.L < 0) return CR_OK;
  int nbp = 0, nbe = 0;
  bool done = false;
  if constexpr (sizeof(T) == 8) {
    if (a.df) {
      int rc = launch_leg_adjoint_df(a, &nbe, st);
      if (rc) return rc;
      done = true;
    }
  }
  if (!done) {
    const int rp = sizeof(T) == 4 ? legal_rp_f32adj(a.rp_adj) : legal_rp(a.rp_adj);
    pair_blocks(a.npolar, a.npairs, rp, &nbp, &nbe, sizeof(T) == 4 ? L32_NT : LEG_NT);
    if (rp == 2) adjoint_launch<T, 2>(a, nbp, nbe, st);
    else if (rp == 8) adjoint_launch<T, 8>(a, nbp, nbe, st);
    else if constexpr (sizeof(T) == 4) {
      if (rp == 16) adjoint_launch<T, 16>(a, nbp, nbe, st);
      else adjoint_launch<T, 4>(a, nbp, nbe, st);
    } else {
      adjoint_launch<T, 4>(a, nbp, nbe, st);
    }
    CR_CHECK_LAUNCH("leg_adjoint_kernel");
  }
  FinalizeArgs<T> ff = f;
  ff.partial = a.partial;
  ff.nblk = nbp + nbe;
  ff.L = a.L;
  return launch_leg_finalize<T>(ff, st);
}

template <typename T>
int launch_leg_finalize(const FinalizeArgs<T>& f, cudaStream_t st) {
  const int64_t nlm = n_lm(f.L);
  int blocks = (int)std::min<int64_t>((nlm + 255) / 256, 152 * 16);
  { leg_finalize_kernel<T><<<blocks, 256, 0, st>>>(f); count_launch(); }
  CR_CHECK_LAUNCH("leg_finalize_kernel");
  return CR_OK;
}

// out_lm = sum_k P~_lm(z_k)^2 ringval_k on the observation grid (FP64)
int launch_leg_diag(cr_plan* P, const double* ringval, double2* out) {
  const Grid& g = P->obs;
  LegArgs<double> a;
  a.ldp = P->lmax + 1;
  a.L = P->lmax;
  a.Lc = P->Lcoef;
  a.c = P->d_c;
  a.s = P->d_s;
  a.z = g.d_z;
  a.ls = g.d_ls64;
  a.st = g.d_st64;
  a.ld_seed = g.npairs;
  a.npairs = g.npairs;
  a.nring = g.nring;
  a.npolar = 0;
  a.ringval = ringval;
  a.partial = reinterpret_cast<double2*>(P->ws.partial);
  int nbp, nbe;
  pair_blocks(0, a.npairs, LEG_RP, &nbp, &nbe);
  { leg_adjoint_kernel<double, false, LEG_RP, true><<<dim3(nbe, a.L + 1), LEG_NT, 0, P->stream>>>(a, 0, 0); count_launch(); }
  CR_CHECK_LAUNCH("leg_adjoint_kernel<SQ>");
  FinalizeArgs<double> ff;
  ff.partial = a.partial;
  ff.nblk = nbe;
  ff.L = a.L;
  ff.out = out;
  const int64_t nlm = n_lm(a.L);
  { leg_finalize_kernel<double><<<(int)std::min<int64_t>((nlm + 255) / 256, 152 * 16), 256, 0, P->stream>>>(ff); count_launch(); }
  CR_CHECK_LAUNCH("leg_finalize_kernel");
  return CR_OK;
}

// Start tables (see Grid): for each m <= Lseed and ring pair, the scaled FP64
// recurrence from the seed P~_mm up to the first l with |P~_lm| >= tau.
__global__ void start_kernel(const double* z, const double* seed, const int* lev, int ld, const double* c,
                             const double* s, int Lc, int Lseed, int npairs, int npolar32, int* ls64,
                             double2* st64, int* ls32, float2* st32, double2* st64b) {
  const int m = blockIdx.y;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const int64_t o = (int64_t)m * ld + p;
  const double zz = z[p];
  const int64_t offc = lm_off(Lc, m);
  const double thr = exp2((double)Tr<double>::THR);
  const double down = exp2(-(double)Tr<double>::S);
  const double tau64 = exp2(-100.0), tau32 = exp2(-60.0);
  double q1 = 0.0, q2 = -seed[o];
  int e = lev[o];
  int f64 = Lseed + 1, f32 = Lseed + 1;
  double2 s64 = make_double2(0.0, 0.0), s64b = make_double2(0.0, 0.0);
  float2 s32 = make_float2(0.f, 0.f);
  for (int l = m; l <= Lseed; ++l) {
    const double q = c[offc + (l - m)] * zz * q1 - q2;
    if (e == 0) {
      const double pv = fabs(s[offc + (l - m)] * q);
      if (f64 > Lseed && pv >= tau64) {
        f64 = l;
        s64 = make_double2(q1, q2);
      }
      if (pv >= tau32) {  // tau32 > tau64: the FP32 start comes last
        f32 = l;
        s32 = (p < npolar32) ? make_float2((float)q1, (float)(q1 - q2)) : make_float2((float)q1, (float)q2);
        s64b = make_double2(q1, q2);
        break;
      }
    }
    q2 = q1;
    q1 = q;
    if (e < 0 && fabs(q1) > thr) {
      q1 *= down;
      q2 *= down;
      ++e;
    }
  }
  ls64[o] = f64;
  st64[o] = s64;
  ls32[o] = f32;
  st32[o] = s32;
  st64b[o] = s64b;
}

int build_start_tables(cr_plan* P, Grid& g) {
  const int Ls = g.Lseed;
  if (Ls < 0) return CR_OK;
  if (Ls > P->Lcoef) return fail(CR_EINVAL, "start tables: grid band limit above the recurrence tables");
  void* ptrs[] = {g.d_ls64, g.d_st64, g.d_ls32, g.d_st32, g.d_st64b};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  const int64_t n = (int64_t)(Ls + 1) * g.npairs;
  CR_CUDA(cudaMalloc(&g.d_ls64, n * sizeof(int)));
  CR_CUDA(cudaMalloc(&g.d_st64, n * sizeof(double2)));
  CR_CUDA(cudaMalloc(&g.d_ls32, n * sizeof(int)));
  CR_CUDA(cudaMalloc(&g.d_st32, n * sizeof(float2)));
  CR_CUDA(cudaMalloc(&g.d_st64b, n * sizeof(double2)));
  dim3 grid((g.npairs + 127) / 128, Ls + 1);
  { start_kernel<<<grid, 128, 0, P->stream>>>(g.d_z, g.d_seed, g.d_lev, g.npairs, P->d_c, P->d_s, P->Lcoef, Ls,
                                               g.npairs, g.npolar32, g.d_ls64, g.d_st64, g.d_ls32, g.d_st32,
                                               g.d_st64b);
    count_launch(); }
  CR_CHECK_LAUNCH("start_kernel");
  CR_CUDA(cudaStreamSynchronize(P->stream));
  return CR_OK;
}

// upper bound on the partial rows of the adjoint: the polar and equatorial
// ranges of 32 * RP pairs (one-warp FP32 blocks; the FP64 blocks of
// LEG_NT * RP pairs are fewer) for the smallest RP, or the double-float
// kernels' blocks
int leg_partial_blocks(int npairs) {
  return std::max((npairs + L32_NT * LEG_RP_MIN - 1) / (L32_NT * LEG_RP_MIN) + 1, df_pair_blocks(npairs));
}

template int launch_leg_synth<double>(const LegArgs<double>&, cudaStream_t);
template int launch_leg_synth<float>(const LegArgs<float>&, cudaStream_t);
template int launch_leg_finalize<double>(const FinalizeArgs<double>&, cudaStream_t);
template int launch_leg_finalize<float>(const FinalizeArgs<float>&, cudaStream_t);
template int launch_leg_adjoint<double>(const LegArgs<double>&, const FinalizeArgs<double>&, cudaStream_t);
template int launch_leg_adjoint<float>(const LegArgs<float>&, const FinalizeArgs<float>&, cudaStream_t);

}  // namespace cr
