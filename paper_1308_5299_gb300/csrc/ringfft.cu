// Per-ring azimuthal stages of synthesis Y and adjoint synthesis Y^T
// (Section 2.1; the per-ring DFTs of Section 3.3), without cuFFT.
//
// Ring r has n (even) pixels at phi_j = pi (2 j + s) / n, s in {0, 1} (HEALPix
// and Gauss-Legendre rings both have this form).
//
// Synthesis of a real field from F_m (m = 0..L):
//   map_j = Re sum_{m} w_m F_m e^{i m phi_j},  w_0 = 1, w_{m>0} = 2
//         = sum_{b<n} H'_b e^{2 pi i b j / n},
//   H_b  = sum_{m = b mod n} w_m F_m e^{i pi s m / n}  (band limits above n/2
//          fold onto the ring's n bins), H'_b = (H_b + conj H_{n-b}) / 2.
// H' is Hermitian, so the length-n real inverse DFT is done as one complex
// inverse DFT of length nh = n/2 on Z_k = (H'_k + conj H'_{nh-k})
// + i w^k (H'_k - conj H'_{nh-k}), w = e^{2 pi i / n}; z = IDFT(Z) gives
// map_{2t} = Re z_t, map_{2t+1} = Im z_t.
// Adjoint: Yhat_b = sum_j y_j e^{-2 pi i b j / n} from a length-nh forward
// DFT of z_t = y_{2t} + i y_{2t+1}; then G_m = e^{-i pi s m / n} Yhat_{m mod n}
// (conjugate-symmetric extension for m mod n > n/2): the exact transpose of
// the folding above.
//
// Length-nh DFTs: radix-2 in shared memory when nh is a power of two,
// otherwise Bluestein's chirp-z with a power-of-two convolution of size
// M >= 2 nh - 1 (decimation-in-frequency forward FFT, pointwise product with
// the precomputed kernel spectrum stored in bit-reversed order,
// decimation-in-time inverse FFT: no bit-reversal passes).  The chirp
// e^{i pi k^2 / nh} = e^{i pi (2 k^2 mod 2n) / n} comes from an exact integer
// reduction into the ring length's table of e^{i pi u / n}, u < 2n.
//
// One CTA per ring; mode 2 keeps the ring's map in shared memory between the
// synthesis and the adjoint (map * N^-1 never touches HBM).
#include <algorithm>
#include <cstdio>
#include <map>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace cr {

constexpr int RF_NT = 256;

// Shared-memory position of FFT buffer element i: bits 4..15 XOR-folded into
// bits 0..3 (a bijection on [0, 2^16)).  With 8-byte elements a bank pair
// holds positions equal mod 16; the fold spreads every access pattern of
// the kernels below -- consecutive, the radix-8 passes' strides 8^p, and the
// bit-reversed scatter and gather -- over all 16 bank pairs.
__device__ __forceinline__ int swz(int i) { return i ^ (((i >> 4) ^ (i >> 8) ^ (i >> 12)) & 15); }

__device__ __forceinline__ int bitrev(int k, int logM) {
  return logM ? (int)(__brev((unsigned)k) >> (32 - logM)) : 0;
}

template <typename C>
__device__ __forceinline__ C twid(const C* __restrict__ tw, int idx, int sign) {
  const C w = tw[idx];
  return sign > 0 ? cconj(w) : w;
}
// radix-2 butterflies: decimation in time a' = a + w b, b' = a - w b;
// decimation in frequency a' = a + b, b' = (a - b) w
template <typename C>
__device__ __forceinline__ void bf_dit(C& a, C& b, C w) {
  const C v = cmul(b, w);
  b = csub(a, v);
  a = cadd(a, v);
}
template <typename C>
__device__ __forceinline__ void bf_dif(C& a, C& b, C w) {
  const C u = a;
  a = cadd(u, b);
  b = cmul(csub(u, b), w);
}

// e^{-2 pi i v / 32}, v < 16: the constant factors of the twiddles inside
// one pass (cos and sin of 2 pi v / 32)
__device__ constexpr double RC32[16] = {1.0, 0.980785280403230449126, 0.923879532511286756128, 0.831469612302545237079,
                                        0.707106781186547524401, 0.555570233019602224743, 0.382683432365089771728,
                                        0.195090322016128267848, 0.0, -0.195090322016128267848, -0.382683432365089771728,
                                        -0.555570233019602224743, -0.707106781186547524401, -0.831469612302545237079,
                                        -0.923879532511286756128, -0.980785280403230449126};
__device__ constexpr double RS32[16] = {0.0, 0.195090322016128267848, 0.382683432365089771728, 0.555570233019602224743,
                                        0.707106781186547524401, 0.831469612302545237079, 0.923879532511286756128,
                                        0.980785280403230449126, 1.0, 0.980785280403230449126, 0.923879532511286756128,
                                        0.831469612302545237079, 0.707106781186547524401, 0.555570233019602224743,
                                        0.382683432365089771728, 0.195090322016128267848};

// One pass of NS consecutive radix-2 stages on groups of 2^NS elements
// j0 + t h (t < 2^NS) held in registers.  Stage s of the pass has span
// 2^s h; its butterfly on (t, t + 2^s), u = t mod 2^s, uses the twiddle
// e^{-+2 pi i (k + u h) / (2^(s+1) h)}.  With CTW (computed twiddles) that
// is base_s e^{-+2 pi i u / 2^(s+1)}: one table value per stage and group
// (base_s, index k Mmax / (2^(s+1) h)) times a compile-time root of unity --
// fewer loads for a few FP32 multiplies; without, every distinct twiddle
// is a table value (FP64, where a multiply costs more than a cached load).
// DIT runs the stages with spans h, 2h, ... (bit-reversed input, natural
// output); DIF the reverse (natural input, bit-reversed output).  post (may
// be null): every element is multiplied by post[its position] before it is
// stored (the pointwise product of a convolution, fused into the last pass).
template <typename C, int NS, bool DIT, bool CTW>
__device__ __forceinline__ void fft_pass(C* buf, int M, int lh, int sign, const C* __restrict__ tw, int Mmax,
                                         const C* __restrict__ post) {
  using T = decltype(C().x);
  constexpr int R = 1 << NS;
  const int h = 1 << lh;
  const int ng = M >> NS;
  for (int g = threadIdx.x; g < ng; g += blockDim.x) {
    const int k = g & (h - 1);
    const int j0 = ((g - k) << NS) + k;
    C base[NS];
    if (CTW) {
#pragma unroll
      for (int s = 0; s < NS; ++s) base[s] = twid(tw, k * (Mmax >> (lh + s + 1)), sign);
    }
    C e[R];
#pragma unroll
    for (int t = 0; t < R; ++t) e[t] = buf[swz(j0 + t * h)];
#pragma unroll
    for (int si = 0; si < NS; ++si) {
      const int s = DIT ? si : NS - 1 - si;
      const int S = 1 << s;
#pragma unroll
      for (int t = 0; t < R; ++t) {
        if (t & S) continue;
        const int u = t & (S - 1);
        C w;
        if (CTW) {
          w = base[s];
          if (u) {
            const int v = u << (4 - s);
            const T cr = (T)RC32[v], ci = (T)(sign > 0 ? RS32[v] : -RS32[v]);
            w = mk(w.x * cr - w.y * ci, w.x * ci + w.y * cr);
          }
        } else {
          w = twid(tw, (k + u * h) * (Mmax >> (lh + s + 1)), sign);
        }
        if (DIT) bf_dit(e[t], e[t + S], w);
        else bf_dif(e[t], e[t + S], w);
      }
    }
    if (post) {
#pragma unroll
      for (int t = 0; t < R; ++t) e[t] = cmul(e[t], post[j0 + t * h]);
    }
#pragma unroll
    for (int t = 0; t < R; ++t) buf[swz(j0 + t * h)] = e[t];
  }
}

// BIG: up to 4 stages per pass with computed twiddles (FP32 rings with
// M >= 4096: fewer barriers and shared-memory round trips, at 75 registers);
// otherwise up to 3 with table twiddles (fewer registers, so more CTAs per
// SM, which the small rings need).  Never more stages than leave one group
// per thread.
template <bool BIG>
__device__ __forceinline__ int fft_pass_cap(int logM) {
  const int lt = 31 - __clz((int)blockDim.x);
  return max(1, min(BIG ? 4 : 3, logM - lt));
}

template <typename C, bool DIT, bool BIG>
__device__ __forceinline__ void fft_pass_ns(int ns, C* buf, int M, int lh, int sign, const C* __restrict__ tw,
                                            int Mmax, const C* __restrict__ post) {
  if (BIG && ns == 4) fft_pass<C, 4, DIT, true>(buf, M, lh, sign, tw, Mmax, post);
  else if (ns >= 3) fft_pass<C, 3, DIT, BIG>(buf, M, lh, sign, tw, Mmax, post);
  else if (ns == 2) fft_pass<C, 2, DIT, BIG>(buf, M, lh, sign, tw, Mmax, post);
  else fft_pass<C, 1, DIT, BIG>(buf, M, lh, sign, tw, Mmax, post);
}

// In-place radix-2 decimation-in-time FFT: bit-reversed input, natural output.
// sign = -1 forward (e^{-2 pi i jk/M}), +1 inverse (unnormalised).  Passes
// of several consecutive stages, one barrier per pass.
template <bool BIG = false, typename C>
__device__ void fft_dit(C* buf, int M, int logM, int sign, const C* __restrict__ tw, int Mmax) {
  const int cap = fft_pass_cap<BIG>(logM);
  int lh = 0;
  while (lh < logM) {
    const int ns = min(cap, logM - lh);
    fft_pass_ns<C, true, BIG>(ns, buf, M, lh, sign, tw, Mmax, nullptr);
    __syncthreads();
    lh += ns;
  }
}

// In-place radix-2 decimation-in-frequency FFT: natural input, bit-reversed
// output; passes of several stages (largest span first).  post (may be
// null): multiply the output, in its bit-reversed positions, by post.
template <bool BIG = false, typename C>
__device__ void fft_dif(C* buf, int M, int logM, int sign, const C* __restrict__ tw, int Mmax,
                        const C* __restrict__ post = nullptr) {
  const int cap = fft_pass_cap<BIG>(logM);
  int lt = logM;  // stages with span >= 2^lt are done
  while (lt > 0) {
    const int ns = min(cap, lt);
    const int lh = lt - ns;  // smallest span of this pass
    fft_pass_ns<C, false, BIG>(ns, buf, M, lh, sign, tw, Mmax, lh == 0 ? post : nullptr);
    __syncthreads();
    lt = lh;
  }
}

template <typename T, int MODE, bool BIG>
__global__ void __launch_bounds__(RF_NT) ring_fft_kernel(RingArgs<T> a) {
  using C = typename Tr<T>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  const int r = a.rings[a.rbase + blockIdx.x];
  const RingFFT f = a.fft[r];
  const C* __restrict__ tab = a.tab + f.tab;
  const C* __restrict__ vh = a.vhat + f.vhat;
  const int n = f.n, nh = f.nh, M = f.M, lg = f.logM;
  const int twon = 2 * n;
  C* row = a.phase + (int64_t)r * a.ldp;
  const int L = a.L;
  const int tid = threadIdx.x;
  const int NT = blockDim.x;
  // e^{i pi (2 k^2 mod 2n) / n}; 2 k^2 < 2^31 for k < 2^15
  auto chirp = [&](int k) -> C { return tab[(int)((2u * (unsigned)k * (unsigned)k) % (unsigned)twon)]; };

  if (MODE != 1) {
    auto fold = [&](int b) -> C {
      // m = b + q n: e^{i pi s m / n} = tab[s (b + (q mod 2) n)]
      C h = mk((T)0, (T)0);
      int u = f.shift ? b : 0;
      const int du = f.shift ? n : 0;
      for (int m = b; m <= L; m += n) {
        const C F = row[m];
        const C v = cmul(F, tab[u]);
        const T w = (m == 0) ? (T)1 : (T)2;
        h.x = fma(w, v.x, h.x);
        h.y = fma(w, v.y, h.y);
        u = (u + du < twon) ? u + du : u + du - twon;
      }
      return h;
    };
    auto Hp = [&](int b) -> C {
      const C h1 = fold(b);
      const C h2 = fold(b == 0 ? 0 : n - b);
      return cscale(cadd(h1, cconj(h2)), (T)0.5);
    };
    // Rings with fewer bins than threads split each bin's fold over g lanes
    // (a power of two <= 32; lane j of a group takes m = b + q n with
    // q = j mod g, whose phase e^{i pi s m / n} is then constant) and sum the
    // g partial Z in a fixed shuffle order: the long serial folds of the
    // small polar rings become g short ones.
    int g = 1;
    while (g < 32 && nh * g * 2 <= NT) g <<= 1;
    if (g == 1) {
      for (int k = tid; k < nh; k += NT) {
        const C A = Hp(k);
        const C B = cconj(Hp(nh - k));
        const C w = tab[2 * k];
        const C Z = cadd(cadd(A, B), cmuli(cmul(w, csub(A, B))));
        if (!f.bluestein) buf[swz(bitrev(k, lg))] = Z;
        else buf[swz(k)] = cmul(Z, chirp(k));
      }
    } else {
      const int k = tid / g, j = tid & (g - 1);
      auto fold_part = [&](int b) -> C {
        C h = mk((T)0, (T)0);
#pragma unroll 4
        for (int m = b + j * n; m <= L; m += g * n) {
          const C F = row[m];
          const T w = (m == 0) ? (T)1 : (T)2;
          h.x = fma(w, F.x, h.x);
          h.y = fma(w, F.y, h.y);
        }
        return f.shift ? cmul(h, tab[b + ((j & 1) ? n : 0)]) : h;
      };
      auto Hpp = [&](int b) -> C {
        const C h1 = fold_part(b);
        const C h2 = fold_part(b == 0 ? 0 : n - b);
        return cscale(cadd(h1, cconj(h2)), (T)0.5);
      };
      C Z = mk((T)0, (T)0);
      if (k < nh) {
        const C A = Hpp(k);
        const C B = cconj(Hpp(nh - k));
        Z = cadd(cadd(A, B), cmuli(cmul(tab[2 * k], csub(A, B))));
      }
      for (int o = g >> 1; o > 0; o >>= 1) {
        Z.x += __shfl_xor_sync(0xffffffffu, Z.x, o);
        Z.y += __shfl_xor_sync(0xffffffffu, Z.y, o);
      }
      if (k < nh && j == 0) {
        if (!f.bluestein) buf[swz(bitrev(k, lg))] = Z;
        else buf[swz(k)] = cmul(Z, chirp(k));
      }
    }
    if (f.bluestein)
      for (int k = nh + tid; k < M; k += NT) buf[swz(k)] = mk((T)0, (T)0);
    __syncthreads();
    if (!f.bluestein) {
      fft_dit<BIG>(buf, M, lg, +1, a.tw, a.Mmax);
    } else {
      fft_dif<BIG>(buf, M, lg, -1, a.tw, a.Mmax, vh);  // times the kernel spectrum
      fft_dit<BIG>(buf, M, lg, +1, a.tw, a.Mmax);
    }
    // z_t = (map_{2t}, map_{2t+1}) = buf[t] (times the chirp for Bluestein rings)
    auto z_of = [&](int t) -> C { return f.bluestein ? cmul(buf[swz(t)], chirp(t)) : buf[swz(t)]; };
    if (MODE == 0) {
      C* out = reinterpret_cast<C*>(a.map_out + f.off);
      for (int t = tid; t < nh; t += NT) out[t] = z_of(t);
      return;
    }
    // MODE 2: multiply by the pixel diagonal and continue with the adjoint.
    const C* dg = reinterpret_cast<const C*>(a.pixdiag + f.off);
    C* mo = a.map_out ? reinterpret_cast<C*>(a.map_out + f.off) : nullptr;
    for (int t = tid; t < nh; t += NT) {
      C z = z_of(t);
      if (mo) mo[t] = z;
      const C d = dg[t];
      z.x *= d.x;
      z.y *= d.y;
      buf[swz(t)] = f.bluestein ? cmul(cconj(z), chirp(t)) : z;
    }
    if (f.bluestein)
      for (int k = nh + tid; k < M; k += NT) buf[swz(k)] = mk((T)0, (T)0);
    __syncthreads();
  } else {
    const C* in = reinterpret_cast<const C*>(a.map_in + f.off);
    for (int t = tid; t < nh; t += NT) {
      const C z = in[t];
      buf[swz(t)] = f.bluestein ? cmul(cconj(z), chirp(t)) : z;
    }
    if (f.bluestein)
      for (int k = nh + tid; k < M; k += NT) buf[swz(k)] = mk((T)0, (T)0);
    __syncthreads();
  }

  // forward length-nh DFT of z_t = y_{2t} + i y_{2t+1}
  if (!f.bluestein) {
    fft_dif<BIG>(buf, M, lg, -1, a.tw, a.Mmax);  // Z'_k at buf[bitrev(k)]
  } else {
    fft_dif<BIG>(buf, M, lg, -1, a.tw, a.Mmax, vh);  // times the kernel spectrum
    fft_dit<BIG>(buf, M, lg, +1, a.tw, a.Mmax);      // Z'_k = conj(buf[k] chirp(k))
  }
  auto getZ = [&](int k) -> C {
    return f.bluestein ? cconj(cmul(buf[swz(k)], chirp(k))) : buf[swz(bitrev(k, lg))];
  };
  auto Yhat = [&](int b) -> C {  // b in [0, nh]
    const C Zb = getZ(b == nh ? 0 : b);
    const C Zc = cconj(getZ(b == 0 ? 0 : nh - b));
    const C E = cscale(cadd(Zb, Zc), (T)0.5);
    const C O = cscale(csub(Zb, Zc), (T)0.5);
    const C wm = cconj(tab[2 * b]);  // e^{-2 pi i b / n}
    // Yhat = E - i w^-b O
    return csub(E, cmuli(cmul(wm, O)));
  };
  for (int m = tid; m <= L; m += NT) {
    const int b = m % n;
    const C Y = (b <= nh) ? Yhat(b) : cconj(Yhat(n - b));
    const C t = tab[f.shift ? m % twon : 0];
    row[m] = cmul(Y, cconj(t));
  }
}

template <typename T, bool BIG>
static int ring_fft_launch(const RingArgs<T>& b, int mode, int cnt, int nt, size_t smem, cudaStream_t st) {
  switch (mode) {
    case 0:
      CR_CUDA(cudaFuncSetAttribute(ring_fft_kernel<T, 0, BIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      { ring_fft_kernel<T, 0, BIG><<<cnt, nt, smem, st>>>(b); count_launch(); }
      break;
    case 1:
      CR_CUDA(cudaFuncSetAttribute(ring_fft_kernel<T, 1, BIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      { ring_fft_kernel<T, 1, BIG><<<cnt, nt, smem, st>>>(b); count_launch(); }
      break;
    default:
      CR_CUDA(cudaFuncSetAttribute(ring_fft_kernel<T, 2, BIG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      { ring_fft_kernel<T, 2, BIG><<<cnt, nt, smem, st>>>(b); count_launch(); }
      break;
  }
  return CR_OK;
}

// One launch per FFT-size class (rings ordered by their FFT size M), each
// with the shared memory and block size its rings need.
template <typename T>
int launch_ring_fft(const RingArgs<T>& a, int mode, cudaStream_t st) {
  using C = typename Tr<T>::C;
  for (int c = 0; c < a.nclass; ++c) {
    const int M = a.cls_M[c];
    const int cnt = a.cls_start[c + 1] - a.cls_start[c];
    if (cnt <= 0) continue;
    const size_t smem = (size_t)M * sizeof(C);
    if (smem > 227 * 1024 || M > 65536) return fail(CR_EINVAL, "ring FFT buffer exceeds shared memory");
    // at least 128 threads: small rings split their folds over the idle lanes
    const int nt = std::max(128, std::min(RF_NT, M / 8));
    RingArgs<T> b = a;
    b.rbase = a.cls_start[c];
    // FP32 rings with M >= 4096: the 4-stage passes with computed twiddles
    int rc;
    if constexpr (sizeof(T) == 4)
      rc = M >= 4096 ? ring_fft_launch<T, true>(b, mode, cnt, nt, smem, st)
                     : ring_fft_launch<T, false>(b, mode, cnt, nt, smem, st);
    else
      rc = ring_fft_launch<T, false>(b, mode, cnt, nt, smem, st);
    if (rc) return rc;
    CR_CHECK_LAUNCH("ring_fft_kernel");
  }
  return CR_OK;
}
template int launch_ring_fft<double>(const RingArgs<double>&, int, cudaStream_t);
template int launch_ring_fft<float>(const RingArgs<float>&, int, cudaStream_t);

// ---------------------------------------------------------------------------
// plan-time tables

struct LenDesc {
  int n, nh, M, logM, bluestein;
  int64_t tab, vhat;
};

__global__ void tab_kernel(const LenDesc* lens, double2* tab) {
  const LenDesc d = lens[blockIdx.x];
  for (int u = threadIdx.x; u < 2 * d.n; u += blockDim.x) {
    double s, c;
    sincospi((double)u / (double)d.n, &s, &c);
    tab[d.tab + u] = make_double2(c, s);
  }
}

__global__ void tw_kernel(double2* tw, int Mmax) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Mmax / 2; j += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)j / (double)Mmax, &s, &c);
    tw[j] = make_double2(c, s);
  }
}

// Bluestein kernel spectrum: v_d = e^{-i pi d^2 / nh}, |d| < nh, wrapped into
// length M, forward FFT, divided by M, kept in bit-reversed order.
__global__ void vhat_kernel(const LenDesc* lens, const double2* tab, const double2* tw, int Mmax, double2* vhat) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* buf = reinterpret_cast<double2*>(smem_raw);
  const LenDesc d = lens[blockIdx.x];
  if (!d.bluestein) return;
  const int64_t twon = 2 * (int64_t)d.n;
  for (int k = threadIdx.x; k < d.M; k += blockDim.x) {
    int dd = -1;
    if (k < d.nh) dd = k;
    else if (k > d.M - d.nh) dd = d.M - k;
    buf[swz(k)] = (dd >= 0) ? cconj(tab[d.tab + (int)((2 * (int64_t)dd * dd) % twon)]) : make_double2(0.0, 0.0);
  }
  __syncthreads();
  fft_dif(buf, d.M, d.logM, -1, tw, Mmax);
  for (int k = threadIdx.x; k < d.M; k += blockDim.x) vhat[d.vhat + k] = cscale(buf[swz(k)], 1.0 / d.M);
}

__global__ void to_f32_kernel(const double2* in, float2* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}
__global__ void to_f32r_kernel(const double* in, float* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

static int ilog2i(int M) {
  int l = 0;
  while ((1 << l) < M) ++l;
  return l;
}

int build_fft_tables(Grid& g, cudaStream_t st) {
  // distinct ring lengths
  std::map<int, int> idx;
  std::vector<LenDesc> lens;
  int64_t tab_len = 0, vhat_len = 0;
  int Mmax = 2;
  for (auto& f : g.fft) {
    if (idx.count(f.n)) continue;
    LenDesc d{};
    d.n = f.n;
    d.nh = f.n / 2;
    const bool p2 = (d.nh & (d.nh - 1)) == 0;
    d.bluestein = p2 ? 0 : 1;
    d.M = p2 ? d.nh : 1;
    if (!p2)
      while (d.M < 2 * d.nh - 1) d.M <<= 1;
    d.logM = ilog2i(d.M);
    d.tab = tab_len;
    tab_len += 2 * (int64_t)d.n;
    d.vhat = vhat_len;
    if (d.bluestein) vhat_len += d.M;
    Mmax = std::max(Mmax, d.M);
    idx[f.n] = (int)lens.size();
    lens.push_back(d);
  }
  for (auto& f : g.fft) {
    const LenDesc& d = lens[idx[f.n]];
    f.nh = d.nh;
    f.M = d.M;
    f.logM = d.logM;
    f.bluestein = d.bluestein;
    f.tab = d.tab;
    f.vhat = d.vhat;
  }
  if ((size_t)Mmax * sizeof(double2) > 227 * 1024) return fail(CR_EINVAL, "ring too long for the shared-memory FFT");
  g.Mmax = Mmax;
  g.tab_len = tab_len;
  g.vhat_len = vhat_len;
  LenDesc* d_lens = nullptr;
  CR_CUDA(cudaMalloc(&d_lens, lens.size() * sizeof(LenDesc)));
  CR_CUDA(cudaMemcpyAsync(d_lens, lens.data(), lens.size() * sizeof(LenDesc), cudaMemcpyHostToDevice, st));
  CR_CUDA(cudaMalloc(&g.d_tab, tab_len * sizeof(double2)));
  CR_CUDA(cudaMalloc(&g.d_tab32, tab_len * sizeof(float2)));
  CR_CUDA(cudaMalloc(&g.d_vhat, std::max<int64_t>(vhat_len, 1) * sizeof(double2)));
  CR_CUDA(cudaMalloc(&g.d_vhat32, std::max<int64_t>(vhat_len, 1) * sizeof(float2)));
  CR_CUDA(cudaMalloc(&g.d_tw, std::max(Mmax / 2, 1) * sizeof(double2)));
  CR_CUDA(cudaMalloc(&g.d_tw32, std::max(Mmax / 2, 1) * sizeof(float2)));
  tab_kernel<<<(int)lens.size(), 256, 0, st>>>(d_lens, g.d_tab);
  CR_CHECK_LAUNCH("tab_kernel");
  tw_kernel<<<std::max(1, std::min(1024, Mmax / 512)), 256, 0, st>>>(g.d_tw, Mmax);
  CR_CHECK_LAUNCH("tw_kernel");
  if (vhat_len > 0) {
    const size_t smem = (size_t)Mmax * sizeof(double2);
    CR_CUDA(cudaFuncSetAttribute(vhat_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    vhat_kernel<<<(int)lens.size(), 256, smem, st>>>(d_lens, g.d_tab, g.d_tw, Mmax, g.d_vhat);
    CR_CHECK_LAUNCH("vhat_kernel");
  }
  to_f32_kernel<<<256, 256, 0, st>>>(g.d_tab, g.d_tab32, tab_len);
  if (vhat_len > 0) to_f32_kernel<<<256, 256, 0, st>>>(g.d_vhat, g.d_vhat32, vhat_len);
  to_f32_kernel<<<64, 256, 0, st>>>(g.d_tw, g.d_tw32, Mmax / 2);
  CR_CHECK_LAUNCH("to_f32_kernel");
  // rings ordered by FFT size; one launch class per distinct size
  {
    std::vector<int> order(g.fft.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return g.fft[x].M < g.fft[y].M; });
    g.cls_M.clear();
    g.cls_start.clear();
    // sizes up to 1024 share one class (their shared memory is small anyway)
    auto key = [&](int r) { return std::max(g.fft[r].M, std::min(1024, Mmax)); };
    for (size_t i = 0; i < order.size(); ++i) {
      if (g.cls_M.empty() || key(order[i]) != g.cls_M.back()) {
        g.cls_M.push_back(key(order[i]));
        g.cls_start.push_back((int)i);
      }
    }
    g.cls_start.push_back((int)order.size());
    CR_CUDA(cudaMalloc(&g.d_rings, order.size() * sizeof(int)));
    CR_CUDA(cudaMemcpyAsync(g.d_rings, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  }
  CR_CUDA(cudaMalloc(&g.d_fft, g.fft.size() * sizeof(RingFFT)));
  CR_CUDA(cudaMemcpyAsync(g.d_fft, g.fft.data(), g.fft.size() * sizeof(RingFFT), cudaMemcpyHostToDevice, st));
  CR_CUDA(cudaStreamSynchronize(st));
  CR_CUDA(cudaFree(d_lens));
  return CR_OK;
}

// Seeds P~_mm(z) = -sqrt((2m+1)/(2m)) sin(theta) P~_{m-1,m-1}, P~_00 = 1/sqrt(4 pi)
// (Section 3.3 normalisation, Condon-Shortley phase), iterated per ring pair
// in FP64 with level tracking, stored [m][pair] for FP64 and FP32.
__global__ void seed_kernel(const double* sth, const double* fac, int Lseed, int npairs, double* seed, int* lev,
                            float* seed32, int* lev32) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const double st = sth[p];
  const double lo = exp2((double)(Tr<double>::THR - Tr<double>::S));
  const double up = exp2((double)Tr<double>::S);
  double v = 0.28209479177387814347;  // 1/sqrt(4 pi)
  int e = 0;
  for (int m = 0; m <= Lseed; ++m) {
    if (m > 0) {
      v = -v * fac[m] * st;
      if (fabs(v) < lo && v != 0.0) {
        v *= up;
        e -= 1;
      }
    }
    const int64_t o = (int64_t)m * npairs + p;
    seed[o] = v;
    lev[o] = e;
    // FP32 representation: true = v 2^(600 e); want v32 in [2^(THR-S), 2^THR)
    float v32 = 0.f;
    int e32 = 0;
    if (v != 0.0) {
      const int E = ilogb(v) + Tr<double>::S * e;
      if (E >= Tr<float>::THR - Tr<float>::S) {
        v32 = (float)ldexp(v, Tr<double>::S * e);
        e32 = 0;
      } else {
        const int k = (Tr<float>::THR - Tr<float>::S - E + Tr<float>::S - 1) / Tr<float>::S;
        v32 = (float)ldexp(v, Tr<double>::S * e + Tr<float>::S * k);
        e32 = -k;
      }
    } else {
      e32 = -1;
    }
    seed32[o] = v32;
    lev32[o] = e32;
  }
}

int build_seeds(Grid& g, int Lseed, cudaStream_t st) {
  std::vector<double> fac(Lseed + 1, 0.0);
  for (int m = 1; m <= Lseed; ++m) fac[m] = std::sqrt((2.0 * m + 1.0) / (2.0 * m));
  double* d_fac = nullptr;
  CR_CUDA(cudaMalloc(&d_fac, (Lseed + 1) * sizeof(double)));
  CR_CUDA(cudaMemcpyAsync(d_fac, fac.data(), (Lseed + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
  const int64_t n = (int64_t)(Lseed + 1) * g.npairs;
  CR_CUDA(cudaMalloc(&g.d_seed, n * sizeof(double)));
  CR_CUDA(cudaMalloc(&g.d_lev, n * sizeof(int)));
  CR_CUDA(cudaMalloc(&g.d_seed32, n * sizeof(float)));
  CR_CUDA(cudaMalloc(&g.d_lev32, n * sizeof(int)));
  seed_kernel<<<(g.npairs + 127) / 128, 128, 0, st>>>(g.d_sth, d_fac, Lseed, g.npairs, g.d_seed, g.d_lev, g.d_seed32,
                                                       g.d_lev32);
  CR_CHECK_LAUNCH("seed_kernel");
  CR_CUDA(cudaStreamSynchronize(st));
  CR_CUDA(cudaFree(d_fac));
  g.Lseed = Lseed;
  return CR_OK;
}

}  // namespace cr
