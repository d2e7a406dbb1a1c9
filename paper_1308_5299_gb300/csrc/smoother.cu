// Pixel-domain error smoother of one level (Section 3.5): explicit
// A_hat_h = D_hat_h + B_hat_h^T N^-1 B_hat_h inside the tile pattern, its
// zero-fill-in incomplete Cholesky factor with the ridge search, and the
// triangular solves that apply M_hat_h = (L L^T)^-1.  All in FP32 (the paper
// runs its smoothers in single precision).
//
// Tiles are the pixels of the HEALPix grid at Nside_h / k (k = 8, so a tile
// holds 64 NESTED level pixels); a tile couples to the tiles it shares a
// vertex with.  Tiles are eliminated colour by colour (a greedy colouring of
// that neighbour graph), so every colour is a batch of independent tiles:
// one CTA per tile, one launch per colour.
//
// D_hat and B_hat entries come from the addition theorem (Eq.
// addition-theorem) g(theta) = sum_l (2l+1)/(4 pi) g_l P_l(cos theta),
// tabulated once per level in FP64 against the chord d = 2 sin(theta/2) and
// interpolated with 4-point Lagrange polynomials (g is even in d).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <iterator>
#include <vector>


#include "common.cuh"
#include "hier.h"
#include "kernels.h"
#include "levels.h"

namespace cr {

constexpr int TK = 64;        // pixels per tile (k = 8)
constexpr int SM_NT = 256;    // threads of the assembly / factorisation kernels

// ---------------------------------------------------------------------------
// coupling tables

__global__ void coupling_table_kernel(const double* gl, int L, double h, int n, float* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double d = i * h;
  const double x = 1.0 - 0.5 * d * d;
  double p0 = 1.0, p1 = x;
  double s = gl[0] * p0;
  if (L >= 1) s += 3.0 * gl[1] * p1;
  for (int l = 2; l <= L; ++l) {
    const double p2 = ((2.0 * l - 1.0) * x * p1 - (l - 1.0) * p0) / l;
    p0 = p1;
    p1 = p2;
    s += (2.0 * l + 1.0) * gl[l] * p1;
  }
  out[i] = (float)(s / (4.0 * M_PI));
}

struct Table {
  const float* g;
  int n;
  float inv_h;
};

__device__ __forceinline__ float table_eval(const Table& t, float d, int* overflow) {
  const float u = d * t.inv_h;
  int i = (int)u;
  const float f = u - (float)i;
  if (i + 2 >= t.n) {
    *overflow = 1;
    i = t.n - 3;
  }
  const float gm = t.g[i == 0 ? 1 : i - 1];  // g(-h) = g(h)
  const float g0 = t.g[i], g1 = t.g[i + 1], g2 = t.g[i + 2];
  const float wm = -f * (f - 1.f) * (f - 2.f) * (1.f / 6.f);
  const float w0 = (f + 1.f) * (f - 1.f) * (f - 2.f) * 0.5f;
  const float w1 = -(f + 1.f) * f * (f - 2.f) * 0.5f;
  const float w2 = (f + 1.f) * f * (f - 1.f) * (1.f / 6.f);
  return wm * gm + w0 * g0 + w1 * g1 + w2 * g2;
}

// ---------------------------------------------------------------------------
// A_hat assembly: one CTA per stored block (p, q), q <= p.

struct AssembleArgs {
  int nside_h, nside_obs, ratio2;     // ratio2 = obs pixels per tile
  const int* order;                   // position -> nested tile
  const int* blk_p;
  const int* blk_q;
  const int64_t* cobs_ptr;            // per block: common obs tiles (nested)
  const int* cobs;
  const double* ninv;                 // obs grid, RING order
  Table gD, gB;
  int with_d, with_noise;             // which terms to assemble
  const float* base;                  // added to the result (or null)
  float* A;
  int* overflow;
};

__device__ __forceinline__ void tile_pixel_vec(int64_t nside, int64_t nest, double* v) {
  int ix, iy, f;
  nest_xyf(nside, nest, &ix, &iy, &f);
  face_vec((double)nside, f, ix + 0.5, iy + 0.5, v);
}

__global__ void __launch_bounds__(SM_NT) assemble_kernel(AssembleArgs a) {
  const int b = blockIdx.x;
  const int p = a.blk_p[b], q = a.blk_q[b];
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  __shared__ double ref[3];
  __shared__ float3 vp[TK], vq[TK], vo[TK];
  __shared__ float No[TK];
  __shared__ __align__(16) float Bi[TK][TK + 4];
  __shared__ __align__(16) float Bj[TK][TK + 4];
  if (tid == 0) {
    double v[3];
    tile_pixel_vec(a.nside_h, (int64_t)a.order[p] * TK, v);
    ref[0] = v[0];
    ref[1] = v[1];
    ref[2] = v[2];
  }
  __syncthreads();
  if (tid < 2 * TK) {
    const int t = tid & (TK - 1);
    const int tile = (tid < TK) ? a.order[p] : a.order[q];
    double v[3];
    tile_pixel_vec(a.nside_h, (int64_t)tile * TK + t, v);
    const float3 o = make_float3((float)(v[0] - ref[0]), (float)(v[1] - ref[1]), (float)(v[2] - ref[2]));
    if (tid < TK) vp[t] = o;
    else vq[t] = o;
  }
  __syncthreads();
  int myovf = 0;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float3 u = vp[4 * ty + i], w = vq[4 * tx + j];
      const float dx = u.x - w.x, dy = u.y - w.y, dz = u.z - w.z;
      acc[i][j] = a.with_d ? table_eval(a.gD, sqrtf(dx * dx + dy * dy + dz * dz), &myovf) : 0.f;
    }
  const int64_t c_end = a.with_noise ? a.cobs_ptr[b + 1] : a.cobs_ptr[b];
  for (int64_t c = a.cobs_ptr[b]; c < c_end; ++c) {
    const int64_t base = (int64_t)a.cobs[c] * a.ratio2;
    for (int c0 = 0; c0 < a.ratio2; c0 += TK) {
      __syncthreads();
      if (tid < TK) {
        const int64_t nest = base + c0 + tid;
        double v[3];
        tile_pixel_vec(a.nside_obs, nest, v);
        vo[tid] = make_float3((float)(v[0] - ref[0]), (float)(v[1] - ref[1]), (float)(v[2] - ref[2]));
        No[tid] = (float)a.ninv[nest2ring(a.nside_obs, nest)];
      }
      __syncthreads();
      if (!__syncthreads_or(tid < TK && No[tid] != 0.f)) continue;
      for (int e = tid; e < TK * 2 * TK; e += SM_NT) {
        const int o = e >> 7, cc = e & 127;
        const float3 u = vo[o];
        const float3 w = (cc < TK) ? vp[cc] : vq[cc - TK];
        const float dx = u.x - w.x, dy = u.y - w.y, dz = u.z - w.z;
        const float g = table_eval(a.gB, sqrtf(dx * dx + dy * dy + dz * dz), &myovf);
        if (cc < TK) Bi[o][cc] = No[o] * g;
        else Bj[o][cc - TK] = g;
      }
      __syncthreads();
#pragma unroll 4
      for (int o = 0; o < TK; ++o) {
        const float4 x = *reinterpret_cast<const float4*>(&Bi[o][4 * ty]);
        const float4 y = *reinterpret_cast<const float4*>(&Bj[o][4 * tx]);
        const float xa[4] = {x.x, x.y, x.z, x.w}, ya[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xa[i], ya[j], acc[i][j]);
      }
    }
  }
  float* out = a.A + (int64_t)b * TK * TK;
  const float* bas = a.base ? a.base + (int64_t)b * TK * TK : nullptr;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t e = (4 * tx + j) * TK + 4 * ty + i;  // column-major
      out[e] = bas ? acc[i][j] + bas[e] : acc[i][j];
    }
  if (myovf) atomicOr(a.overflow, 1);
}

// symmetrise the diagonal blocks (A_pp = (A_pp + A_pp^T) / 2)
__global__ void symmetrise_diag_kernel(float* A, const int64_t* diag_blk) {
  float* B = A + diag_blk[blockIdx.x] * TK * TK;
  for (int e = threadIdx.x; e < TK * TK; e += blockDim.x) {
    const int i = e % TK, j = e / TK;
    if (i > j) {
      const float s = 0.5f * (B[j * TK + i] + B[i * TK + j]);
      B[j * TK + i] = s;
      B[i * TK + j] = s;
    }
  }
}

__global__ void absmax_kernel(const float* A, int64_t n, unsigned int* out) {
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(A[i]));
  for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// ---------------------------------------------------------------------------
// block ICC(0), one colour per launch, one CTA per tile

struct IccArgs {
  const float* A;
  float* L;
  const int64_t* upd_ptr;
  const int64_t* tgt_blk;
  const int* tgt_u;
  const int64_t* tgt_ptr;
  const int64_t* pair_a;
  const int64_t* pair_b;
  float alpha;
  int* fail;
};

// S -= X Y^T for column-major 64x64 blocks X, Y in global memory, staged
// through shared memory.
__device__ void sub_xyT(float (*S)[TK + 1], const float* X, const float* Y, float (*sx)[TK + 1], float (*sy)[TK + 1]) {
  const int tid = threadIdx.x;
  __syncthreads();
  for (int e = tid; e < TK * TK; e += SM_NT) {
    const int i = e % TK, k = e / TK;
    sx[i][k] = X[e];
    sy[i][k] = Y[e];
  }
  __syncthreads();
  const int ty = tid >> 4, tx = tid & 15;
  float acc[4][4] = {};
  for (int k = 0; k < TK; ++k) {
    float xa[4], ya[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      xa[i] = sx[4 * ty + i][k];
      ya[i] = sy[4 * tx + i][k];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xa[i], ya[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) S[4 * ty + i][4 * tx + j] -= acc[i][j];
}

__global__ void __launch_bounds__(SM_NT) icc_colour_kernel(IccArgs a, int p0) {
  const int p = p0 + blockIdx.x;
  extern __shared__ __align__(16) float sm[];
  float(*S)[TK + 1] = reinterpret_cast<float(*)[TK + 1]>(sm);
  float(*Li)[TK + 1] = reinterpret_cast<float(*)[TK + 1]>(sm + TK * (TK + 1));
  float(*sx)[TK + 1] = reinterpret_cast<float(*)[TK + 1]>(sm + 2 * TK * (TK + 1));
  float(*sy)[TK + 1] = reinterpret_cast<float(*)[TK + 1]>(sm + 3 * TK * (TK + 1));
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int64_t t = a.upd_ptr[p]; t < a.upd_ptr[p + 1]; ++t) {
    const int u = a.tgt_u[t];
    const float* Ab = a.A + a.tgt_blk[t] * TK * TK;
    __syncthreads();
    for (int e = tid; e < TK * TK; e += SM_NT) {
      const int i = e % TK, j = e / TK;
      S[i][j] = Ab[e] + ((u == p && i == j) ? a.alpha : 0.f);
    }
    for (int64_t c = a.tgt_ptr[t]; c < a.tgt_ptr[t + 1]; ++c)
      sub_xyT(S, a.L + a.pair_a[c] * TK * TK, a.L + a.pair_b[c] * TK * TK, sx, sy);
    __syncthreads();
    float* Lb = a.L + a.tgt_blk[t] * TK * TK;
    if (u == p) {
      // Cholesky of S (lower), right-looking
      for (int j = 0; j < TK; ++j) {
        if (tid == 0) {
          const float d = S[j][j];
          if (!(d > 0.f) || !isfinite(d)) bad = 1;
          S[j][j] = sqrtf(fmaxf(d, 1e-30f));
        }
        __syncthreads();
        const float djj = S[j][j];
        for (int i = j + 1 + tid; i < TK; i += SM_NT) S[i][j] /= djj;
        __syncthreads();
        const int m = TK - j - 1;
        for (int e = tid; e < m * m; e += SM_NT) {
          const int i = j + 1 + e % m, k = j + 1 + e / m;
          if (k <= i) S[i][k] -= S[i][j] * S[k][j];
        }
        __syncthreads();
      }
      // inverse of the lower factor, one column per thread
      if (tid < TK) {
        const int c = tid;
        for (int i = 0; i < TK; ++i) {
          float s = (i == c) ? 1.f : 0.f;
          if (i > c)
            for (int k = c; k < i; ++k) s -= S[i][k] * Li[k][c];
          Li[i][c] = (i >= c) ? s / S[i][i] : 0.f;
        }
      }
      __syncthreads();
      for (int e = tid; e < TK * TK; e += SM_NT) {
        const int i = e % TK, j = e / TK;
        Lb[e] = Li[i][j];  // diagonal block stores inv(L_pp)
      }
    } else {
      // L_up = S L_pp^-T = S Li^T
      __syncthreads();
      const int ty = tid >> 4, tx = tid & 15;
      float acc[4][4] = {};
      for (int k = 0; k < TK; ++k) {
        float xa[4], ya[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          xa[i] = S[4 * ty + i][k];
          ya[i] = Li[4 * tx + i][k];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xa[i], ya[j], acc[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) Lb[(4 * tx + j) * TK + 4 * ty + i] = acc[i][j];
    }
  }
  __syncthreads();
  if (tid == 0 && bad) atomicOr(a.fail, 1);
}

// ---------------------------------------------------------------------------
// triangular solves.  y is the tile-ordered work vector (FP32).

// Triangular solves of one colour (tiles of a colour are independent).  One
// CTA of 64 threads per tile: thread (rq, jg) = (tid & 15, tid >> 4) owns rows
// 4 rq .. 4 rq + 3 and the column group j = 16 jg .. 16 jg + 15 of every
// 64 x 64 block, read as float4 rows of the column-major block (coalesced);
// the neighbours' vectors are staged once, the four column groups are summed
// through shared memory.  The diagonal block holds inv(L_pp).
// Forward: y_p = inv(L_pp) (r_p - sum_{q<p} L_pq y_q), blocks of row p.
// Backward: x_p = inv(L_pp)^T (y_p - sum_{u>p} L_up^T x_u), using the
// transposed copies of column p's blocks (LT, built after factorisation).
__device__ __forceinline__ float4 f4fma(float4 a, float s, float4 c) {
  c.x = fmaf(a.x, s, c.x);
  c.y = fmaf(a.y, s, c.y);
  c.z = fmaf(a.z, s, c.z);
  c.w = fmaf(a.w, s, c.w);
  return c;
}

// acc(rows 4 rq..) = sum_k sum_{j in group} B_k(:, j) v_k[j]
__device__ __forceinline__ float4 block_gemv(const float* __restrict__ B, const float* __restrict__ v, int rq,
                                             int jg, float4 acc) {
  const float4* B4 = reinterpret_cast<const float4*>(B);
#pragma unroll 8
  for (int jj = 0; jj < 16; ++jj) {
    const int j = jg * 16 + jj;
    acc = f4fma(__ldg(B4 + j * (TK / 4) + rq), v[j], acc);
  }
  return acc;
}

// sum the four column groups' partials: row i of the result
__device__ __forceinline__ float reduce_groups(float4 acc, float4 (*part)[16], int rq, int jg, int tid) {
  part[jg][rq] = acc;
  __syncthreads();
  const int r = tid >> 2, e = tid & 3;  // thread tid returns row tid: quad tid >> 2, lane tid & 3
  float s = 0.f;
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const float4 v = part[g][r];
    s += (e == 0) ? v.x : (e == 1) ? v.y : (e == 2) ? v.z : v.w;
  }
  __syncthreads();
  return s;
}

template <typename T>
__device__ __forceinline__ void fwd_tile(const float* L, const int64_t* row_ptr, const int* row_col, const int* perm,
                                         const T* map_in, float* y, int p) {
  const int tid = threadIdx.x, rq = tid & 15, jg = tid >> 4;
  __shared__ float vs[8][TK];
  __shared__ float ts[TK];
  __shared__ float4 part[4][16];
  const int64_t b0 = row_ptr[p];
  const int nb = (int)(row_ptr[p + 1] - 1 - b0);  // lower blocks; the last one is the diagonal
  const float r = (float)map_in[perm[(int64_t)p * TK + tid]];
  for (int k = 0; k < nb; ++k) vs[k][tid] = y[(int64_t)row_col[b0 + k] * TK + tid];
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k = 0; k < nb; ++k) acc = block_gemv(L + (b0 + k) * TK * TK, vs[k], rq, jg, acc);
  ts[tid] = r - reduce_groups(acc, part, rq, jg, tid);
  __syncthreads();
  acc = block_gemv(L + (b0 + nb) * TK * TK, ts, rq, jg, make_float4(0.f, 0.f, 0.f, 0.f));
  y[(int64_t)p * TK + tid] = reduce_groups(acc, part, rq, jg, tid);
}

template <typename T>
__device__ __forceinline__ void bwd_tile(const float* LT, const int64_t* col_ptr, const int* col_row, const int* perm,
                                         float* y, T* map_out, int p) {
  const int tid = threadIdx.x, rq = tid & 15, jg = tid >> 4;
  __shared__ float vs[8][TK];
  __shared__ float ts[TK];
  __shared__ float4 part[4][16];
  const int64_t c0 = col_ptr[p];
  const int nc = (int)(col_ptr[p + 1] - c0);
  const float t = y[(int64_t)p * TK + tid];
  for (int k = 0; k < nc; ++k) vs[k][tid] = y[(int64_t)col_row[c0 + k] * TK + tid];
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const float* Lp = LT + (c0 + p) * TK * TK;  // column p's transposed blocks, then inv(L_pp)^T
  for (int k = 0; k < nc; ++k) acc = block_gemv(Lp + (int64_t)k * TK * TK, vs[k], rq, jg, acc);
  ts[tid] = t - reduce_groups(acc, part, rq, jg, tid);
  __syncthreads();
  acc = block_gemv(Lp + (int64_t)nc * TK * TK, ts, rq, jg, make_float4(0.f, 0.f, 0.f, 0.f));
  const float s = reduce_groups(acc, part, rq, jg, tid);
  y[(int64_t)p * TK + tid] = s;
  map_out[perm[(int64_t)p * TK + tid]] = (T)s;
}

template <typename T>
__global__ void __launch_bounds__(TK) fwd_colour_kernel(const float* L, const int64_t* row_ptr, const int* row_col,
                                                        const int* perm, const T* map_in, float* y, int p0) {
  fwd_tile<T>(L, row_ptr, row_col, perm, map_in, y, p0 + blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(TK) bwd_colour_kernel(const float* LT, const int64_t* col_ptr, const int* col_row,
                                                        const int* perm, float* y, T* map_out, int p0) {
  bwd_tile<T>(LT, col_ptr, col_row, perm, y, map_out, p0 + blockIdx.x);
}

// Coarse levels have few tiles per colour, so a colour's latency, not HBM,
// bounds the sweep: there each tile gets 256 threads (16 column groups of 4
// columns), which cuts every thread's chain of dependent loads by four.
constexpr int TKW = 256;

__device__ __forceinline__ float4 block_gemv_w(const float* __restrict__ B, const float* __restrict__ v, int rq,
                                               int jg, float4 acc) {
  const float4* B4 = reinterpret_cast<const float4*>(B);
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    const int j = jg * 4 + jj;
    acc = f4fma(__ldg(B4 + j * (TK / 4) + rq), v[j], acc);
  }
  return acc;
}

// the same product with the block in shared memory (plain loads: the
// read-only global path of block_gemv_w cannot address shared memory)
__device__ __forceinline__ float4 block_gemv_w_smem(const float* B, const float* __restrict__ v, int rq, int jg,
                                                    float4 acc) {
  const float4* B4 = reinterpret_cast<const float4*>(B);
#pragma unroll
  for (int jj = 0; jj < 4; ++jj) {
    const int j = jg * 4 + jj;
    acc = f4fma(B4[j * (TK / 4) + rq], v[j], acc);
  }
  return acc;
}

// rows of the result for threads tid < 64 (sum of the 16 column groups)
__device__ __forceinline__ float reduce_groups_w(float4 acc, float4 (*part)[16], int rq, int jg, int tid) {
  part[jg][rq] = acc;
  __syncthreads();
  float s = 0.f;
  if (tid < TK) {
    const int r = tid >> 2, e = tid & 3;
#pragma unroll
    for (int g = 0; g < 16; ++g) {
      const float4 v = part[g][r];
      s += (e == 0) ? v.x : (e == 1) ? v.y : (e == 2) ? v.z : v.w;
    }
  }
  __syncthreads();
  return s;
}

template <typename T>
__global__ void __launch_bounds__(TKW) fwd_colour_w_kernel(const float* L, const int64_t* row_ptr, const int* row_col,
                                                           const int* perm, const T* map_in, float* y, int p0) {
  const int p = p0 + blockIdx.x;
  const int tid = threadIdx.x, rq = tid & 15, jg = tid >> 4;
  __shared__ float vs[8][TK];
  __shared__ float ts[TK];
  __shared__ float4 part[16][16];
  const int64_t b0 = row_ptr[p];
  const int nb = (int)(row_ptr[p + 1] - 1 - b0);
  for (int e = tid; e < nb * TK; e += TKW) vs[e / TK][e % TK] = y[(int64_t)row_col[b0 + e / TK] * TK + (e % TK)];
  const float r = (tid < TK) ? (float)map_in[perm[(int64_t)p * TK + tid]] : 0.f;
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int k = 0; k < nb; ++k) acc = block_gemv_w(L + (b0 + k) * TK * TK, vs[k], rq, jg, acc);
  const float s1 = reduce_groups_w(acc, part, rq, jg, tid);
  if (tid < TK) ts[tid] = r - s1;
  __syncthreads();
  acc = block_gemv_w(L + (b0 + nb) * TK * TK, ts, rq, jg, make_float4(0.f, 0.f, 0.f, 0.f));
  const float s2 = reduce_groups_w(acc, part, rq, jg, tid);
  if (tid < TK) y[(int64_t)p * TK + tid] = s2;
}

template <typename T>
__global__ void __launch_bounds__(TKW) bwd_colour_w_kernel(const float* LT, const int64_t* col_ptr, const int* col_row,
                                                           const int* perm, float* y, T* map_out, int p0) {
  const int p = p0 + blockIdx.x;
  const int tid = threadIdx.x, rq = tid & 15, jg = tid >> 4;
  __shared__ float vs[8][TK];
  __shared__ float ts[TK];
  __shared__ float4 part[16][16];
  const int64_t c0 = col_ptr[p];
  const int nc = (int)(col_ptr[p + 1] - c0);
  for (int e = tid; e < nc * TK; e += TKW) vs[e / TK][e % TK] = y[(int64_t)col_row[c0 + e / TK] * TK + (e % TK)];
  const float t = (tid < TK) ? y[(int64_t)p * TK + tid] : 0.f;
  __syncthreads();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const float* Lp = LT + (c0 + p) * TK * TK;
  for (int k = 0; k < nc; ++k) acc = block_gemv_w(Lp + (int64_t)k * TK * TK, vs[k], rq, jg, acc);
  const float s1 = reduce_groups_w(acc, part, rq, jg, tid);
  if (tid < TK) ts[tid] = t - s1;
  __syncthreads();
  acc = block_gemv_w(Lp + (int64_t)nc * TK * TK, ts, rq, jg, make_float4(0.f, 0.f, 0.f, 0.f));
  const float s = reduce_groups_w(acc, part, rq, jg, tid);
  if (tid < TK) {
    y[(int64_t)p * TK + tid] = s;
    map_out[perm[(int64_t)p * TK + tid]] = (T)s;
  }
}

// ---------------------------------------------------------------------------
// Both triangular sweeps of one smoother application in ONE persistent,
// cooperatively launched kernel (levels with few tiles per colour, where one
// launch per colour leaves the GPU waiting on launch and load latency).
//
// Work: the host splits the tiles over the CTAs (tile p of colour c goes to
// CTA (p - colour_start[c]) mod gridDim) and writes each CTA's task list --
// its forward tiles colour by colour ascending, then its backward tiles
// colour by colour descending -- with everything a task needs: position,
// sweep, the neighbours its solve reads and its first factor block.  A
// tile's factor blocks are contiguous (row p of L: its lower blocks then
// inv(L_pp); for the backward sweep the transposed column blocks then
// inv(L_pp)^T in LT), so the CTA's whole sequence of 16 KB blocks is known.
//
// Roles: one producer warp streams that sequence into a ring of SF_NS
// shared-memory slots with bulk asynchronous copies (cp.async.bulk; a "full"
// mbarrier per slot counts the bytes, an "empty" one the consumer warps done
// with it), as far ahead as the ring allows; eight consumer warps run the
// tasks: wait for the inputs, multiply the slots' blocks (256 threads per
// 64 x 64 block as in the per-colour kernels), synchronise among themselves
// on a named barrier only.  The consumers never wait for the producer's
// index arithmetic, only for data.
//
// There is no grid-wide barrier between colours: the sweeps run as a data
// flow over the tiles.  flag[p] becomes 2 e + 1 when tile p's forward solve
// is in y and 2 e + 2 when its backward solve is, e being the launch's epoch
// (epoch[0], read by every CTA at its start and advanced by the last CTA to
// leave, so no reset between launches is needed); a task starts when the
// flags of the neighbours its solve reads have reached that value, so a
// tile of colour c waits for its own neighbours only.  Forward
// solves read lower colours only and backward solves higher colours only;
// every CTA takes its forward tasks by ascending and its backward tasks by
// descending colour, and all CTAs are resident (the cooperative launch): so
// the CTAs holding an unfinished forward tile of the lowest such colour --
// or, once none is left, an unfinished backward tile of the highest such
// colour -- are at that task and its inputs are there; the flow cannot
// stall.  The work vector y is read through L2 (ld.global.cg) because other
// SMs wrote it.
//
// Every wait is bounded (slot mbarriers and tile flags): on a timeout the
// CTA records it in *status; the producer waits (bounded) for its copies in
// flight and every role leaves; the CTAs waiting for this CTA's tiles then
// time out too, and the host reports the status as an error.
constexpr int SF_CONS = 256;                        // consumer threads
constexpr int SF_NT = SF_CONS + 32;                 // + the producer warp
constexpr int SF_NS = 12;                           // shared-memory block slots
constexpr int SF_MAXT = 192;                        // tasks per CTA
constexpr int SW_BLOCK_BYTES = TK * TK * (int)sizeof(float);
constexpr uint32_t SW_WAIT = 1u << 22;              // polls per wait (about a second)

struct FlowTask {
  int p, sweep, nb, pad;
  int64_t blk0;   // first factor block (in L for the forward sweep, LT for the backward)
  int nbr[8];     // positions of the neighbours the solve reads
};
static_assert(sizeof(FlowTask) == 56, "FlowTask layout");

struct SweepArgs {
  const float* L;
  const float* LT;
  const int* perm;
  const FlowTask* task;     // all CTAs' task lists, CTA b's at [task_off[b], task_off[b + 1])
  const int* task_off;
  float* y;
  int* flag;                // [ntile]: 2 epoch + 1 forward done, 2 epoch + 2 backward done
  unsigned int* epoch;      // [2]: the launch epoch, CTAs that have left this launch
  int* status;
};

__device__ __forceinline__ uint32_t sw_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void sw_bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sw_smem(mbar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sw_smem(dst)),
      "l"(src), "r"(bytes), "r"(sw_smem(mbar))
      : "memory");
}

__device__ __forceinline__ bool sw_wait(uint64_t* mbar, uint32_t parity) {
  const uint32_t a = sw_smem(mbar);
  for (uint32_t it = 0; it < SW_WAIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void sw_arrive(uint64_t* mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sw_smem(mbar)) : "memory");
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// barrier of the consumer warps (named barrier 1) that also ANDs a predicate
__device__ __forceinline__ bool cons_sync_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(SF_CONS)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void cons_sync() { asm volatile("bar.sync 1, %0;" ::"n"(SF_CONS) : "memory"); }

// rows of the result for consumer threads tid < 64 (sum of the 16 column
// groups), synchronised on the consumers' barrier
__device__ __forceinline__ float reduce_groups_c(float4 acc, float4 (*part)[16], int rq, int jg, int tid) {
  part[jg][rq] = acc;
  cons_sync();
  float s = 0.f;
  if (tid < TK) {
    const int r = tid >> 2, e = tid & 3;
#pragma unroll
    for (int g = 0; g < 16; ++g) {
      const float4 v = part[g][r];
      s += (e == 0) ? v.x : (e == 1) ? v.y : (e == 2) ? v.z : v.w;
    }
  }
  cons_sync();
  return s;
}

template <typename T>
__device__ __forceinline__ void sweep_flow_consumers(const SweepArgs& a, const T* map_in, T* map_out,
                                                     const FlowTask* tk, int nt, unsigned int fbase, const float* slots,
                                                     uint64_t* full, uint64_t* empty, float (*vs)[TK], float* ts,
                                                     float4 (*part)[16], volatile int* s_abort);

template <typename T>
__global__ void __launch_bounds__(SF_NT, 1) sweep_flow_kernel(SweepArgs a, const T* map_in, T* map_out) {
  extern __shared__ __align__(128) unsigned char sw_raw[];
  float* slots = reinterpret_cast<float*>(sw_raw);
  __shared__ uint64_t full[SF_NS], empty[SF_NS];
  __shared__ FlowTask tk[SF_MAXT];
  __shared__ float vs[8][TK];
  __shared__ float ts[TK];
  __shared__ float4 part[16][16];
  __shared__ volatile int s_abort;
  const int tid = threadIdx.x;
  const int t0 = a.task_off[blockIdx.x], nt = a.task_off[blockIdx.x + 1] - t0;
  const unsigned int fbase = 2u * *(volatile unsigned int*)a.epoch;  // modulo 2^32
  // the CTA's task list into shared memory (host-checked: nt <= SF_MAXT)
  for (int i = tid; i < nt * (int)(sizeof(FlowTask) / 4); i += SF_NT)
    reinterpret_cast<int*>(tk)[i] = reinterpret_cast<const int*>(a.task + t0)[i];
  if (tid == 0) {
    s_abort = 0;
    for (int i = 0; i < SF_NS; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sw_smem(&full[i])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sw_smem(&empty[i])), "r"(SF_CONS / 32) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (tid >= SF_CONS) {
    // producer warp: lane 0 streams the blocks of every task in order
    if (tid == SF_CONS) {
      long issued = 0;
      bool ok = true;
      for (int t = 0; t < nt && ok; ++t) {
        const float* base = (tk[t].sweep == 0 ? a.L : a.LT) + tk[t].blk0 * (int64_t)(TK * TK);
        for (int j = 0; j <= tk[t].nb && ok; ++j) {
          const int slot = (int)(issued % SF_NS);
          if (issued >= SF_NS) {
            ok = sw_wait(&empty[slot], (uint32_t)(((issued / SF_NS) - 1) & 1)) && !s_abort;
            if (!ok) break;
          }
          sw_bulk_load(slots + slot * (TK * TK), base + (int64_t)j * (TK * TK), SW_BLOCK_BYTES, &full[slot]);
          ++issued;
        }
      }
      if (!ok) {
        s_abort = 1;
        atomicExch(a.status, 1);
      }
      // every copy still in flight lands in this CTA's shared memory: wait
      // (bounded) for the last phase of each slot before the CTA can leave
      for (long i = issued > SF_NS ? issued - SF_NS : 0; i < issued; ++i)
        sw_wait(&full[i % SF_NS], (uint32_t)((i / SF_NS) & 1));
    }
  } else {
    sweep_flow_consumers<T>(a, map_in, map_out, tk, nt, fbase, slots, full, empty, vs, ts, part, &s_abort);
  }
  // the last CTA to leave advances the epoch for the next launch
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(a.epoch + 1, 1u) == gridDim.x - 1) {
      atomicExch(a.epoch + 1, 0u);
      atomicAdd(a.epoch, 1u);
    }
  }
}

template <typename T>
__device__ __forceinline__ void sweep_flow_consumers(const SweepArgs& a, const T* map_in, T* map_out,
                                                     const FlowTask* tk, int nt, unsigned int fbase, const float* slots,
                                                     uint64_t* full, uint64_t* empty, float (*vs)[TK], float* ts,
                                                     float4 (*part)[16], volatile int* s_abort) {
  const int tid = threadIdx.x;

  // consumer warps
  const int rq = tid & 15, jg = tid >> 4, lane = tid & 31;
  long used = 0;
  bool ok = true;
  auto take = [&]() -> const float* {  // the next block, once it has landed
    const int slot = (int)(used % SF_NS);
    ok = sw_wait(&full[slot], (uint32_t)((used / SF_NS) & 1)) && !*s_abort;
    return slots + slot * (TK * TK);
  };
  auto release = [&]() {  // this warp is done with the current block
    __syncwarp();
    if (lane == 0) sw_arrive(&empty[used % SF_NS]);
    ++used;
  };
  for (int t = 0; t < nt && ok; ++t) {
    const int p = tk[t].p, sweep = tk[t].sweep, nb = tk[t].nb;
    // the tile's own input and output index first: they wait for no tile
    float r = 0.f;
    int pix = 0;
    if (tid < TK) {
      pix = a.perm[(int64_t)p * TK + tid];
      r = sweep == 0 ? (float)map_in[pix] : __ldcg(a.y + (int64_t)p * TK + tid);
    }
    bool w = true;
    if (tid < nb) {
      const int* f = a.flag + tk[t].nbr[tid];
      const unsigned int want = fbase + (unsigned int)sweep + 1u;
      uint32_t it = 0;
      // flags advance by at most a few epochs: compare modulo 2^32
      while ((int)((unsigned int)ld_acquire_gpu(f) - want) < 0) {
        if (++it > SW_WAIT || *s_abort) {
          w = false;
          break;
        }
      }
    }
    ok = cons_sync_and(w);
    if (!ok) break;
    for (int e = tid; e < nb * TK; e += SF_CONS) vs[e / TK][e % TK] = __ldcg(a.y + (int64_t)tk[t].nbr[e / TK] * TK + (e % TK));
    cons_sync();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < nb; ++k) {
      const float* B = take();
      if (!cons_sync_and(ok)) {
        ok = false;
        break;
      }
      acc = block_gemv_w_smem(B, vs[k], rq, jg, acc);
      release();
    }
    if (!ok) break;
    const float s1 = reduce_groups_c(acc, part, rq, jg, tid);
    if (tid < TK) ts[tid] = r - s1;
    const float* D = take();
    ok = cons_sync_and(ok);  // also publishes ts
    if (!ok) break;
    acc = block_gemv_w_smem(D, ts, rq, jg, make_float4(0.f, 0.f, 0.f, 0.f));
    release();
    const float v = reduce_groups_c(acc, part, rq, jg, tid);
    if (tid < TK) {
      a.y[(int64_t)p * TK + tid] = v;
      if (sweep == 1) map_out[pix] = (T)v;
    }
    // publish the tile: every consumer's y stores precede the barrier, and
    // the release store orders them (cumulatively) before the flag
    cons_sync();
    if (tid == 0)
      asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(a.flag + p), "r"(fbase + (unsigned int)sweep + 1u) : "memory");
  }
  if (!ok && tid == 0) {
    *s_abort = 1;
    atomicExch(a.status, 1);
  }
}

// ---------------------------------------------------------------------------
// The triangular sweeps for up to SM_NR right-hand sides at once (the
// batched cycles): every factor block is read once from HBM for all of them
// and multiplied into a 64 x nr panel of vectors -- the fine levels' sweeps,
// HBM-bound for one right-hand side, become a small dense product per block.
// One CTA of 256 threads per tile of a colour: thread (i, g) = (tid & 63,
// tid >> 6) owns row i of right-hand sides 4 g .. 4 g + 3; the block is staged
// in shared memory (coalesced float4 loads) and read by column, the panel of
// the neighbours' vectors is kept transposed [k][j][r] (rows padded to 17, so
// the coalesced global reads along j store without bank conflicts) and read
// as broadcasts.  y: [SM_NR][ntile * 64] at stride ly; maps at stride ld.
constexpr int SM_NR = 16;
constexpr int MR_NT = 256;
constexpr int SM_VP = SM_NR + 1;  // padded panel row
constexpr size_t SM_SMEM = (size_t)(TK * TK + 8 * TK * SM_VP + TK * SM_VP) * sizeof(float);

__device__ __forceinline__ void mr_stage_block(float* Bs, const float* __restrict__ B) {
  const float4* B4 = reinterpret_cast<const float4*>(B);
  float4* S4 = reinterpret_cast<float4*>(Bs);
#pragma unroll
  for (int e = threadIdx.x; e < TK * TK / 4; e += MR_NT) S4[e] = __ldg(B4 + e);
}

// acc[c] += sum_j B(i, j) V[j][4 g + c] with B column-major in Bs
__device__ __forceinline__ void mr_block_panel(const float* Bs, const float* V, int i, int g, float acc[4]) {
#pragma unroll 8
  for (int j = 0; j < TK; ++j) {
    const float b = Bs[j * TK + i];
    const float* v = V + j * SM_VP + 4 * g;
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] = fmaf(b, v[c], acc[c]);
  }
}

template <typename T>
__global__ void __launch_bounds__(MR_NT) fwd_colour_mr_kernel(const float* L, const int64_t* row_ptr,
                                                             const int* row_col, const int* perm, const T* map_in,
                                                             int64_t ld, float* y, int64_t ly, int nr, int p0) {
  extern __shared__ __align__(16) float mr_smem[];
  float* Bs = mr_smem;
  float* vs = Bs + TK * TK;       // [8][TK][SM_VP]
  float* ts = vs + 8 * TK * SM_VP;  // [TK][SM_VP]
  const int p = p0 + blockIdx.x;
  const int tid = threadIdx.x, i = tid & (TK - 1), g = tid >> 6;
  const int64_t b0 = row_ptr[p];
  const int nb = (int)(row_ptr[p + 1] - 1 - b0);
  for (int e = tid; e < nb * SM_NR * TK; e += MR_NT) {
    const int j = e & (TK - 1), r = (e >> 6) & (SM_NR - 1), k = e >> 10;
    vs[(k * TK + j) * SM_VP + r] = r < nr ? y[r * ly + (int64_t)row_col[b0 + k] * TK + j] : 0.f;
  }
  const int pix = perm[(int64_t)p * TK + i];
  float rin[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) rin[c] = (4 * g + c < nr) ? (float)map_in[(4 * g + c) * ld + pix] : 0.f;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k = 0; k < nb; ++k) {
    mr_stage_block(Bs, L + (b0 + k) * TK * TK);
    __syncthreads();  // also publishes the panel on the first pass
    mr_block_panel(Bs, vs + k * TK * SM_VP, i, g, acc);
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) ts[i * SM_VP + 4 * g + c] = rin[c] - acc[c];
  mr_stage_block(Bs, L + (b0 + nb) * TK * TK);
  __syncthreads();
  float out[4] = {0.f, 0.f, 0.f, 0.f};
  mr_block_panel(Bs, ts, i, g, out);
#pragma unroll
  for (int c = 0; c < 4; ++c)
    if (4 * g + c < nr) y[(4 * g + c) * ly + (int64_t)p * TK + i] = out[c];
}

template <typename T>
__global__ void __launch_bounds__(MR_NT) bwd_colour_mr_kernel(const float* LT, const int64_t* col_ptr,
                                                             const int* col_row, const int* perm, float* y,
                                                             int64_t ly, T* map_out, int64_t ld, int nr, int p0) {
  extern __shared__ __align__(16) float mr_smem[];
  float* Bs = mr_smem;
  float* vs = Bs + TK * TK;
  float* ts = vs + 8 * TK * SM_VP;
  const int p = p0 + blockIdx.x;
  const int tid = threadIdx.x, i = tid & (TK - 1), g = tid >> 6;
  const int64_t c0 = col_ptr[p];
  const int nc = (int)(col_ptr[p + 1] - c0);
  for (int e = tid; e < nc * SM_NR * TK; e += MR_NT) {
    const int j = e & (TK - 1), r = (e >> 6) & (SM_NR - 1), k = e >> 10;
    vs[(k * TK + j) * SM_VP + r] = r < nr ? y[r * ly + (int64_t)col_row[c0 + k] * TK + j] : 0.f;
  }
  float tin[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) tin[c] = (4 * g + c < nr) ? y[(4 * g + c) * ly + (int64_t)p * TK + i] : 0.f;
  const float* Lp = LT + (c0 + p) * TK * TK;  // column p's transposed blocks, then inv(L_pp)^T
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k = 0; k < nc; ++k) {
    mr_stage_block(Bs, Lp + (int64_t)k * TK * TK);
    __syncthreads();
    mr_block_panel(Bs, vs + k * TK * SM_VP, i, g, acc);
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) ts[i * SM_VP + 4 * g + c] = tin[c] - acc[c];
  mr_stage_block(Bs, Lp + (int64_t)nc * TK * TK);
  __syncthreads();
  float out[4] = {0.f, 0.f, 0.f, 0.f};
  mr_block_panel(Bs, ts, i, g, out);
  const int pix = perm[(int64_t)p * TK + i];
#pragma unroll
  for (int c = 0; c < 4; ++c)
    if (4 * g + c < nr) {
      y[(4 * g + c) * ly + (int64_t)p * TK + i] = out[c];
      map_out[(4 * g + c) * ld + pix] = (T)out[c];
    }
}

// LT[col_ptr[p] + p + k] = (block (col_row[..], p))^T for column p's entries,
// then LT[col_ptr[p + 1] + p] = (inv(L_pp))^T; one CTA per position p.
__global__ void transpose_blocks_kernel(const float* L, const int64_t* row_ptr, const int64_t* col_ptr,
                                        const int64_t* col_blk, float* LT) {
  const int p = blockIdx.x;
  __shared__ float tile[TK][TK + 1];
  const int64_t c0 = col_ptr[p], c1 = col_ptr[p + 1];
  for (int64_t c = c0; c <= c1; ++c) {
    const int64_t src = (c < c1) ? col_blk[c] : row_ptr[p + 1] - 1;
    const float* S = L + src * TK * TK;
    float* D = LT + (c + p) * TK * TK;
    __syncthreads();
    for (int e = threadIdx.x; e < TK * TK; e += blockDim.x) tile[e / TK][e % TK] = S[e];  // tile[col][row]
    __syncthreads();
    for (int e = threadIdx.x; e < TK * TK; e += blockDim.x) D[e] = tile[e % TK][e / TK];
  }
}

// ---------------------------------------------------------------------------
// host side

template <typename X>
static int upload_vec(X** d, const std::vector<X>& h) {
  CR_CUDA(cudaMalloc(d, std::max<size_t>(1, h.size()) * sizeof(X)));
  if (!h.empty()) CR_CUDA(cudaMemcpy(*d, h.data(), h.size() * sizeof(X), cudaMemcpyHostToDevice));
  return CR_OK;
}

// Assembly inputs kept with the level so that the C_l-dependent numerical
// part (coupling tables, assembly, ridge search) can be redone alone.
struct SmootherBuild {
  int nd = 0;        // coupling-table entries
  double h = 0.0;    // coupling-table spacing in the chord
  // the inverse-noise term of A_hat alone (observation-dependent; it sees
  // the prior only through the set of l with C_l > 0, recorded in an_active)
  float* d_AN = nullptr;
  std::vector<char> an_active;
  int* d_order = nullptr;
  int* d_blk_p = nullptr;
  int* d_blk_q = nullptr;
  int64_t* d_cobs_ptr = nullptr;
  int* d_cobs = nullptr;
  int64_t* d_diag = nullptr;
  float* d_gD = nullptr;
  float* d_gB = nullptr;
  double* d_gl = nullptr;
  int* d_ovf = nullptr;
  unsigned* d_amax = nullptr;
  ~SmootherBuild() {
    void* ptrs[] = {d_order, d_blk_p, d_blk_q, d_cobs_ptr, d_cobs, d_diag, d_gD, d_gB, d_gl, d_ovf, d_amax, d_AN};
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }
};

// ---------------------------------------------------------------------------
// Additive Schwarz smoother without overlap (block Jacobi over tiles): the
// subdomain solve of tile p is (A_hat_pp + alpha I)^-1, formed once per ridge
// (Cholesky in shared memory, inverse of the factor L^-1, then L^-T L^-1) and
// stored as a full symmetric 64 x 64 block at block p of the factor array;
// one launch applies all tiles in parallel.
__global__ void __launch_bounds__(256) schwarz_factor_kernel(const float* A, const int64_t* diag, float alpha,
                                                             float* S, int* fail) {
  const int p = blockIdx.x, tid = threadIdx.x;
  __shared__ float M[TK][TK + 1];
  __shared__ float Li[TK][TK + 1];
  __shared__ int bad;
  const float* Ab = A + diag[p] * TK * TK;  // column-major
  for (int e = tid; e < TK * TK; e += 256) {
    const int i = e % TK, j = e / TK;
    M[i][j] = Ab[e] + (i == j ? alpha : 0.f);
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < TK; ++j) {
    if (tid == 0) {
      const float d = M[j][j];
      if (!(d > 0.f) || !isfinite(d)) bad = 1;
      M[j][j] = sqrtf(fmaxf(d, 1e-30f));
    }
    __syncthreads();
    const float djj = M[j][j];
    for (int i = j + 1 + tid; i < TK; i += 256) M[i][j] /= djj;
    __syncthreads();
    const int m = TK - j - 1;
    for (int e = tid; e < m * m; e += 256) {
      const int i = j + 1 + e % m, k = j + 1 + e / m;
      if (k <= i) M[i][k] -= M[i][j] * M[k][j];
    }
    __syncthreads();
  }
  if (tid < TK) {
    const int c = tid;
    for (int i = 0; i < TK; ++i) {
      float s = (i == c) ? 1.f : 0.f;
      if (i > c)
        for (int k = c; k < i; ++k) s -= M[i][k] * Li[k][c];
      Li[i][c] = (i >= c) ? s / M[i][i] : 0.f;
    }
  }
  __syncthreads();
  float* Sb = S + (int64_t)p * TK * TK;
  for (int e = tid; e < TK * TK; e += 256) {
    const int i = e % TK, j = e / TK;
    float s = 0.f;
    for (int k = max(i, j); k < TK; ++k) s = fmaf(Li[k][i], Li[k][j], s);
    Sb[e] = s;
  }
  if (tid == 0 && bad) atomicOr(fail, 1);
}

template <typename T>
__global__ void __launch_bounds__(TK) schwarz_apply_kernel(const float* S, const int* perm, const T* map_in,
                                                           T* map_out) {
  const int p = blockIdx.x, tid = threadIdx.x, rq = tid & 15, jg = tid >> 4;
  __shared__ float vs[TK];
  __shared__ float4 part[4][16];
  const int pix = perm[(int64_t)p * TK + tid];
  vs[tid] = (float)map_in[pix];
  __syncthreads();
  const float4 acc = block_gemv(S + (int64_t)p * TK * TK, vs, rq, jg, make_float4(0.f, 0.f, 0.f, 0.f));
  map_out[pix] = (T)reduce_groups(acc, part, rq, jg, tid);
}

int factorise(cr_plan* P, PixLevel& lev, float alpha, bool* ok) {
  const BlockPattern& pat = lev.pat;
  if (P->hier && P->hier->smoother_kind == 1) {
    if (!lev.sb) return fail(CR_ESTATE, "smoother: structure not built");
    CR_CUDA(cudaMemsetAsync(lev.d_fail, 0, sizeof(int), P->stream));
    { schwarz_factor_kernel<<<pat.ntile, 256, 0, P->stream>>>(lev.d_A, lev.sb->d_diag, alpha, lev.d_L, lev.d_fail);
      count_launch(); }
    CR_CHECK_LAUNCH("schwarz_factor_kernel");
    int fl = 0;
    CR_CUDA(cudaMemcpyAsync(&fl, lev.d_fail, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
    CR_CUDA(cudaStreamSynchronize(P->stream));
    *ok = (fl == 0);
    return CR_OK;
  }
  IccArgs a;
  a.A = lev.d_A;
  a.L = lev.d_L;
  a.upd_ptr = lev.d_upd_ptr;
  a.tgt_blk = lev.d_tgt_blk;
  a.tgt_u = lev.d_tgt_u;
  a.tgt_ptr = lev.d_tgt_ptr;
  a.pair_a = lev.d_pair_a;
  a.pair_b = lev.d_pair_b;
  a.alpha = alpha;
  a.fail = lev.d_fail;
  const size_t smem = 4 * TK * (TK + 1) * sizeof(float);
  CR_CUDA(cudaFuncSetAttribute(icc_colour_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CR_CUDA(cudaMemsetAsync(lev.d_fail, 0, sizeof(int), P->stream));
  lev.lt_valid = false;
  for (size_t c = 0; c + 1 < pat.colour_start.size(); ++c) {
    const int p0 = pat.colour_start[c], p1 = pat.colour_start[c + 1];
    if (p1 > p0) { icc_colour_kernel<<<p1 - p0, MR_NT, smem, P->stream>>>(a, p0); count_launch(); }
  }
  CR_CHECK_LAUNCH("icc_colour_kernel");
  int fail = 0;
  CR_CUDA(cudaMemcpyAsync(&fail, lev.d_fail, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  CR_CUDA(cudaStreamSynchronize(P->stream));
  *ok = (fail == 0);
  return CR_OK;
}

// Levels with at most SW_MAX_TILES tiles (Nside_h <= 64) run both
// triangular sweeps of a smoother application in one cooperative launch of
// min(SMs, largest colour) CTAs (one per SM: the block slots take most of
// its shared memory); larger levels keep one launch per colour, which is
// faster there (measured at Nside_h 128 and up: the wide colours stream the
// factor at close to the HBM rate).
constexpr int SW_MAX_TILES = 1024;

// Plans the cooperative data-flow sweeps of a level: the grid (at most one
// CTA per SM and no more CTAs than the widest colour has tiles) and every
// CTA's task list.  coop_grid stays 0 (one launch per colour) when the
// sweep mode asks for that, the device cannot launch cooperatively, or a CTA
// would hold more than SF_MAXT tasks.
static int plan_flow(cr_plan* P, PixLevel& lev, const std::vector<int64_t>& col_ptr, const std::vector<int>& col_row) {
  lev.coop_grid = 0;
  const BlockPattern& pat = lev.pat;
  const int mode = P->hier ? P->hier->sweep_mode : 0;
  if ((P->hier && P->hier->smoother_kind == 1) || mode == 1 || (mode == 0 && pat.ntile > SW_MAX_TILES)) return CR_OK;
  int dev = 0, nsm = 0, coop = 0, nb_d = 0, nb_f = 0;
  CR_CUDA(cudaGetDevice(&dev));
  CR_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CR_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return CR_OK;
  const int smem = SF_NS * SW_BLOCK_BYTES;
  CR_CUDA(cudaFuncSetAttribute(sweep_flow_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  CR_CUDA(cudaFuncSetAttribute(sweep_flow_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  CR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_d, sweep_flow_kernel<double>, SF_NT, smem));
  CR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_f, sweep_flow_kernel<float>, SF_NT, smem));
  if (nb_d < 1 || nb_f < 1) return CR_OK;
  const int ncol = (int)pat.colour_start.size() - 1;
  int widest = 0;
  for (int c = 0; c < ncol; ++c) widest = std::max(widest, pat.colour_start[c + 1] - pat.colour_start[c]);
  const int G = std::max(1, std::min(nsm, widest));
  std::vector<FlowTask> tasks;
  std::vector<int> off(G + 1, 0);
  for (int b = 0; b < G; ++b) {
    off[b] = (int)tasks.size();
    for (int sweep = 0; sweep < 2; ++sweep)
      for (int k = 0; k < ncol; ++k) {
        const int c = sweep == 0 ? k : ncol - 1 - k;
        for (int p = pat.colour_start[c] + b; p < pat.colour_start[c + 1]; p += G) {
          FlowTask t{};
          t.p = p;
          t.sweep = sweep;
          if (sweep == 0) {
            t.nb = (int)(pat.row_ptr[p + 1] - 1 - pat.row_ptr[p]);
            t.blk0 = pat.row_ptr[p];
          } else {
            t.nb = (int)(col_ptr[p + 1] - col_ptr[p]);
            t.blk0 = col_ptr[p] + p;
          }
          if (t.nb > 8) return fail(CR_EINVAL, "smoother: a tile with more than 8 neighbours");
          for (int j = 0; j < t.nb; ++j)
            t.nbr[j] = sweep == 0 ? pat.row_col[pat.row_ptr[p] + j] : col_row[col_ptr[p] + j];
          tasks.push_back(t);
        }
      }
    if ((int)tasks.size() - off[b] > SF_MAXT) return CR_OK;
  }
  off[G] = (int)tasks.size();
  CR_CUDA(cudaMalloc(&lev.d_flow_task, tasks.size() * sizeof(FlowTask)));
  CR_CUDA(cudaMemcpy(lev.d_flow_task, tasks.data(), tasks.size() * sizeof(FlowTask), cudaMemcpyHostToDevice));
  int rc = upload_vec(&lev.d_flow_off, off);
  if (rc) return rc;
  lev.coop_grid = G;
  return CR_OK;
}

// Tile pattern, elimination order, ICC update lists, solve lists and the
// assembly index lists of a level (geometry only); allocates A_hat and the
// factor.
int smoother_structure(cr_plan* P, PixLevel& lev) {
  if (lev.k != 8) return fail(CR_EINVAL, "smoother: only k = 8 tiles are supported");
  lev.nside_t = lev.nside_h / lev.k;
  const int nobs = P->obs.nside;
  if (lev.nside_t < 1 || nobs % lev.nside_t) return fail(CR_EINVAL, "smoother: Nside_h / k must divide the obs Nside");
  BlockPattern& pat = lev.pat;
  tile_pattern(lev.nside_t, pat);
  pat.kk = TK;
  const int nt = pat.ntile;
  // per-block (p, q) and common observation tiles
  std::vector<int> blk_p(pat.nblocks), blk_q(pat.nblocks);
  std::vector<int64_t> cobs_ptr(pat.nblocks + 1, 0), diag(nt);
  std::vector<int> cobs;
  for (int p = 0; p < nt; ++p) {
    for (int64_t b = pat.row_ptr[p]; b < pat.row_ptr[p + 1]; ++b) {
      const int q = pat.row_col[b];
      blk_p[b] = p;
      blk_q[b] = q;
      const auto& A = pat.nb[pat.order[p]];
      const auto& B = pat.nb[pat.order[q]];
      std::vector<int> common;
      std::set_intersection(A.begin(), A.end(), B.begin(), B.end(), std::back_inserter(common));
      for (int t : common) cobs.push_back(t);
      cobs_ptr[b + 1] = (int64_t)cobs.size();
    }
    diag[p] = pat.row_ptr[p + 1] - 1;
  }
  // ICC update lists (targets: the diagonal first, then later neighbours u)
  std::vector<int64_t> upd_ptr(nt + 1, 0), tgt_blk, tgt_ptr(1, 0), pair_a, pair_b;
  std::vector<int> tgt_u;
  std::vector<std::vector<int>> later(nt);  // positions u > p coupled to p
  std::vector<std::vector<int>> nbpos(nt);
  for (int p = 0; p < nt; ++p) {
    for (int u : pat.nb[pat.order[p]]) nbpos[p].push_back(pat.pos[u]);
    std::sort(nbpos[p].begin(), nbpos[p].end());
    for (int u : nbpos[p])
      if (u > p) later[p].push_back(u);
  }
  for (int p = 0; p < nt; ++p) {
    std::vector<int> targets(1, p);
    targets.insert(targets.end(), later[p].begin(), later[p].end());
    for (int u : targets) {
      tgt_blk.push_back(pat.block_of(u, p));
      tgt_u.push_back(u);
      // k < p coupled to both u and p
      for (int k : nbpos[p]) {
        if (k >= p) break;
        if (!std::binary_search(nbpos[u].begin(), nbpos[u].end(), k)) continue;
        pair_a.push_back(pat.block_of(u, k));
        pair_b.push_back(pat.block_of(p, k));
      }
      tgt_ptr.push_back((int64_t)pair_a.size());
    }
    upd_ptr[p + 1] = (int64_t)tgt_blk.size();
  }
  // backward-solve column lists: blocks (u, p), u > p
  std::vector<int64_t> col_ptr(nt + 1, 0), col_blk;
  std::vector<int> col_row;
  for (int p = 0; p < nt; ++p) {
    for (int u : later[p]) {
      col_row.push_back(u);
      col_blk.push_back(pat.block_of(u, p));
    }
    col_ptr[p + 1] = (int64_t)col_row.size();
  }
  // every sweep kernel stages the vectors of at most 8 neighbours of a tile
  // (a HEALPix tile has at most 8), below and above it in the order
  for (int p = 0; p < nt; ++p)
    if (pat.row_ptr[p + 1] - 1 - pat.row_ptr[p] > 8 || col_ptr[p + 1] - col_ptr[p] > 8)
      return fail(CR_EINVAL, "smoother: a tile with more than 8 neighbours");
  // tile-ordered level pixel -> RING index
  const int64_t npix_h = 12LL * lev.nside_h * lev.nside_h;
  std::vector<int> perm(npix_h);
  for (int p = 0; p < nt; ++p)
    for (int j = 0; j < TK; ++j) perm[(int64_t)p * TK + j] = (int)nest2ring(lev.nside_h, (int64_t)pat.order[p] * TK + j);

  if (!lev.sb) lev.sb = new SmootherBuild();
  SmootherBuild& sb = *lev.sb;
  int rc = CR_OK;
  if ((rc = upload_vec(&lev.d_perm, perm))) return rc;
  if ((rc = upload_vec(&lev.d_colour_start, pat.colour_start))) return rc;
  if ((rc = upload_vec(&lev.d_row_ptr, pat.row_ptr))) return rc;
  if ((rc = upload_vec(&lev.d_row_col, pat.row_col))) return rc;
  if ((rc = upload_vec(&lev.d_col_ptr, col_ptr))) return rc;
  if ((rc = upload_vec(&lev.d_col_row, col_row))) return rc;
  if ((rc = upload_vec(&lev.d_col_blk, col_blk))) return rc;
  if ((rc = plan_flow(P, lev, col_ptr, col_row))) return rc;
  if ((rc = upload_vec(&lev.d_upd_ptr, upd_ptr))) return rc;
  if ((rc = upload_vec(&lev.d_tgt_blk, tgt_blk))) return rc;
  if ((rc = upload_vec(&lev.d_tgt_u, tgt_u))) return rc;
  if ((rc = upload_vec(&lev.d_tgt_ptr, tgt_ptr))) return rc;
  if ((rc = upload_vec(&lev.d_pair_a, pair_a))) return rc;
  if ((rc = upload_vec(&lev.d_pair_b, pair_b))) return rc;
  if ((rc = upload_vec(&sb.d_order, pat.order))) return rc;
  if ((rc = upload_vec(&sb.d_blk_p, blk_p))) return rc;
  if ((rc = upload_vec(&sb.d_blk_q, blk_q))) return rc;
  if ((rc = upload_vec(&sb.d_cobs_ptr, cobs_ptr))) return rc;
  if ((rc = upload_vec(&sb.d_cobs, cobs))) return rc;
  if ((rc = upload_vec(&sb.d_diag, diag))) return rc;
  CR_CUDA(cudaMalloc(&lev.d_fail, sizeof(int)));
  CR_CUDA(cudaMalloc(&sb.d_ovf, sizeof(int)));
  CR_CUDA(cudaMalloc(&sb.d_amax, sizeof(unsigned)));
  const int64_t nel = pat.nblocks * TK * TK;
  CR_CUDA(cudaMalloc(&lev.d_A, nel * sizeof(float)));
  CR_CUDA(cudaMalloc(&lev.d_L, nel * sizeof(float)));
  CR_CUDA(cudaMalloc(&sb.d_AN, nel * sizeof(float)));

  // coupling tables in the chord d; d_max covers any pixel pair of two
  // vertex-sharing tiles (4 tile radii, measured) with a margin
  double rmax = 0.0;
  for (int t = 0; t < nt; ++t) {
    int ix, iy, f;
    nest_xyf(lev.nside_t, t, &ix, &iy, &f);
    double c[3];
    face_vec(lev.nside_t, f, ix + 0.5, iy + 0.5, c);
    for (int dx = 0; dx <= 1; ++dx)
      for (int dy = 0; dy <= 1; ++dy) {
        double v[3];
        face_vec(lev.nside_t, f, ix + dx, iy + dy, v);
        const double d = std::sqrt((v[0] - c[0]) * (v[0] - c[0]) + (v[1] - c[1]) * (v[1] - c[1]) +
                                   (v[2] - c[2]) * (v[2] - c[2]));
        rmax = std::max(rmax, d);
      }
  }
  const double dmax = std::min(2.0, 4.5 * rmax + 4.0 * std::sqrt(4.0 * M_PI / (12.0 * nobs * nobs)));
  const int Lh = lev.lmax_h;
  sb.h = 2.0 * M_PI / (128.0 * (Lh + 1));
  sb.nd = (int)std::ceil(dmax / sb.h) + 4;
  CR_CUDA(cudaMalloc(&sb.d_gl, (Lh + 1) * sizeof(double)));
  CR_CUDA(cudaMalloc(&sb.d_gD, sb.nd * sizeof(float)));
  CR_CUDA(cudaMalloc(&sb.d_gB, sb.nd * sizeof(float)));
  return CR_OK;
}

// The C_l-dependent numerical part of a level's smoother: coupling tables of
// D_h and B_h, assembly of A_hat, the ridge search and the factorisation.
int smoother_numeric(cr_plan* P, PixLevel& lev, double ridge_factor, int bisections, double fixed_alpha) {
  if (!lev.sb) return fail(CR_ESTATE, "smoother: structure not built");
  SmootherBuild& sb = *lev.sb;
  const BlockPattern& pat = lev.pat;
  const int nt = pat.ntile;
  const int nobs = P->obs.nside;
  const int Lh = lev.lmax_h;
  const double h = sb.h;
  const int nd = sb.nd;
  const int64_t nel = pat.nblocks * TK * TK;
  int rc = CR_OK;
  CR_CUDA(cudaMemsetAsync(sb.d_ovf, 0, sizeof(int), P->stream));
  CR_CUDA(cudaMemsetAsync(sb.d_amax, 0, sizeof(unsigned), P->stream));
  std::vector<double> gD(Lh + 1, 0.0), gB(Lh + 1, 0.0);
  for (int l = 0; l <= Lh; ++l) {
    const double cl = P->h_cl[l];
    if (cl > 0) {
      gD[l] = lev.fl[l] * lev.fl[l] / cl;
      gB[l] = lev.fl[l] * P->h_bl[l];
    }
  }
  CR_CUDA(cudaStreamSynchronize(P->stream));
  CR_CUDA(cudaMemcpy(sb.d_gl, gD.data(), (Lh + 1) * sizeof(double), cudaMemcpyHostToDevice));
  coupling_table_kernel<<<(nd + 127) / 128, 128, 0, P->stream>>>(sb.d_gl, Lh, h, nd, sb.d_gD);
  CR_CUDA(cudaStreamSynchronize(P->stream));
  CR_CUDA(cudaMemcpy(sb.d_gl, gB.data(), (Lh + 1) * sizeof(double), cudaMemcpyHostToDevice));
  coupling_table_kernel<<<(nd + 127) / 128, 128, 0, P->stream>>>(sb.d_gl, Lh, h, nd, sb.d_gB);
  CR_CHECK_LAUNCH("coupling_table_kernel");

  AssembleArgs aa;
  aa.nside_h = lev.nside_h;
  aa.nside_obs = nobs;
  aa.ratio2 = (nobs / lev.nside_t) * (nobs / lev.nside_t);
  aa.order = sb.d_order;
  aa.blk_p = sb.d_blk_p;
  aa.blk_q = sb.d_blk_q;
  aa.cobs_ptr = sb.d_cobs_ptr;
  aa.cobs = sb.d_cobs;
  aa.ninv = P->d_ninv;
  aa.gD = Table{sb.d_gD, nd, (float)(1.0 / h)};
  aa.gB = Table{sb.d_gB, nd, (float)(1.0 / h)};
  aa.overflow = sb.d_ovf;
  auto assemble = [&](bool with_d, bool with_noise, const float* base, float* out) {
    for (int64_t b0 = 0; b0 < pat.nblocks; b0 += (1 << 20)) {
      const int nb = (int)std::min<int64_t>(1 << 20, pat.nblocks - b0);
      AssembleArgs ab = aa;
      ab.with_d = with_d;
      ab.with_noise = with_noise;
      ab.base = base ? base + b0 * TK * TK : nullptr;
      ab.blk_p = sb.d_blk_p + b0;
      ab.blk_q = sb.d_blk_q + b0;
      ab.cobs_ptr = sb.d_cobs_ptr + b0;
      ab.A = out + b0 * TK * TK;
      { assemble_kernel<<<nb, MR_NT, 0, P->stream>>>(ab); count_launch(); }
    }
  };
  // the inverse-noise term B_h Y^T N^-1 Y B_h (observation-dependent) is
  // assembled once and kept; the prior term D_h is added to it for every C_l
  std::vector<char> active(Lh + 1);
  for (int l = 0; l <= Lh; ++l) active[l] = P->h_cl[l] > 0;
  if (sb.an_active != active) {
    TimerScope ts(P->timing, P->stream, "smoother_assemble_noise");
    assemble(false, true, nullptr, sb.d_AN);
    CR_CHECK_LAUNCH("assemble_kernel");
    sb.an_active = active;
  }
  {
    TimerScope ts(P->timing, P->stream, "smoother_assemble_prior");
    assemble(true, false, sb.d_AN, lev.d_A);
    CR_CHECK_LAUNCH("assemble_kernel");
    symmetrise_diag_kernel<<<nt, 256, 0, P->stream>>>(lev.d_A, sb.d_diag);
    CR_CHECK_LAUNCH("symmetrise_diag_kernel");
  }
  int ovf = 0;
  CR_CUDA(cudaMemcpyAsync(&ovf, sb.d_ovf, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  absmax_kernel<<<1024, 256, 0, P->stream>>>(lev.d_A, nel, sb.d_amax);
  unsigned amax_bits = 0;
  CR_CUDA(cudaMemcpyAsync(&amax_bits, sb.d_amax, sizeof(unsigned), cudaMemcpyDeviceToHost, P->stream));
  CR_CUDA(cudaStreamSynchronize(P->stream));
  if (ovf) return fail(CR_EINVAL, "smoother: pixel pair beyond the coupling table (tile geometry bound)");
  float amaxf;
  std::memcpy(&amaxf, &amax_bits, sizeof(float));
  lev.amax = amaxf;

  // ridge search (Section 3.5): smallest alpha letting ICC(0) succeed, used x ridge_factor
  TimerScope ts(P->timing, P->stream, "smoother_icc");
  bool ok = false;
  if (fixed_alpha >= 0.0) {
    lev.alpha = fixed_alpha;
    if ((rc = factorise(P, lev, (float)fixed_alpha, &ok))) return rc;
    if (!ok) return fail(CR_EICC, "smoother: ICC(0) failed with the given ridge");
    return CR_OK;
  }
  if ((rc = factorise(P, lev, 0.f, &ok))) return rc;
  double alpha = 0.0;
  if (!ok) {
    if ((rc = factorise(P, lev, (float)lev.amax, &ok))) return rc;
    if (!ok) return fail(CR_EICC, "smoother: ICC(0) fails even with a ridge of max|A_hat|");
    double lo = std::log(1e-12), hi = 0.0;
    for (int it = 0; it < bisections; ++it) {
      const double mid = 0.5 * (lo + hi);
      if ((rc = factorise(P, lev, (float)(lev.amax * std::exp(mid)), &ok))) return rc;
      if (ok) hi = mid;
      else lo = mid;
    }
    alpha = lev.amax * std::exp(hi);
  }
  lev.alpha = ridge_factor * alpha;
  if ((rc = factorise(P, lev, (float)lev.alpha, &ok))) return rc;
  if (!ok) return fail(CR_EICC, "smoother: final ICC(0) factorisation failed");
  return CR_OK;
}

// the backward sweep's transposed copy of the factor, made on first use
static int ensure_lt(cr_plan* P, PixLevel& lev) {
  if (lev.lt_valid) return CR_OK;
  const BlockPattern& pat = lev.pat;
  if (!lev.d_LT) CR_CUDA(cudaMalloc(&lev.d_LT, (size_t)pat.nblocks * TK * TK * sizeof(float)));
  { transpose_blocks_kernel<<<pat.ntile, 256, 0, P->stream>>>(lev.d_L, lev.d_row_ptr, lev.d_col_ptr, lev.d_col_blk,
                                                                lev.d_LT); count_launch(); }
  CR_CHECK_LAUNCH("transpose_blocks_kernel");
  lev.lt_valid = true;
  return CR_OK;
}

template <typename T>
int apply_smoother(cr_plan* P, PixLevel& lev, T* map_in, T* map_out) {
  const BlockPattern& pat = lev.pat;
  if (P->hier && P->hier->smoother_kind == 1) {
    { schwarz_apply_kernel<T><<<pat.ntile, TK, 0, P->stream>>>(lev.d_L, lev.d_perm, map_in, map_out); count_launch(); }
    CR_CHECK_LAUNCH("schwarz_apply_kernel");
    return CR_OK;
  }
  int rc = ensure_lt(P, lev);
  if (rc) return rc;
  float* y = reinterpret_cast<float*>(P->hier_tile_work);
  const int nc = (int)pat.colour_start.size() - 1;
  if (lev.coop_grid > 0) {
    // both sweeps in one cooperative launch (few tiles per colour)
    SweepArgs sa;
    sa.L = lev.d_L;
    sa.LT = lev.d_LT;
    sa.perm = lev.d_perm;
    sa.task = reinterpret_cast<const FlowTask*>(lev.d_flow_task);
    sa.task_off = lev.d_flow_off;
    sa.y = y;
    sa.flag = P->hier->d_sweep_flag;
    sa.epoch = P->hier->d_sweep_epoch;
    sa.status = P->hier->d_sweep_status;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(lev.coop_grid);
    cfg.blockDim = dim3(SF_NT);
    cfg.dynamicSmemBytes = (size_t)SF_NS * SW_BLOCK_BYTES;
    cfg.stream = P->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    CR_CUDA(cudaLaunchKernelEx(&cfg, sweep_flow_kernel<T>, sa, (const T*)map_in, map_out));
    count_launch();
    return CR_OK;
  }
  // colours with few tiles are latency-bound: they get the 256-thread tiles
  // (coarse levels throughout, and the small leftover colours of the fine
  // levels); wide colours stream the factor with the 64-thread tiles
  auto wide = [&](int c) { return pat.ntile <= 16384 || pat.colour_start[c + 1] - pat.colour_start[c] < 2048; };
  for (int c = 0; c < nc; ++c) {
    const int p0 = pat.colour_start[c], p1 = pat.colour_start[c + 1];
    if (p1 <= p0) continue;
    if (wide(c))
      { fwd_colour_w_kernel<T><<<p1 - p0, TKW, 0, P->stream>>>(lev.d_L, lev.d_row_ptr, lev.d_row_col, lev.d_perm,
                                                             map_in, y, p0); count_launch(); }
    else
      { fwd_colour_kernel<T><<<p1 - p0, TK, 0, P->stream>>>(lev.d_L, lev.d_row_ptr, lev.d_row_col, lev.d_perm, map_in,
                                                          y, p0); count_launch(); }
  }
  CR_CHECK_LAUNCH("fwd_colour_kernel");
  for (int c = nc - 1; c >= 0; --c) {
    const int p0 = pat.colour_start[c], p1 = pat.colour_start[c + 1];
    if (p1 <= p0) continue;
    if (wide(c))
      { bwd_colour_w_kernel<T><<<p1 - p0, TKW, 0, P->stream>>>(lev.d_LT, lev.d_col_ptr, lev.d_col_row, lev.d_perm, y,
                                                             map_out, p0); count_launch(); }
    else
      { bwd_colour_kernel<T><<<p1 - p0, TK, 0, P->stream>>>(lev.d_LT, lev.d_col_ptr, lev.d_col_row, lev.d_perm, y,
                                                          map_out, p0); count_launch(); }
  }
  CR_CHECK_LAUNCH("bwd_colour_kernel");
  return CR_OK;
}
// Device-side wait timeouts of the cooperative sweeps since the last check
// (synchronises the plan's stream; clears the flag).
int sweep_status(cr_plan* P) {
  if (!P->hier || !P->hier->d_sweep_status || P->capturing) return CR_OK;
  int st = 0;
  CR_CUDA(cudaMemcpyAsync(&st, P->hier->d_sweep_status, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  CR_CUDA(cudaStreamSynchronize(P->stream));
  if (!st) return CR_OK;
  CR_CUDA(cudaMemsetAsync(P->hier->d_sweep_status, 0, sizeof(int), P->stream));
  return fail(CR_ECUDA, "pixel smoother: a bounded wait of the cooperative triangular sweeps gave up");
}

template int apply_smoother<double>(cr_plan*, PixLevel&, double*, double*);
template int apply_smoother<float>(cr_plan*, PixLevel&, float*, float*);

// The pixel smoother of one level for nr <= SM_NR maps at once (map_in,
// map_out: [nr][npix_h] at stride ld): the ICC(0) sweeps with every factor
// block read once for all maps; the Schwarz form, and a single map, take
// the one-map path per map.  The tile work vectors of the batch live in
// the hierarchy's batch buffer (ensure_smoother_batch).
template <typename T>
int apply_smoother_mr(cr_plan* P, PixLevel& lev, int nr, const T* map_in, T* map_out, int64_t ld) {
  if (nr < 1 || nr > SM_NR) return fail(CR_EINVAL, "pixel smoother: 1 to 16 maps per call");
  Hierarchy& H = *P->hier;
  if (H.smoother_kind == 1 || nr == 1) {
    for (int r = 0; r < nr; ++r) {
      int rc = apply_smoother<T>(P, lev, const_cast<T*>(map_in) + r * ld, map_out + r * ld);
      if (rc) return rc;
    }
    return CR_OK;
  }
  const BlockPattern& pat = lev.pat;
  const int64_t ly = (int64_t)pat.ntile * TK;
  if (!H.d_mr_y || H.mr_y_len < ly) return fail(CR_ESTATE, "pixel smoother: batch buffer missing");
  int rc = ensure_lt(P, lev);
  if (rc) return rc;
  CR_CUDA(cudaFuncSetAttribute(fwd_colour_mr_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_SMEM));
  CR_CUDA(cudaFuncSetAttribute(bwd_colour_mr_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_SMEM));
  float* y = H.d_mr_y;
  const int nc = (int)pat.colour_start.size() - 1;
  for (int c = 0; c < nc; ++c) {
    const int p0 = pat.colour_start[c], p1 = pat.colour_start[c + 1];
    if (p1 <= p0) continue;
    { fwd_colour_mr_kernel<T><<<p1 - p0, MR_NT, SM_SMEM, P->stream>>>(lev.d_L, lev.d_row_ptr, lev.d_row_col,
                                                                     lev.d_perm, map_in, ld, y, ly, nr, p0); count_launch(); }
  }
  CR_CHECK_LAUNCH("fwd_colour_mr_kernel");
  for (int c = nc - 1; c >= 0; --c) {
    const int p0 = pat.colour_start[c], p1 = pat.colour_start[c + 1];
    if (p1 <= p0) continue;
    { bwd_colour_mr_kernel<T><<<p1 - p0, MR_NT, SM_SMEM, P->stream>>>(lev.d_LT, lev.d_col_ptr, lev.d_col_row,
                                                                     lev.d_perm, y, ly, map_out, ld, nr, p0); count_launch(); }
  }
  CR_CHECK_LAUNCH("bwd_colour_mr_kernel");
  return CR_OK;
}
template int apply_smoother_mr<double>(cr_plan*, PixLevel&, int, const double*, double*, int64_t);
template int apply_smoother_mr<float>(cr_plan*, PixLevel&, int, const float*, float*, int64_t);

// batch buffers of the many-map smoother: tile work vectors and two map
// panels, SM_NR x the largest level
int ensure_smoother_batch(cr_plan* P) {
  Hierarchy& H = *P->hier;
  int64_t need = 0;
  for (const PixLevel& lev : H.pix) need = std::max(need, (int64_t)lev.pat.ntile * TK);
  if (H.d_mr_y && H.mr_y_len >= need) return CR_OK;
  void* q[] = {H.d_mr_y, H.d_mr_m1, H.d_mr_m2};
  for (void* x : q)
    if (x) cudaFree(x);
  H.d_mr_y = H.d_mr_m1 = H.d_mr_m2 = nullptr;
  CR_CUDA(cudaMalloc(&H.d_mr_y, (size_t)SM_NR * need * sizeof(float)));
  CR_CUDA(cudaMalloc(&H.d_mr_m1, (size_t)SM_NR * need * sizeof(float)));
  CR_CUDA(cudaMalloc(&H.d_mr_m2, (size_t)SM_NR * need * sizeof(float)));
  H.mr_y_len = need;
  return CR_OK;
}

void free_smoother(PixLevel& lev) {
  delete lev.sb;
  lev.sb = nullptr;
  void* ptrs[] = {lev.d_A, lev.d_L, lev.d_LT, lev.d_perm, lev.d_colour_start, lev.d_row_ptr, lev.d_row_col,
                  lev.d_col_ptr, lev.d_col_row,
                  lev.d_col_blk, lev.d_upd_ptr, lev.d_tgt_blk, lev.d_tgt_u, lev.d_tgt_ptr, lev.d_pair_a, lev.d_pair_b,
                  lev.d_fail, lev.d_flow_task, lev.d_flow_off};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

}  // namespace cr
