// Level table, HEALPix nested-scheme tile geometry and the small vector
// kernels of the multi-level cycle (Sections 3.2-3.5).
#include <algorithm>
#include <cmath>
#include <map>
#include <numeric>
#include <tuple>
#include <unordered_map>

#include "common.cuh"
#include "hier.h"
#include "kernels.h"
#include "levels.h"

namespace cr {

int LArr::upload(const std::vector<double>& h) {
  release();
  n = (int)h.size();
  std::vector<float> hf(h.begin(), h.end());
  CR_CUDA(cudaMalloc(&d, std::max<size_t>(1, h.size()) * sizeof(double)));
  CR_CUDA(cudaMalloc(&f, std::max<size_t>(1, h.size()) * sizeof(float)));
  if (!h.empty()) {
    CR_CUDA(cudaMemcpy(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
    CR_CUDA(cudaMemcpy(f, hf.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  return CR_OK;
}

int LArr::assign(const std::vector<double>& h) {
  if (!d || n != (int)h.size() || h.empty()) return upload(h);
  std::vector<float> hf(h.begin(), h.end());
  CR_CUDA(cudaMemcpy(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice));
  CR_CUDA(cudaMemcpy(f, hf.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
  return CR_OK;
}

void LArr::release() {
  if (d) cudaFree(d);
  if (f) cudaFree(f);
  d = nullptr;
  f = nullptr;
  n = 0;
}

// ---------------------------------------------------------------------------
// filters (Section 3.3, Eq. fourth-power-beam) and the level table

std::vector<double> q_filter(int lmax, double ell_star, double value) {
  std::vector<double> q(lmax + 1);
  const double lam = -std::log(value) / (ell_star * ell_star * (ell_star + 1.0) * (ell_star + 1.0));
  for (int l = 0; l <= lmax; ++l) q[l] = std::exp(-(double)l * l * (l + 1.0) * (l + 1.0) * lam);
  return q;
}

std::vector<double> gauss_filter(int lmax, int nside_h) {
  const double fwhm = 2.0 * std::sqrt(4.0 * M_PI / (12.0 * (double)nside_h * nside_h));
  const double s = fwhm / std::sqrt(8.0 * std::log(2.0));
  std::vector<double> g(lmax + 1);
  for (int l = 0; l <= lmax; ++l) g[l] = std::exp(-0.5 * l * (l + 1.0) * s * s);
  return g;
}

// Default levels: the paper's Planck table for Nside 2048 / lmax 3000
// (Table cycle-cost); otherwise pixel levels N_1, N_1/2, ... >= k, where N_1
// is the power of two nearest lmax / 2.93 (the paper's 3000 / 1024, so that
// the top level's high-pass 1 - f^1 only acts on the same noise-dominated
// share of the band) clipped to [k, Nside], with
// lmax_1 = lmax, lmax_2 = min(lmax, 4 Nside_2), lmax_h = min(lmax_{h-1},
// 6 Nside_h); filters: q with q_{2.51 Nside_1} = 0.1, times q with
// q_{3 Nside_2} = 0.1, then Gaussians of FWHM 2 pixels clipped to the level
// above; filter values below 1e-8 are cut and the band limit follows.
int first_level_nside(int nside, int lmax, int k) {
  const double e = std::log2(std::max(1.0, lmax / 2.93));
  int nh = 1 << std::max(0, (int)std::lround(e));
  nh = std::min(nh, nside);
  return std::max(nh, k);
}

void default_levels(int nside, int lmax, int k, std::vector<LevelSpec>& out, int* lmax_dense) {
  out.clear();
  std::vector<std::pair<int, int>> spec;
  const bool planck = (nside == 2048 && lmax == 3000);
  if (planck) {
    spec = {{1024, 3000}, {512, 2048}, {256, 1280}, {128, 768}, {64, 384}, {32, 224}};
  } else {
    for (int nh = first_level_nside(nside, lmax, k); nh >= k; nh /= 2) {
      int lh;
      if (spec.empty()) lh = lmax;
      else if (spec.size() == 1) lh = std::min(lmax, 4 * nh);
      else lh = std::min(spec.back().second, 6 * nh);
      spec.push_back({nh, lh});
    }
  }
  std::vector<double> prev(lmax + 1, 1.0);
  for (size_t i = 0; i < spec.size(); ++i) {
    const int nh = spec[i].first;
    int lh = spec[i].second;
    std::vector<double> f;
    if (i == 0) {
      f = q_filter(lmax, planck ? 2570.0 : 2.51 * nh, 0.1);
    } else if (i == 1) {
      f = q_filter(lmax, planck ? 1536.0 : 3.0 * nh, 0.1);
      for (int l = 0; l <= lmax; ++l) f[l] *= prev[l];
    } else {
      f = gauss_filter(lmax, nh);
      for (int l = 0; l <= lmax; ++l) f[l] = std::min(f[l], prev[l]);
    }
    for (int l = lh + 1; l <= lmax; ++l) f[l] = 0.0;
    for (int l = 0; l <= lmax; ++l)
      if (f[l] < 1e-8) f[l] = 0.0;
    int last = -1;
    for (int l = 0; l <= lmax; ++l)
      if (f[l] > 0.0) last = l;
    lh = std::max(0, std::min(lh, last));
    for (int l = lh + 1; l <= lmax; ++l) f[l] = 0.0;
    LevelSpec s;
    s.nside_h = nh;
    s.lmax_h = lh;
    s.n_rec = 2;
    s.fl = f;
    out.push_back(s);
    prev = f;
  }
  if (!out.empty()) {
    out.back().n_rec = 1;
    *lmax_dense = std::min(40, out.back().lmax_h / 2);
  } else {
    *lmax_dense = std::min(40, lmax);
  }
}

// ---------------------------------------------------------------------------
// HEALPix nested scheme (Gorski et al. 2005)

static const int JRLL[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
static const int JPLL[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};

// Exact integer key of a lattice point (x, y) of face f: its ring coordinate
// jr = jrll N - x - y and azimuth numerator (jpll nr + x - y) mod 8 nr, which
// identify the same sphere point seen from every face that contains it.
static inline std::pair<int64_t, int64_t> vertex_key(int64_t N, int f, int64_t x, int64_t y) {
  const int64_t jr = JRLL[f] * N - x - y;
  int64_t nr;
  if (jr < N) nr = jr;
  else if (jr > 3 * N) nr = 4 * N - jr;
  else nr = N;
  if (nr == 0) return {jr, 0};
  const int64_t M = 8 * nr;
  int64_t num = (JPLL[f] * nr + x - y) % M;
  if (num < 0) num += M;
  return {jr, num};
}

// Tiles = pixels of the Nside_t grid; neighbours share at least one vertex.
void tile_pattern(int nside_t, BlockPattern& P) {
  const int nt = 12 * nside_t * nside_t;
  P.ntile = nt;
  std::map<std::pair<int64_t, int64_t>, std::vector<int>> keys;
  for (int t = 0; t < nt; ++t) {
    int ix, iy, f;
    nest_xyf(nside_t, t, &ix, &iy, &f);
    for (int dx = 0; dx <= 1; ++dx)
      for (int dy = 0; dy <= 1; ++dy) keys[vertex_key(nside_t, f, ix + dx, iy + dy)].push_back(t);
  }
  P.nb.assign(nt, {});
  for (auto& kv : keys)
    for (int t : kv.second)
      for (int u : kv.second) P.nb[t].push_back(u);
  for (auto& v : P.nb) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  }
  // greedy colouring in nested order; order colour-major, then tile index
  std::vector<int> col(nt, -1);
  int ncol = 0;
  for (int t = 0; t < nt; ++t) {
    std::vector<char> used(32, 0);
    for (int u : P.nb[t])
      if (col[u] >= 0 && col[u] < 32) used[col[u]] = 1;
    int c = 0;
    while (used[c]) ++c;
    col[t] = c;
    ncol = std::max(ncol, c + 1);
  }
  P.order.resize(nt);
  std::iota(P.order.begin(), P.order.end(), 0);
  std::stable_sort(P.order.begin(), P.order.end(), [&](int a, int b) { return col[a] < col[b]; });
  P.pos.assign(nt, 0);
  for (int p = 0; p < nt; ++p) P.pos[P.order[p]] = p;
  P.colour_start.assign(ncol + 1, nt);
  for (int p = nt - 1; p >= 0; --p) P.colour_start[col[P.order[p]]] = p;
  P.colour_start[ncol] = nt;
  for (int c = ncol - 1; c >= 0; --c)
    if (P.colour_start[c] > P.colour_start[c + 1]) P.colour_start[c] = P.colour_start[c + 1];
  // rows: blocks (p, q) for neighbouring q < p ascending, then the diagonal
  P.row_ptr.assign(nt + 1, 0);
  P.row_col.clear();
  for (int p = 0; p < nt; ++p) {
    std::vector<int> qs;
    for (int u : P.nb[P.order[p]])
      if (P.pos[u] < p) qs.push_back(P.pos[u]);
    std::sort(qs.begin(), qs.end());
    for (int q : qs) P.row_col.push_back(q);
    P.row_col.push_back(p);
    P.row_ptr[p + 1] = (int64_t)P.row_col.size();
  }
  P.nblocks = (int64_t)P.row_col.size();
}

int64_t BlockPattern::block_of(int p, int q) const {
  const int* b = row_col.data() + row_ptr[p];
  const int* e = row_col.data() + row_ptr[p + 1];
  const int* it = std::lower_bound(b, e, q);
  if (it == e || *it != q) return -1;
  return row_ptr[p] + (it - b);
}

// ---------------------------------------------------------------------------
// vector kernels (one CTA per m; threads over l)

template <typename T>
__global__ void restrict_kernel(const typename Tr<T>::C* in, int Lh, typename Tr<T>::C* out, int LH, const T* ratio) {
  const int m = blockIdx.x;
  const int64_t oh = lm_off(Lh, m), oH = lm_off(LH, m);
  for (int l = m + threadIdx.x; l <= LH; l += blockDim.x) out[oH + l - m] = cscale(in[oh + l - m], ratio[l]);
}

template <typename T>
__global__ void prolong_add_kernel(typename Tr<T>::C* x, int Lh, const typename Tr<T>::C* c, int LH, const T* ratio) {
  const int m = blockIdx.x;
  const int64_t oh = lm_off(Lh, m), oH = lm_off(LH, m);
  for (int l = m + threadIdx.x; l <= LH; l += blockDim.x) {
    typename Tr<T>::C v = x[oh + l - m];
    const typename Tr<T>::C a = c[oH + l - m];
    v.x = fma(ratio[l], a.x, v.x);
    v.y = fma(ratio[l], a.y, v.y);
    x[oh + l - m] = v;
  }
}

// x += d .* r with d indexed like the coefficients (complex storage index)
template <typename T>
__global__ void diag_axpy_kernel(typename Tr<T>::C* x, const typename Tr<T>::C* r, const T* d, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    typename Tr<T>::C v = x[i];
    const typename Tr<T>::C a = r[i];
    v.x = fma(d[i], a.x, v.x);
    v.y = fma(d[i], a.y, v.y);
    x[i] = v;
  }
}

// sum over (l, m) of w_m wl[l] Re(a conj b), w_0 = 1, w_m = 2, accumulated in
// FP64: one partial sum per m, then a fixed-order sum of the partials, so the
// result is bitwise reproducible
template <typename T>
__global__ void dot_kernel(const typename Tr<T>::C* a, const typename Tr<T>::C* b, const double* wl, int L,
                           double* part) {
  const int m = blockIdx.x;
  const int64_t o = lm_off(L, m);
  double s = 0.0;
  for (int l = m + threadIdx.x; l <= L; l += blockDim.x) {
    const typename Tr<T>::C u = a[o + l - m], v = b[o + l - m];
    const double w = wl ? wl[l] : 1.0;
    s += w * ((double)u.x * (double)v.x + (double)u.y * (double)v.y);
  }
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    part[m] = (m == 0 ? 1.0 : 2.0) * t;
  }
}

__global__ void dot_sum_kernel(const double* part, int n, double* out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    *out = t;
  }
}

// deterministic pseudo-random FP32 coefficients in [-1, 1) (integer hash of
// the index), Im(a_l0) = 0: start vectors of the plan-time power iterations
__global__ void fill_random_kernel(float2* v, int L, uint32_t seed) {
  const int m = blockIdx.x;
  const int64_t o = lm_off(L, m);
  for (int l = m + threadIdx.x; l <= L; l += blockDim.x) {
    uint32_t h = (uint32_t)(o + l - m) * 2654435761u ^ seed;
    h ^= h >> 16;
    h *= 2246822519u;
    h ^= h >> 13;
    h *= 3266489917u;
    h ^= h >> 16;
    const float a = (float)(h & 0xffff) / 32768.f - 1.f;
    const float b = (float)(h >> 16) / 32768.f - 1.f;
    v[o + l - m] = make_float2(a, m == 0 ? 0.f : b);
  }
}

template <typename TI, typename TO>
__global__ void convert_kernel(const TI* in, TO* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
}

// x += y (element type TY converted to TX)
template <typename TX, typename TY>
__global__ void add_convert_kernel(TX* x, const TY* y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += (TX)y[i];
}

template <typename T>
int launch_restrict(const void* in, int Lh, void* out, int LH, const T* ratio, cudaStream_t st) {
  { restrict_kernel<T><<<LH + 1, 128, 0, st>>>((const typename Tr<T>::C*)in, Lh, (typename Tr<T>::C*)out, LH, ratio); count_launch(); }
  CR_CHECK_LAUNCH("restrict_kernel");
  return CR_OK;
}
template <typename T>
int launch_prolong_add(void* x, int Lh, const void* c, int LH, const T* ratio, cudaStream_t st) {
  { prolong_add_kernel<T><<<LH + 1, 128, 0, st>>>((typename Tr<T>::C*)x, Lh, (const typename Tr<T>::C*)c, LH, ratio); count_launch(); }
  CR_CHECK_LAUNCH("prolong_add_kernel");
  return CR_OK;
}
template <typename T>
int launch_diag_axpy(void* x, const void* r, const T* d, int64_t n, cudaStream_t st) {
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  { diag_axpy_kernel<T><<<std::max(blocks, 1), 256, 0, st>>>((typename Tr<T>::C*)x, (const typename Tr<T>::C*)r, d, n); count_launch(); }
  CR_CHECK_LAUNCH("diag_axpy_kernel");
  return CR_OK;
}
template <typename T>
int launch_dot(const void* a, const void* b, const double* wl, int L, double* out, double* part, cudaStream_t st) {
  { dot_kernel<T><<<L + 1, 256, 0, st>>>((const typename Tr<T>::C*)a, (const typename Tr<T>::C*)b, wl, L, part); count_launch(); }
  { dot_sum_kernel<<<1, 1024, 0, st>>>(part, L + 1, out); count_launch(); }
  CR_CHECK_LAUNCH("dot_kernel");
  return CR_OK;
}
__global__ void scale_copy_kernel(const float2* in, float2* out, float s, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_float2(in[i].x * s, in[i].y * s);
}

int launch_scale_copy(const void* in, void* out, float s, int64_t n, cudaStream_t st) {
  scale_copy_kernel<<<(int)std::min<int64_t>((n + 255) / 256 + 1, 152 * 8), 256, 0, st>>>((const float2*)in,
                                                                                          (float2*)out, s, n);
  CR_CHECK_LAUNCH("scale_copy_kernel");
  return CR_OK;
}

// y = a x + b y on interleaved complex FP64 vectors of n complex elements
__global__ void axpby_kernel(double2* y, double a, const double2* x, double b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 u = x[i], v = y[i];
    y[i] = make_double2(fma(a, u.x, b * v.x), fma(a, u.y, b * v.y));
  }
}

int launch_axpby(void* y, double a, const void* x, double b, int64_t n, cudaStream_t st) {
  { axpby_kernel<<<(int)std::min<int64_t>((n + 255) / 256 + 1, 152 * 8), 256, 0, st>>>((double2*)y, a, (const double2*)x, b, n); count_launch(); }
  CR_CHECK_LAUNCH("axpby_kernel");
  return CR_OK;
}

int launch_fill_random(void* v, int L, uint32_t seed, cudaStream_t st) {
  fill_random_kernel<<<L + 1, 128, 0, st>>>((float2*)v, L, seed);
  CR_CHECK_LAUNCH("fill_random_kernel");
  return CR_OK;
}

int launch_convert_d2f(const double* in, float* out, int64_t n, cudaStream_t st) {
  { convert_kernel<double, float><<<(int)std::min<int64_t>((n + 255) / 256 + 1, 152 * 8), 256, 0, st>>>(in, out, n); count_launch(); }
  CR_CHECK_LAUNCH("convert_kernel");
  return CR_OK;
}
int launch_add_f2d(double* x, const float* y, int64_t n, cudaStream_t st) {
  { add_convert_kernel<double, float><<<(int)std::min<int64_t>((n + 255) / 256 + 1, 152 * 8), 256, 0, st>>>(x, y, n); count_launch(); }
  CR_CHECK_LAUNCH("add_convert_kernel");
  return CR_OK;
}

template int launch_restrict<double>(const void*, int, void*, int, const double*, cudaStream_t);
template int launch_restrict<float>(const void*, int, void*, int, const float*, cudaStream_t);
template int launch_prolong_add<double>(void*, int, const void*, int, const double*, cudaStream_t);
template int launch_prolong_add<float>(void*, int, const void*, int, const float*, cudaStream_t);
template int launch_diag_axpy<double>(void*, const void*, const double*, int64_t, cudaStream_t);
template int launch_diag_axpy<float>(void*, const void*, const float*, int64_t, cudaStream_t);
template int launch_dot<double>(const void*, const void*, const double*, int, double*, double*, cudaStream_t);
template int launch_dot<float>(const void*, const void*, const double*, int, double*, double*, cudaStream_t);

}  // namespace cr
