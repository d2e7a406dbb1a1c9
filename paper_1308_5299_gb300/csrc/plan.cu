// Plan construction and the C ABI entry points for transforms and A.
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"
#include "hier.h"
#include "kernels.h"
#include "levels.h"

namespace cr {

static thread_local std::string g_last_error;
static std::atomic<long> g_launches{0};
void count_launch(long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long launch_count() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return CR_ECUDA;
}

cudaEvent_t Timing::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Timing::flush() {
  for (auto& r : pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      auto& v = acc[r.name];
      v.ms += ms;
      v.n += 1;
      v.work += r.work;
      v.work_exec += r.work_exec;
    }
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  pending.clear();
}

Timing::~Timing() {
  for (auto& r : pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : pool) cudaEventDestroy(e);
}

TimerScope::TimerScope(Timing& t, cudaStream_t st, const char* name, double work, double work_exec)
    : TimerScope(t, st, std::string(name), work, work_exec) {}

TimerScope::TimerScope(Timing& t, cudaStream_t st, const std::string& name, double work, double work_exec)
    : t_(&t), st_(st), idx_(-1) {
  if (!t.enabled) return;
  Timing::Rec r{name, t.get(), t.get(), work, work_exec};
  cudaEventRecord(r.a, st);
  t.pending.push_back(r);
  idx_ = (int)t.pending.size() - 1;
}

TimerScope::~TimerScope() {
  if (idx_ >= 0) cudaEventRecord(t_->pending[idx_].b, st_);
}

// HEALPix RING-scheme rings (Gorski et al. 2005): polar ring i < N has 4i
// pixels at z = 1 - i^2/(3N^2), phi = pi (2j + 1) / (4i); equatorial ring
// N <= i <= 3N has 4N pixels at z = 4/3 - 2i/(3N), phi = pi (2j + s) / (4N),
// s = (i - N + 1) mod 2; the south cap mirrors the north.
void healpix_rings(Grid& g, int N) {
  g.kind = CR_GRID_HEALPIX;
  g.nside = N;
  g.nring = 4 * N - 1;
  g.z.resize(g.nring);
  g.sth.resize(g.nring);
  g.fft.resize(g.nring);
  int64_t off = 0;
  for (int i = 1; i <= 4 * N - 1; ++i) {
    const int k = i - 1;
    double z, sth;
    int n, s;
    if (i < N || i > 3 * N) {
      const int ii = (i < N) ? i : 4 * N - i;
      const double omz = (double)ii * ii / (3.0 * N * N);
      z = 1.0 - omz;
      sth = std::sqrt(omz * (2.0 - omz));
      if (i > 3 * N) z = -z;
      n = 4 * ii;
      s = 1;
    } else {
      z = 4.0 / 3.0 - 2.0 * i / (3.0 * N);
      sth = std::sqrt((1.0 - z) * (1.0 + z));
      n = 4 * N;
      s = (i - N + 1) % 2;
    }
    g.z[k] = z;
    g.sth[k] = sth;
    RingFFT f{};
    f.n = n;
    f.shift = s;
    f.off = off;
    g.fft[k] = f;
    off += n;
  }
  g.npix = off;
  g.npairs = (g.nring + 1) / 2;
}

// Gauss-Legendre rings: nodes of P_ntheta by Newton iteration in theta
// (accurate near the poles), nphi pixels per ring at phi = 2 pi j / nphi.
void gl_rings(Grid& g, int ntheta, int nphi, std::vector<double>* weights) {
  g.kind = CR_GRID_GL;
  g.nside = 0;
  g.nring = ntheta;
  g.z.resize(ntheta);
  g.sth.resize(ntheta);
  g.fft.resize(ntheta);
  if (weights) weights->resize(ntheta);
  const int n = ntheta;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double th = M_PI * (i + 0.75) / (n + 0.5);
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      const double x = std::cos(th);
      double p0 = 1.0, p1 = x;
      for (int l = 2; l <= n; ++l) {
        const double p2 = ((2.0 * l - 1.0) * x * p1 - (l - 1.0) * p0) / l;
        p0 = p1;
        p1 = p2;
      }
      // dP_n/dtheta = -sin(theta) dP_n/dx = n (x P_n - P_{n-1}) / sin(theta)... use the
      // identity (1 - x^2) P_n' = n (P_{n-1} - x P_n)
      const double s = std::sin(th);
      const double dPdx = n * (p0 - x * p1) / (s * s);
      const double dPdth = -s * dPdx;
      const double step = p1 / dPdth;
      th -= step;
      dp = dPdx;
      if (std::fabs(step) < 1e-16 * std::max(1.0, th)) {
        // one more derivative evaluation at the converged node
        const double xx = std::cos(th);
        double q0 = 1.0, q1 = xx;
        for (int l = 2; l <= n; ++l) {
          const double q2 = ((2.0 * l - 1.0) * xx * q1 - (l - 1.0) * q0) / l;
          q0 = q1;
          q1 = q2;
        }
        const double ss = std::sin(th);
        dp = n * (q0 - xx * q1) / (ss * ss);
        break;
      }
    }
    const double x = std::cos(th), s = std::sin(th);
    const double w = 2.0 / (s * s * dp * dp);
    g.z[i] = x;
    g.sth[i] = s;
    g.z[n - 1 - i] = -x;
    g.sth[n - 1 - i] = s;
    if (weights) {
      (*weights)[i] = w;
      (*weights)[n - 1 - i] = w;
    }
  }
  int64_t off = 0;
  for (int k = 0; k < n; ++k) {
    RingFFT f{};
    f.n = nphi;
    f.shift = 0;
    f.off = off;
    g.fft[k] = f;
    off += nphi;
  }
  g.npix = off;
  g.npairs = (g.nring + 1) / 2;
}

int grid_upload(Grid& g, int Lseed, cudaStream_t st) {
  std::vector<float> z32(g.z.begin(), g.z.end());
  // FP32 polar form for north rings with z > 1/2 (rings are ordered north to
  // south, so these are the first pairs); 1 - z is exact in FP64 there.
  std::vector<float> w32(g.nring);
  g.npolar32 = 0;
  for (int k = 0; k < g.nring; ++k) {
    w32[k] = (float)(1.0 - g.z[k]);
    if (k < g.npairs && g.z[k] > 0.5) g.npolar32 = k + 1;
  }
  CR_CUDA(cudaMalloc(&g.d_w32, g.nring * sizeof(float)));
  CR_CUDA(cudaMemcpyAsync(g.d_w32, w32.data(), g.nring * sizeof(float), cudaMemcpyHostToDevice, st));
  // pair tables use the north ring of each pair
  CR_CUDA(cudaMalloc(&g.d_z, g.nring * sizeof(double)));
  CR_CUDA(cudaMalloc(&g.d_z32, g.nring * sizeof(float)));
  CR_CUDA(cudaMalloc(&g.d_sth, g.nring * sizeof(double)));
  CR_CUDA(cudaMemcpyAsync(g.d_z, g.z.data(), g.nring * sizeof(double), cudaMemcpyHostToDevice, st));
  CR_CUDA(cudaMemcpyAsync(g.d_z32, z32.data(), g.nring * sizeof(float), cudaMemcpyHostToDevice, st));
  CR_CUDA(cudaMemcpyAsync(g.d_sth, g.sth.data(), g.nring * sizeof(double), cudaMemcpyHostToDevice, st));
  int rc = build_fft_tables(g, st);
  if (rc) return rc;
  return build_seeds(g, Lseed, st);
}

void grid_free(Grid& g) {
  void* ptrs[] = {g.d_z, g.d_z32, g.d_w32, g.d_sth, g.d_fft, g.d_tab, g.d_tab32, g.d_vhat, g.d_vhat32,
                  g.d_tw, g.d_tw32, g.d_seed, g.d_lev, g.d_seed32, g.d_lev32, g.d_ls64, g.d_st64, g.d_ls32,
                  g.d_st32, g.d_st64b, g.d_rings};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

// Recurrence tables for the rescaled recurrence Q_l = c_lm z Q_{l-1} - Q_{l-2},
// P~_lm = s_lm Q_l, derived from the normalised three-term recurrence
// P~_lm = a_lm (z P~_{l-1,m} - P~_{l-2,m} / a_{l-1,m}),
// a_lm = sqrt((4 l^2 - 1) / (l^2 - m^2)):
//   s_l = (a_l / a_{l-1}) s_{l-2},  c_l = a_l s_{l-1} / s_l.
// The even (l - m even) and odd chains of s are independent; s_m = 1 and the
// odd chain is scaled so both chains end at the same value at l = Lc.  Then
// c_l -> 2 for l >> m, so near the poles Q varies slowly in l and c - 2 is
// small, which the FP32 difference form of the recurrence relies on.
static int build_coef(cr_plan* P, int Lc) {
  const int64_t nlm = n_lm(Lc);
  std::vector<double> c(nlm), s(nlm), a(Lc + 1);
  for (int m = 0; m <= Lc; ++m) {
    const int64_t o = lm_off(Lc, m);
    const int K = Lc - m;
    for (int l = m + 1; l <= Lc; ++l) a[l - m] = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
    s[o] = 1.0;
    if (K >= 1) s[o + 1] = 1.0;
    for (int k = 2; k <= K; ++k) s[o + k] = (a[k] / a[k - 1]) * s[o + k - 2];
    if (K >= 2) {
      const int ke = (K % 2 == 0) ? K : K - 1, ko = (K % 2 == 1) ? K : K - 1;
      const double r = s[o + ke] / s[o + ko];
      for (int k = 1; k <= K; k += 2) s[o + k] *= r;
    }
    c[o] = 0.0;
    for (int k = 1; k <= K; ++k) c[o + k] = a[k] * s[o + k - 1] / s[o + k];
  }
  std::vector<float> c32(c.begin(), c.end()), s32(s.begin(), s.end()), c2_32(nlm);
  for (int64_t i = 0; i < nlm; ++i) c2_32[i] = (float)(c[i] - 2.0);
  CR_CUDA(cudaMalloc(&P->d_c, nlm * sizeof(double)));
  CR_CUDA(cudaMalloc(&P->d_s, nlm * sizeof(double)));
  CR_CUDA(cudaMalloc(&P->d_c32, nlm * sizeof(float)));
  CR_CUDA(cudaMalloc(&P->d_s32, nlm * sizeof(float)));
  CR_CUDA(cudaMalloc(&P->d_c2_32, nlm * sizeof(float)));
  CR_CUDA(cudaMemcpy(P->d_c2_32, c2_32.data(), nlm * sizeof(float), cudaMemcpyHostToDevice));
  CR_CUDA(cudaMemcpy(P->d_c, c.data(), nlm * sizeof(double), cudaMemcpyHostToDevice));
  CR_CUDA(cudaMemcpy(P->d_s, s.data(), nlm * sizeof(double), cudaMemcpyHostToDevice));
  CR_CUDA(cudaMemcpy(P->d_c32, c32.data(), nlm * sizeof(float), cudaMemcpyHostToDevice));
  CR_CUDA(cudaMemcpy(P->d_s32, s32.data(), nlm * sizeof(float), cudaMemcpyHostToDevice));
  P->Lcoef = Lc;
  return CR_OK;
}

// Recurrence tables for a larger band limit (the plan's transforms at any
// L <= Lc keep working: the layout is off_m(Lc) + l - m).
int rebuild_coef(cr_plan* P, int Lc) {
  float** f[] = {&P->d_c32, &P->d_c2_32, &P->d_s32};
  for (float** q : f) {
    if (*q) cudaFree(*q);
    *q = nullptr;
  }
  if (P->d_c) cudaFree(P->d_c);
  if (P->d_s) cudaFree(P->d_s);
  P->d_c = P->d_s = nullptr;
  return build_coef(P, Lc);
}

// Legendre seeds of a grid for a larger band limit.
int grid_reseed(Grid& g, int Lseed, cudaStream_t st) {
  CR_CUDA(cudaStreamSynchronize(st));
  void* ptrs[] = {g.d_seed, g.d_lev, g.d_seed32, g.d_lev32, g.d_ls64, g.d_st64, g.d_ls32, g.d_st32, g.d_st64b};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  g.d_seed = nullptr;
  g.d_lev = nullptr;
  g.d_seed32 = nullptr;
  g.d_lev32 = nullptr;
  g.d_ls64 = nullptr;
  g.d_st64 = nullptr;
  g.d_ls32 = nullptr;
  g.d_st32 = nullptr;
  g.d_st64b = nullptr;
  return build_seeds(g, Lseed, st);
}

int ensure_workspace(cr_plan* P, const Grid& g, int L) {
  const int64_t phase = (int64_t)g.nring * (L + 1) * (int64_t)sizeof(double2);
  const int64_t partial = (int64_t)leg_partial_blocks(g.npairs) * n_lm(L) * (int64_t)sizeof(double2);
  if (phase > P->ws.phase_bytes) {
    if (P->ws.phase) cudaFree(P->ws.phase);
    P->ws.phase = nullptr;
    CR_CUDA(cudaMalloc(&P->ws.phase, phase));
    P->ws.phase_bytes = phase;
  }
  if (partial > P->ws.partial_bytes) {
    if (P->ws.partial) cudaFree(P->ws.partial);
    P->ws.partial = nullptr;
    CR_CUDA(cudaMalloc(&P->ws.partial, partial));
    P->ws.partial_bytes = partial;
  }
  return CR_OK;
}

static void plan_free(cr_plan* P) {
  free_hierarchy(P);
  grid_free(P->obs);
  for (Grid* g : P->level_grids) {
    grid_free(*g);
    delete g;
  }
  void* ptrs[] = {P->d_c, P->d_s, P->d_c32, P->d_c2_32, P->d_s32, P->d_bl, P->d_sinv, P->d_bl32, P->d_sinv32,
                  P->d_ninv, P->d_ninv32, P->ws.phase, P->ws.partial, P->ws_mr.phase, P->ws_mr.partial, P->d_tc_r64, P->d_pcinv,
                  P->cgv[0], P->cgv[1],
                  P->cgv[2], P->cgv[3], P->d_cgdot, P->tc_phase, P->d_tc_status, P->tc_partial, P->d_dotpart};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

__global__ void ninv32_kernel(const double* in, float* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// ---- transform drivers ------------------------------------------------------

// Choices of the Legendre autotuner: ring pairs per thread (2, 4 or 8, the
// ring-block size of one CTA) per (grid shape, band limit, precision,
// stage 0 synthesis / 1 adjoint), kept for the process and shared by every
// plan with the same shapes; 4 where nothing was tuned.
struct TuneKey {
  int nring;
  int64_t npix;
  int L, bytes, stage;
  bool operator<(const TuneKey& o) const {
    if (nring != o.nring) return nring < o.nring;
    if (npix != o.npix) return npix < o.npix;
    if (L != o.L) return L < o.L;
    if (bytes != o.bytes) return bytes < o.bytes;
    return stage < o.stage;
  }
};
struct TuneVal {
  int rp;
  int mt;         // m tile: 1 (one m per CTA) or 2 (m and L - m per CTA)
  double ms[8];   // measured ms for 2, 4, 8, 16 pairs per thread, m tile 1 then 2 (-1: not a choice)
};

// 16 ring pairs per thread exist for the packed FP32 adjoint only
static bool rp_allowed(int rp, int bytes, int stage) {
  return rp == 2 || rp == 4 || rp == 8 || (rp == 16 && bytes == 4 && stage == 1);
}
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneVal> g_tune;

// the cached (pairs per thread, m tile) of a stage; (4, 1) when not tuned
static void tuned_shape(const Grid& g, int L, int bytes, int stage, int* rp, int* mt) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(TuneKey{g.nring, g.npix, L, bytes, stage});
  *rp = it == g_tune.end() ? 4 : it->second.rp;
  *mt = it == g_tune.end() ? 1 : it->second.mt;
}

// Tensor-core stage shapes are cached under precision 2 (BF16 operands),
// stage 2 (batched synthesis); the value is the shape variant of
// launch_tc_synth (default 2: K 16 per parity, 3 stages)
constexpr int TC_TUNE_BYTES = 2, TC_TUNE_SYNTH = 2, TC_NVARIANT = 3, TC_DEFAULT_VARIANT = 2;
static int tuned_tc(const Grid& g, int L) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(TuneKey{g.nring, g.npix, L, TC_TUNE_BYTES, TC_TUNE_SYNTH});
  return it == g_tune.end() ? TC_DEFAULT_VARIANT : it->second.rp;
}

template <typename T>
static LegArgs<T> leg_args(cr_plan* P, const Grid& g, int L) {
  LegArgs<T> a;
  tuned_shape(g, L, (int)sizeof(T), 0, &a.rp_synth, &a.mt_synth);
  tuned_shape(g, L, (int)sizeof(T), 1, &a.rp_adj, &a.mt_adj);
  a.tc_split = P->tc_split;
  a.tc_variant = tuned_tc(g, L);
  a.ldp = L + 1;
  a.L = L;
  a.Lc = P->Lcoef;
  if constexpr (sizeof(T) == 8) {
    a.c = P->d_c;
    a.s = P->d_s;
    a.z = g.d_z;
    // FP64 starts where |P~_lm| first reaches 2^-60 (the FP32 start table,
    // with the FP64 state there): the terms left out are below 1e-18 of the
    // largest and decay geometrically away from the start
    a.ls = g.d_ls32;
    a.st = g.d_st64b;
    a.npolar = 0;
    a.df = P->fp64_df;
    a.ls_df = g.d_ls32;
    a.st_df = g.d_st64b;
    a.npolar_df = g.npolar32;
  } else {
    a.c = P->d_c32;
    a.c2 = P->d_c2_32;
    a.s = P->d_s32;
    a.z = g.d_z32;
    a.w = g.d_w32;
    a.npolar = g.npolar32;
    a.ls = g.d_ls32;
    a.st = g.d_st32;
  }
  a.ld_seed = g.npairs;
  a.npairs = g.npairs;
  a.nring = g.nring;
  a.phase = reinterpret_cast<typename Tr<T>::C*>(P->ws.phase);
  a.partial = reinterpret_cast<typename Tr<T>::C*>(P->ws.partial);
  return a;
}

template <typename T>
static RingArgs<T> ring_args(cr_plan* P, const Grid& g, int L) {
  RingArgs<T> r;
  r.fft = g.d_fft;
  if constexpr (sizeof(T) == 8) {
    r.tab = g.d_tab;
    r.vhat = g.d_vhat;
    r.tw = g.d_tw;
  } else {
    r.tab = g.d_tab32;
    r.vhat = g.d_vhat32;
    r.tw = g.d_tw32;
  }
  r.Mmax = g.Mmax;
  r.rings = g.d_rings;
  r.nclass = (int)g.cls_M.size();
  r.cls_M = g.cls_M.data();
  r.cls_start = g.cls_start.data();
  r.phase = reinterpret_cast<typename Tr<T>::C*>(P->ws.phase);
  r.ldp = L + 1;
  r.L = L;
  r.nring = g.nring;
  return r;
}

template <typename T>
static const char* ptag() {
  return sizeof(T) == 8 ? "_f64" : "_f32";
}
// algorithmic flops of one Legendre stage on grid g at band limit L (the
// dense count: every ring pair and (l, m))
static double leg_work(const Grid& g, int L) { return 8.0 * g.npairs * (double)n_lm(L); }

// flops of the terms one Legendre stage evaluates: 8 per (ring pair, l, m)
// at or past the (m, pair)'s start in the 2^-60 start table, which both
// precisions use.  Counted once per (grid, band limit) from the table on the
// host while timing is on (it synchronises, so not inside a graph capture,
// where the dense count stands in).
static double leg_work_exec(cr_plan* P, const Grid& gc, int L) {
  if (!P->timing.enabled || L < 0) return 0.0;
  Grid& g = const_cast<Grid&>(gc);
  auto it = g.exec_terms.find(L);
  if (it != g.exec_terms.end()) return 8.0 * it->second;
  if (P->capturing || !g.d_ls32 || L > g.Lseed) return leg_work(g, L);
  std::vector<int> ls((size_t)(L + 1) * g.npairs);
  if (cudaStreamSynchronize(P->stream) != cudaSuccess ||
      cudaMemcpy(ls.data(), g.d_ls32, ls.size() * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return leg_work(g, L);
  double n = 0.0;
  for (int m = 0; m <= L; ++m) {
    const int* row = ls.data() + (size_t)m * g.npairs;
    int64_t s = 0;
    for (int p = 0; p < g.npairs; ++p)
      if (row[p] <= L) s += L + 1 - row[p];
    n += (double)s;
  }
  g.exec_terms[L] = n;
  return 8.0 * n;
}
// algorithmic HBM bytes of one ring-FFT stage: the phase array [nring][L+1]
// once, plus `maps` pixel arrays of T (map in or out, pixel diagonal, copy)
template <typename T>
static double fft_bytes(const Grid& g, int L, int maps) {
  return (double)g.nring * (L + 1) * sizeof(typename Tr<T>::C) + (double)maps * g.npix * sizeof(T);
}

template <typename T>
int do_synth(cr_plan* P, const Grid& g, int L, const void* alm, void* map, const T* dl) {
  LegArgs<T> a = leg_args<T>(P, g, L);
  a.alm = reinterpret_cast<const typename Tr<T>::C*>(alm);
  a.dl = dl;
  int rc;
  {
    TimerScope ts(P->timing, P->stream, std::string("legendre_synth") + ptag<T>(), leg_work(g, L),
                  leg_work_exec(P, g, L));
    rc = launch_leg_synth<T>(a, P->stream);
  }
  if (rc) return rc;
  RingArgs<T> r = ring_args<T>(P, g, L);
  r.map_out = reinterpret_cast<T*>(map);
  TimerScope ts(P->timing, P->stream, std::string("ring_fft_synth") + ptag<T>(), fft_bytes<T>(g, L, 1));
  return launch_ring_fft<T>(r, 0, P->stream);
}

template <typename T>
int do_adjoint(cr_plan* P, const Grid& g, int L, const void* map, void* alm, const T* dl_out, const T* dadd,
               const void* xadd, int accumulate) {
  RingArgs<T> r = ring_args<T>(P, g, L);
  r.map_in = reinterpret_cast<const T*>(map);
  int rc;
  {
    TimerScope ts(P->timing, P->stream, std::string("ring_fft_adjoint") + ptag<T>(), fft_bytes<T>(g, L, 1));
    rc = launch_ring_fft<T>(r, 1, P->stream);
  }
  if (rc) return rc;
  LegArgs<T> a = leg_args<T>(P, g, L);
  FinalizeArgs<T> f;
  f.dl_out = dl_out;
  f.dadd = dadd;
  f.xadd = reinterpret_cast<const typename Tr<T>::C*>(xadd);
  f.accumulate = accumulate;
  f.out = reinterpret_cast<typename Tr<T>::C*>(alm);
  TimerScope ts(P->timing, P->stream, std::string("legendre_adjoint") + ptag<T>(), leg_work(g, L),
                  leg_work_exec(P, g, L));
  return launch_leg_adjoint<T>(a, f, P->stream);
}

// y = dl_out Y^T diag(pix) Y (dl_in x) + dadd x  on grid g at band limit L
// (or y = bsub - that, when bsub is given).
template <typename T>
int do_sandwich(cr_plan* P, const Grid& g, int L, const void* x, void* y, const T* dl_in, const T* pix,
                const T* dl_out, const T* dadd, T* map_copy, const void* bsub) {
  LegArgs<T> a = leg_args<T>(P, g, L);
  a.alm = reinterpret_cast<const typename Tr<T>::C*>(x);
  a.dl = dl_in;
  int rc;
  {
    TimerScope ts(P->timing, P->stream, std::string("legendre_synth") + ptag<T>(), leg_work(g, L),
                  leg_work_exec(P, g, L));
    rc = launch_leg_synth<T>(a, P->stream);
  }
  if (rc) return rc;
  RingArgs<T> r = ring_args<T>(P, g, L);
  r.pixdiag = pix;
  r.map_out = map_copy;
  {
    // phase read and written back, pixel diagonal read (+ the map copy)
    TimerScope ts(P->timing, P->stream, std::string("ring_fft_apply") + ptag<T>(),
                  fft_bytes<T>(g, L, map_copy ? 2 : 1) + (double)g.nring * (L + 1) * sizeof(typename Tr<T>::C));
    rc = launch_ring_fft<T>(r, 2, P->stream);
  }
  if (rc) return rc;
  FinalizeArgs<T> f;
  f.dl_out = dl_out;
  f.dadd = dadd;
  f.xadd = reinterpret_cast<const typename Tr<T>::C*>(x);
  f.bsub = reinterpret_cast<const typename Tr<T>::C*>(bsub);
  f.out = reinterpret_cast<typename Tr<T>::C*>(y);
  TimerScope ts(P->timing, P->stream, std::string("legendre_adjoint") + ptag<T>(), leg_work(g, L),
                  leg_work_exec(P, g, L));
  return launch_leg_adjoint<T>(a, f, P->stream);
}

// FP64 y_r = dl_out Y^T diag(pix) Y (dl_in x_r) + dadd x_r (or bsub_r - that)
// for nr <= 8 right-hand sides at stride n_lm(L): the two Legendre stages of
// all of them at once (legendre_mr.cu), the ring FFTs and the finalisation
// per right-hand side.  The phase slots and partial rows of the batch live
// in ws_mr.
int ensure_mr_workspace(cr_plan* P, const Grid& g, int L) {
  const int64_t nlm = n_lm(L), ld_phase = (int64_t)g.nring * (L + 1);
  const int nblk = mr_blocks(g.npairs);
  const int64_t phase = 8 * ld_phase * (int64_t)sizeof(double2);
  const int64_t partial = 8 * (int64_t)nblk * nlm * (int64_t)sizeof(double2);
  if (phase > P->ws_mr.phase_bytes || partial > P->ws_mr.partial_bytes) {
    if (P->capturing) return fail(CR_ESTATE, "FP64 batch: buffers missing (run once outside a capture)");
    if (phase > P->ws_mr.phase_bytes) {
      if (P->ws_mr.phase) cudaFree(P->ws_mr.phase);
      P->ws_mr.phase = nullptr;
      CR_CUDA(cudaMalloc(&P->ws_mr.phase, phase));
      P->ws_mr.phase_bytes = phase;
    }
    if (partial > P->ws_mr.partial_bytes) {
      if (P->ws_mr.partial) cudaFree(P->ws_mr.partial);
      P->ws_mr.partial = nullptr;
      CR_CUDA(cudaMalloc(&P->ws_mr.partial, partial));
      P->ws_mr.partial_bytes = partial;
    }
  }
  return CR_OK;
}

int do_sandwich_mr(cr_plan* P, const Grid& g, int L, int nr, const double2* x, double2* y, const double* dl_in,
                   const double* pix, const double* dl_out, const double* dadd, const double2* bsub) {
  if (nr < 1 || nr > 8) return fail(CR_EINVAL, "FP64 batch: 1 to 8 right-hand sides");
  int rc = ensure_mr_workspace(P, g, L);
  if (rc) return rc;
  const int64_t nlm = n_lm(L), ld_phase = (int64_t)g.nring * (L + 1);
  double2* ph = reinterpret_cast<double2*>(P->ws_mr.phase);
  double2* part = reinterpret_cast<double2*>(P->ws_mr.partial);
  LegArgs<double> a = leg_args<double>(P, g, L);
  a.dl = dl_in;
  {
    TimerScope ts(P->timing, P->stream, "legendre_synth_f64", leg_work(g, L) * nr, leg_work_exec(P, g, L) * nr);
    rc = launch_leg_synth_mr(a, x, nlm, nr, ph, ld_phase, P->stream);
  }
  for (int r = 0; r < nr && !rc; ++r) {
    RingArgs<double> ra = ring_args<double>(P, g, L);
    ra.phase = ph + r * ld_phase;
    ra.pixdiag = pix;
    TimerScope ts(P->timing, P->stream, "ring_fft_apply_f64",
                  fft_bytes<double>(g, L, 1) + (double)g.nring * (L + 1) * sizeof(double2));
    rc = launch_ring_fft<double>(ra, 2, P->stream);
  }
  if (rc) return rc;
  int nb = 0;
  {
    TimerScope ts(P->timing, P->stream, "legendre_adjoint_f64", leg_work(g, L) * nr, leg_work_exec(P, g, L) * nr);
    rc = launch_leg_adjoint_mr(a, ph, ld_phase, nr, part, &nb, P->stream);
  }
  for (int r = 0; r < nr && !rc; ++r) {
    FinalizeArgs<double> f;
    f.partial = part + (int64_t)r * nb * nlm;
    f.nblk = nb;
    f.L = L;
    f.dl_out = dl_out;
    f.dadd = dadd;
    f.xadd = x + r * nlm;
    f.bsub = bsub ? bsub + r * nlm : nullptr;
    f.out = y + r * nlm;
    rc = launch_leg_finalize<double>(f, P->stream);
  }
  return rc;
}

template int do_synth<double>(cr_plan*, const Grid&, int, const void*, void*, const double*);
template int do_synth<float>(cr_plan*, const Grid&, int, const void*, void*, const float*);
template int do_adjoint<double>(cr_plan*, const Grid&, int, const void*, void*, const double*, const double*,
                                const void*, int);
template int do_adjoint<float>(cr_plan*, const Grid&, int, const void*, void*, const float*, const float*,
                               const void*, int);
template int do_sandwich<double>(cr_plan*, const Grid&, int, const void*, void*, const double*, const double*,
                                 const double*, const double*, double*, const void*);
template int do_sandwich<float>(cr_plan*, const Grid&, int, const void*, void*, const float*, const float*,
                                const float*, const float*, float*, const void*);

static const Grid* grid_of(cr_plan* P, int grid, int* L) {
  if (grid == CR_OBS) {
    *L = P->lmax;
    return &P->obs;
  }
  const int h = grid - CR_OBS;
  if (h >= 1 && h <= (int)P->level_grids.size()) {
    *L = P->levels[h].lmax_h;
    return P->level_grids[h - 1];
  }
  return nullptr;
}

// Time one Legendre stage of grid g at band limit L for 2, 4 and 8 ring
// pairs per thread (16 for the FP32 adjoint), each with one m per CTA and
// with m paired with L - m (one untimed launch, then `reps` timed with CUDA
// events on the plan's stream; native kernels, zero coefficients -- the work
// does not depend on the data) and record the fastest shape.
template <typename T>
static int tune_stage(cr_plan* P, const Grid& g, int L, int stage, int reps) {
  using C = typename Tr<T>::C;
  int rc = ensure_workspace(P, g, L);
  if (rc) return rc;
  C* alm = nullptr;
  CR_CUDA(cudaMalloc(&alm, n_lm(L) * sizeof(C)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemsetAsync(alm, 0, n_lm(L) * sizeof(C), P->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) rc = cuda_fail(e, "autotune setup");
  TuneVal v{4, 1, {-1.0, -1.0, -1.0, -1.0, -1.0, -1.0, -1.0, -1.0}};
  const int rps[4] = {2, 4, 8, 16};
  const int nchoice = rp_allowed(16, (int)sizeof(T), stage) ? 4 : 3;
  for (int ci = 0; ci < 8 && !rc; ++ci) {
    const int i = ci & 3, mt = 1 + (ci >> 2);
    if (i >= nchoice) continue;
    LegArgs<T> a = leg_args<T>(P, g, L);
    a.df = 0;
    a.alm = alm;
    a.rp_synth = a.rp_adj = rps[i];
    a.mt_synth = a.mt_adj = mt;
    FinalizeArgs<T> f;
    f.out = alm;
    auto run = [&]() { return stage == 0 ? launch_leg_synth<T>(a, P->stream) : launch_leg_adjoint<T>(a, f, P->stream); };
    if ((rc = run())) break;
    if ((e = cudaEventRecord(e0, P->stream)) != cudaSuccess) rc = cuda_fail(e, "autotune event");
    for (int k = 0; k < reps && !rc; ++k) rc = run();
    if (!rc && (e = cudaEventRecord(e1, P->stream)) != cudaSuccess) rc = cuda_fail(e, "autotune event");
    if (!rc && (e = cudaEventSynchronize(e1)) != cudaSuccess) rc = cuda_fail(e, "autotune event");
    float ms = 0.f;
    if (!rc && (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) rc = cuda_fail(e, "autotune event");
    v.ms[ci] = ms / reps;
  }
  if (!rc) {
    int best = 1;
    for (int ci = 0; ci < 8; ++ci)
      if (v.ms[ci] >= 0.0 && v.ms[ci] < v.ms[best]) best = ci;
    v.rp = rps[best & 3];
    v.mt = 1 + (best >> 2);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(alm);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[TuneKey{g.nring, g.npix, L, (int)sizeof(T), stage}] = v;
  return CR_OK;
}

// Time the batched tensor-core synthesis (16 right-hand sides of zeros; the
// work does not depend on the data) on grid g at band limit L for every
// stage-shape variant and record the fastest.
static int tune_tc_stage(cr_plan* P, const Grid& g, int L, int reps) {
  int rc = tc_begin(P, g, L, false, true);
  if (rc) return rc;
  float2* alm = nullptr;
  const int64_t nlm = n_lm(L);
  CR_CUDA(cudaMalloc(&alm, 16 * nlm * sizeof(float2)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemsetAsync(alm, 0, 16 * nlm * sizeof(float2), P->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) rc = cuda_fail(e, "autotune setup");
  TuneVal v{TC_DEFAULT_VARIANT, 1, {-1.0, -1.0, -1.0, -1.0, -1.0, -1.0, -1.0, -1.0}};
  for (int i = 0; i < TC_NVARIANT && !rc; ++i) {
    LegArgs<float> la = leg_args<float>(P, g, L);
    la.tc_variant = i;
    la.tc_split = 0;
    auto run = [&]() { return launch_tc_synth(la, alm, nlm, 16, tc_slot(P, g, L, 0), P->d_tc_status, P->stream); };
    if ((rc = run())) break;
    if ((e = cudaEventRecord(e0, P->stream)) != cudaSuccess) rc = cuda_fail(e, "autotune event");
    for (int k = 0; k < reps && !rc; ++k) rc = run();
    if (!rc && (e = cudaEventRecord(e1, P->stream)) != cudaSuccess) rc = cuda_fail(e, "autotune event");
    if (!rc && (e = cudaEventSynchronize(e1)) != cudaSuccess) rc = cuda_fail(e, "autotune event");
    float ms = 0.f;
    if (!rc && (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) rc = cuda_fail(e, "autotune event");
    v.ms[i] = ms / reps;
  }
  if (!rc) {
    int best = 0;
    for (int i = 0; i < TC_NVARIANT; ++i)
      if (v.ms[i] < v.ms[best]) best = i;
    v.rp = best;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(alm);
  if (!rc) rc = tc_end(P, "autotune: a tensor-core completion wait gave up");
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[TuneKey{g.nring, g.npix, L, TC_TUNE_BYTES, TC_TUNE_SYNTH}] = v;
  return CR_OK;
}

// every (grid, band limit) the plan transforms on: the observation grid at
// lmax and, with levels, each pixel level's grid and inverse-noise grid at
// lmax_h; both precisions, both stages, and the tensor-core synthesis shape
int autotune_plan(cr_plan* P, int reps) {
  std::vector<std::pair<const Grid*, int>> todo{{&P->obs, P->lmax}};
  if (P->hier)
    for (const PixLevel& lev : P->hier->pix) {
      todo.push_back({lev.grid, lev.lmax_h});
      todo.push_back({lev.gl ? lev.gl : &P->obs, lev.lmax_h});
    }
  for (auto& t : todo) {
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      if (g_tune.count(TuneKey{t.first->nring, t.first->npix, t.second, 8, 1})) continue;
    }
    for (int stage = 0; stage < 2; ++stage) {
      int rc = tune_stage<float>(P, *t.first, t.second, stage, reps);
      if (!rc) rc = tune_stage<double>(P, *t.first, t.second, stage, reps);
      if (rc) return rc;
    }
    int rc = tune_tc_stage(P, *t.first, t.second, reps);
    if (rc) return rc;
  }
  return CR_OK;
}

int tune_entry(int i, int* nring, int64_t* npix, int* lmax, int* bytes, int* stage, int* rp, int* mt, double* ms) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (i < 0 || i >= (int)g_tune.size()) return fail(CR_EINVAL, "cr_tune_entry: index out of range");
  auto it = g_tune.begin();
  std::advance(it, i);
  if (nring) *nring = it->first.nring;
  if (npix) *npix = it->first.npix;
  if (lmax) *lmax = it->first.L;
  if (bytes) *bytes = it->first.bytes;
  if (stage) *stage = it->first.stage;
  if (rp) *rp = it->second.rp;
  if (mt) *mt = it->second.mt;
  if (ms)
    for (int k = 0; k < 8; ++k) ms[k] = it->second.ms[k];
  return CR_OK;
}

int tune_set(int nring, int64_t npix, int lmax, int bytes, int stage, int rp, int mt) {
  const bool tc = bytes == TC_TUNE_BYTES && stage == TC_TUNE_SYNTH && rp >= 0 && rp < TC_NVARIANT && mt == 1;
  if (!tc && ((bytes != 4 && bytes != 8) || (stage != 0 && stage != 1) || lmax < 0 || !rp_allowed(rp, bytes, stage) ||
              (mt != 1 && mt != 2)))
    return fail(CR_EINVAL, "cr_tune_set: bad choice");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[TuneKey{nring, npix, lmax, bytes, stage}] = TuneVal{rp, mt, {-1.0, -1.0, -1.0, -1.0, -1.0, -1.0, -1.0, -1.0}};
  return CR_OK;
}

int tune_count() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  return (int)g_tune.size();
}

}  // namespace cr

using namespace cr;

extern "C" {

const char* cr_last_error(void) { return g_last_error.c_str(); }

// Prior-dependent operator diagonals from h_cl and h_bl: B (b_l p_l, 0
// where C_l = 0) and S^-1 (1 / C_l, 0 where C_l = 0) in FP64 and FP32,
// copied into the existing device arrays when the plan already has them.
static int upload_prior(cr_plan* P) {
  const int L = P->lmax;
  std::vector<double> bl(L + 1), sinv(L + 1);
  for (int l = 0; l <= L; ++l) {
    if (!(P->h_cl[l] >= 0.0) || !std::isfinite(P->h_cl[l])) return fail(CR_EINVAL, "C_l must be finite and >= 0");
    const bool act = P->h_cl[l] > 0.0;
    bl[l] = act ? P->h_bl[l] : 0.0;
    sinv[l] = act ? 1.0 / P->h_cl[l] : 0.0;
  }
  std::vector<float> bl32(bl.begin(), bl.end()), sinv32(sinv.begin(), sinv.end());
  auto up = [&](auto** d, const auto& h) -> int {
    const size_t bytes = h.size() * sizeof(h[0]);
    if (!*d) CR_CUDA(cudaMalloc(d, bytes));
    CR_CUDA(cudaMemcpy(*d, h.data(), bytes, cudaMemcpyHostToDevice));
    return CR_OK;
  };
  int rc = up(&P->d_bl, bl);
  if (!rc) rc = up(&P->d_sinv, sinv);
  if (!rc) rc = up(&P->d_bl32, bl32);
  if (!rc) rc = up(&P->d_sinv32, sinv32);
  return rc;
}

// Everything of cr_plan_create after the argument checks; on an error the
// caller frees the partly built plan.
static int plan_init(cr_plan* P, const cr_params* p) {
  P->p = *p;
  P->stream = reinterpret_cast<cudaStream_t>(p->stream);
  P->fp64_df = p->fp64_df ? 1 : 0;
  P->tc_split = P->tc_split_param = p->tc_split ? 1 : 0;
  P->lmax = p->lmax;
  P->levels.resize(1);
  P->levels[0].lmax_h = p->lmax;
  int rc = CR_OK;
  if (p->grid_kind == CR_GRID_HEALPIX) healpix_rings(P->obs, p->nside);
  else gl_rings(P->obs, p->gl_ntheta, p->gl_nphi, nullptr);
  rc = grid_upload(P->obs, P->lmax, P->stream);
  if (!rc) rc = build_coef(P, P->lmax);
  if (!rc) rc = build_start_tables(P, P->obs);
  if (!rc) rc = ensure_workspace(P, P->obs, P->lmax);
  if (!rc) {
    cudaError_t e = cudaMalloc(&P->d_dotpart, (P->lmax + 1) * sizeof(double));
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(dot partials)");
  }
  if (!rc && p->cl) {
    const int L = P->lmax;
    P->h_cl.assign(p->cl, p->cl + L + 1);
    P->h_bl.assign(L + 1, 1.0);
    if (p->bl) P->h_bl.assign(p->bl, p->bl + L + 1);
    rc = upload_prior(P);
    if (!rc) {
      const int64_t npix = P->obs.npix;
      if (!rc) {
        cudaError_t e = cudaMalloc(&P->d_ninv, npix * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&P->d_ninv32, npix * sizeof(float));
        if (e != cudaSuccess) rc = cuda_fail(e, "cudaMalloc(ninv)");
      }
      if (!rc) {
        cudaError_t e = p->ninv ? cudaMemcpyAsync(P->d_ninv, p->ninv, npix * sizeof(double),
                                                  cudaMemcpyDeviceToDevice, P->stream)
                                : cudaMemsetAsync(P->d_ninv, 0, npix * sizeof(double), P->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy ninv");
      }
      if (!rc && p->ninv) {
        // N^-1 must be finite and >= 0 (0 = masked): checked on the host in
        // bounded chunks, so a NaN or a negative weight is refused here
        // instead of surfacing later as a failed factorisation or a
        // non-finite residual
        const int64_t chunk = (int64_t)1 << 22;
        std::vector<double> h((size_t)std::min<int64_t>(chunk, npix));
        for (int64_t o = 0; o < npix && !rc; o += chunk) {
          const int64_t n = std::min(chunk, npix - o);
          cudaError_t e = cudaMemcpyAsync(h.data(), P->d_ninv + o, n * sizeof(double), cudaMemcpyDeviceToHost,
                                          P->stream);
          if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
          if (e != cudaSuccess) {
            rc = cuda_fail(e, "check ninv");
            break;
          }
          for (int64_t i = 0; i < n; ++i)
            if (!(h[i] >= 0.0) || !std::isfinite(h[i])) {
              rc = fail(CR_EINVAL, "cr_plan_create: N^-1 must be finite and >= 0 (pixel " + std::to_string(o + i) + ")");
              break;
            }
        }
      }
      if (!rc) {
        ninv32_kernel<<<1024, 256, 0, P->stream>>>(P->d_ninv, P->d_ninv32, npix);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(P->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "ninv32");
      }
      if (!rc) P->has_op = true;
    }
    if (!rc && p->nlevels != 0) {
      if (p->grid_kind != CR_GRID_HEALPIX) rc = fail(CR_EINVAL, "cr_plan_create: levels need a HEALPix grid");
      else rc = build_hierarchy(P, p);
    }
  }
  if (!rc && p->autotune) rc = autotune_plan(P, 3);
  return rc;
}

int cr_plan_create(cr_plan** out, const cr_params* p) {
  if (!out || !p) return fail(CR_EINVAL, "cr_plan_create: null argument");
  if (p->struct_size != (int)sizeof(cr_params)) return fail(CR_EINVAL, "cr_plan_create: struct_size mismatch");
  if (p->lmax < 0 || p->lmax > 16384) return fail(CR_EINVAL, "cr_plan_create: lmax out of range");
  if (p->grid_kind == CR_GRID_HEALPIX) {
    if (p->nside < 1 || (p->nside & (p->nside - 1)) || p->nside > 16384)
      return fail(CR_EINVAL, "cr_plan_create: nside must be a power of two in [1, 16384]");
  } else if (p->grid_kind == CR_GRID_GL) {
    if (p->gl_ntheta < 1 || p->gl_nphi < 2 || (p->gl_nphi & 1))
      return fail(CR_EINVAL, "cr_plan_create: GL grid needs ntheta >= 1 and even nphi >= 2");
  } else {
    return fail(CR_EINVAL, "cr_plan_create: unknown grid kind");
  }
  cr_plan* P = nullptr;
  try {
    P = new cr_plan();
  } catch (std::bad_alloc&) {
    return fail(CR_ENOMEM, "cr_plan_create: host allocation");
  }
  int rc = CR_OK;
  try {
    rc = plan_init(P, p);
  } catch (const std::bad_alloc&) {
    rc = fail(CR_ENOMEM, "cr_plan_create: host allocation");
  }
  if (rc) {
    plan_free(P);
    delete P;
    return rc;
  }
  *out = P;
  return CR_OK;
}

int cr_plan_autotune(cr_plan* plan, int* nentries) {
  if (!plan) return fail(CR_EINVAL, "cr_plan_autotune: null plan");
  CR_CUDA(cudaStreamSynchronize(plan->stream));
  int rc = autotune_plan(plan, 3);
  if (nentries) *nentries = tune_count();
  return rc;
}

int cr_tune_entry(int i, int* nring, int64_t* npix, int* lmax, int* precision_bytes, int* stage, int* rp,
                  int* m_tile, double* ms) {
  return tune_entry(i, nring, npix, lmax, precision_bytes, stage, rp, m_tile, ms);
}

int cr_tune_set(int nring, int64_t npix, int lmax, int precision_bytes, int stage, int rp, int m_tile) {
  return tune_set(nring, npix, lmax, precision_bytes, stage, rp, m_tile);
}

int cr_plan_update_cl(cr_plan* plan, const double* cl) {
  if (!plan || !cl) return fail(CR_EINVAL, "cr_plan_update_cl: null argument");
  if (!plan->has_op) return fail(CR_ESTATE, "cr_plan_update_cl: plan was created without C_l");
  const int L = plan->lmax;
  for (int l = 0; l <= L; ++l)
    if (!(cl[l] >= 0.0) || !std::isfinite(cl[l])) return fail(CR_EINVAL, "cr_plan_update_cl: C_l must be finite and >= 0");
  CR_CUDA(cudaStreamSynchronize(plan->stream));
  if (plan->hier) plan->hier->numeric_ready = false;
  plan->h_cl.assign(cl, cl + L + 1);
  int rc = upload_prior(plan);
  if (rc) return rc;
  if (plan->d_pcinv) {
    cudaFree(plan->d_pcinv);
    plan->d_pcinv = nullptr;
  }
  if (plan->hier) {
    TimerScope ts(plan->timing, plan->stream, "precompute_cl");
    try {
      rc = build_numeric(plan);
    } catch (const std::bad_alloc&) {
      rc = fail(CR_ENOMEM, "cr_plan_update_cl: host allocation");
    }
  }
  return rc;
}

int cr_plan_destroy(cr_plan* plan) {
  if (!plan) return CR_OK;
  cudaStreamSynchronize(plan->stream);
  plan_free(plan);
  delete plan;
  return CR_OK;
}

int cr_plan_sizes(const cr_plan* plan, int grid, int64_t* npix, int* nring, int* lmax, int64_t* nlm) {
  if (!plan) return fail(CR_EINVAL, "cr_plan_sizes: null plan");
  int L = 0;
  const Grid* g = grid_of(const_cast<cr_plan*>(plan), grid, &L);
  if (!g) return fail(CR_EINVAL, "cr_plan_sizes: unknown grid");
  if (npix) *npix = g->npix;
  if (nring) *nring = g->nring;
  if (lmax) *lmax = L;
  if (nlm) *nlm = n_lm(L);
  return CR_OK;
}

static int check_ptr(const void* p, int dtype) {
  const uintptr_t a = (uintptr_t)p;
  const uintptr_t al = dtype == CR_F64 ? 16 : 8;
  if (!p || (a % al)) return fail(CR_EINVAL, "buffer pointer null or not aligned to a complex element");
  return CR_OK;
}

}  // extern "C"

namespace cr {

// Batched transforms with the Legendre contractions on the tensor cores
// (BF16 operands, FP32 accumulation; legendre_tc.cu) on FP32 data, 16
// right-hand sides per Legendre launch; the ring FFTs run per right-hand side.
static int grow(void** buf, int64_t* have, int64_t need) {
  if (need <= *have) return CR_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *have = 0;
  CR_CUDA(cudaMalloc(buf, need));
  *have = need;
  return CR_OK;
}

int tc_begin(cr_plan* P, const Grid& g, int L, bool adjoint, bool reset_status) {
  int rc = grow(&P->tc_phase, &P->tc_phase_bytes, (int64_t)16 * g.nring * (L + 1) * (int64_t)sizeof(float2));
  if (!rc && adjoint) {
    const int64_t nblk = tc_adjoint_blocks(g.npolar32, g.npairs);
    rc = grow(&P->tc_partial, &P->tc_partial_bytes, 16 * nblk * n_lm(L) * (int64_t)sizeof(float2));
  }
  if (rc) return rc;
  if (!P->d_tc_status) {
    CR_CUDA(cudaMalloc(&P->d_tc_status, sizeof(int)));
    reset_status = true;
  }
  if (reset_status) CR_CUDA(cudaMemsetAsync(P->d_tc_status, 0, sizeof(int), P->stream));
  return CR_OK;
}

int tc_end(cr_plan* P, const char* what) {
  int st = 0;
  CR_CUDA(cudaMemcpyAsync(&st, P->d_tc_status, sizeof(int), cudaMemcpyDeviceToHost, P->stream));
  CR_CUDA(cudaStreamSynchronize(P->stream));
  if (st) return fail(CR_ECUDA, what);
  return CR_OK;
}

float2* tc_slot(cr_plan* P, const Grid& g, int L, int r) {
  return reinterpret_cast<float2*>(P->tc_phase) + (int64_t)r * g.nring * (L + 1);
}

// the synthesis Legendre stage of nr <= 16 right-hand sides x [nr][n_lm(L)]
// (times dl, may be null) into the phase slots
int tc_synth_stage(cr_plan* P, const Grid& g, int L, const float2* x, int nr, const float* dl) {
  LegArgs<float> la = leg_args<float>(P, g, L);
  la.dl = dl;
  TimerScope ts(P->timing, P->stream, "legendre_synth_tc", leg_work(g, L) * nr, leg_work_exec(P, g, L) * nr);
  return launch_tc_synth(la, x, n_lm(L), nr, tc_slot(P, g, L, 0), P->d_tc_status, P->stream);
}

// the adjoint Legendre stage of nr right-hand sides from the phase slots,
// then per right-hand side r (vectors at stride n_lm(L)):
//   out_r (+)= dl_out sum_blk partial + dadd xadd_r   (or bsub_r - that)
int tc_adjoint_tail(cr_plan* P, const Grid& g, int L, int nr, const TcTail& t) {
  LegArgs<float> la = leg_args<float>(P, g, L);
  const int64_t nlm = n_lm(L);
  int nblk = 0, rc;
  {
    TimerScope ts(P->timing, P->stream, "legendre_adjoint_tc", leg_work(g, L) * nr,
                  leg_work_exec(P, g, L) * nr);
    rc = launch_tc_adjoint(la, tc_slot(P, g, L, 0), nr, reinterpret_cast<float2*>(P->tc_partial), &nblk,
                           P->d_tc_status, P->stream);
  }
  if (rc) return rc;
  for (int r = 0; r < nr; ++r) {
    FinalizeArgs<float> f;
    f.partial = reinterpret_cast<const float2*>(P->tc_partial) + (int64_t)r * nblk * nlm;
    f.nblk = nblk;
    f.L = L;
    f.dl_out = t.dl_out;
    f.dadd = t.dadd;
    f.xadd = t.xadd ? t.xadd + r * nlm : nullptr;
    f.bsub = t.bsub ? t.bsub + r * nlm : nullptr;
    f.accumulate = t.accumulate;
    f.out = t.out + r * nlm;
    TimerScope ts(P->timing, P->stream, "legendre_finalize_tc", (double)(nblk + 1) * nlm * sizeof(float2));
    if ((rc = launch_leg_finalize<float>(f, P->stream))) return rc;
  }
  return CR_OK;
}

// ring FFT stage of phase slot r: mode 0 slot -> map_out, mode 1 map_in -> slot
int tc_ring(cr_plan* P, const Grid& g, int L, int r, int mode, const float* map_in, float* map_out) {
  RingArgs<float> ra = ring_args<float>(P, g, L);
  ra.phase = tc_slot(P, g, L, r);
  ra.map_in = map_in;
  ra.map_out = map_out;
  TimerScope ts(P->timing, P->stream, mode == 0 ? "ring_fft_synth_f32" : "ring_fft_adjoint_f32",
                fft_bytes<float>(g, L, 1));
  return launch_ring_fft<float>(ra, mode, P->stream);
}

// y_r = dl_out Y^T diag(pix) Y (dl_in x_r) + dadd x_r (or bsub_r - that) for
// nr <= 16 right-hand sides at stride n_lm(L), both Legendre stages on the
// tensor cores
int tc_sandwich(cr_plan* P, const Grid& g, int L, int nr, const float2* x, const float* dl_in, const float* pix,
                const TcTail& t) {
  int rc = tc_synth_stage(P, g, L, x, nr, dl_in);
  if (rc) return rc;
  for (int r = 0; r < nr; ++r) {
    RingArgs<float> ra = ring_args<float>(P, g, L);
    ra.phase = tc_slot(P, g, L, r);
    ra.pixdiag = pix;
    TimerScope ts(P->timing, P->stream, "ring_fft_apply_f32",
                  fft_bytes<float>(g, L, 1) + (double)g.nring * (L + 1) * sizeof(float2));
    if ((rc = launch_ring_fft<float>(ra, 2, P->stream))) return rc;
  }
  return tc_adjoint_tail(P, g, L, nr, t);
}

}  // namespace cr

extern "C" {

static int tc_synth(cr_plan* P, const Grid& g, int L, const void* alm, void* map, int nrhs) {
  int rc = tc_begin(P, g, L, false, true);
  if (rc) return rc;
  const int64_t nlm = n_lm(L);
  for (int r0 = 0; r0 < nrhs; r0 += 16) {
    const int nr = std::min(16, nrhs - r0);
    if ((rc = tc_synth_stage(P, g, L, reinterpret_cast<const float2*>(alm) + (int64_t)r0 * nlm, nr, nullptr)))
      return rc;
    for (int r = 0; r < nr; ++r) {
      RingArgs<float> ra = ring_args<float>(P, g, L);
      ra.phase = tc_slot(P, g, L, r);
      ra.map_out = reinterpret_cast<float*>(map) + (int64_t)(r0 + r) * g.npix;
      TimerScope ts(P->timing, P->stream, "ring_fft_synth_f32", fft_bytes<float>(g, L, 1));
      if ((rc = launch_ring_fft<float>(ra, 0, P->stream))) return rc;
    }
  }
  return tc_end(P, "tensor-core synthesis: a completion wait gave up");
}

static int tc_adjoint(cr_plan* P, const Grid& g, int L, const void* map, void* alm, int nrhs) {
  int rc = tc_begin(P, g, L, true, true);
  if (rc) return rc;
  const int64_t nlm = n_lm(L);
  for (int r0 = 0; r0 < nrhs; r0 += 16) {
    const int nr = std::min(16, nrhs - r0);
    for (int r = 0; r < nr; ++r) {
      RingArgs<float> ra = ring_args<float>(P, g, L);
      ra.phase = tc_slot(P, g, L, r);
      ra.map_in = reinterpret_cast<const float*>(map) + (int64_t)(r0 + r) * g.npix;
      TimerScope ts(P->timing, P->stream, "ring_fft_adjoint_f32", fft_bytes<float>(g, L, 1));
      if ((rc = launch_ring_fft<float>(ra, 1, P->stream))) return rc;
    }
    TcTail t;
    t.out = reinterpret_cast<float2*>(alm) + r0 * nlm;
    if ((rc = tc_adjoint_tail(P, g, L, nr, t))) return rc;
  }
  return tc_end(P, "tensor-core adjoint: a completion wait gave up");
}

// y = (S^-1 + B Y^T N^-1 Y B) x for nrhs right-hand sides on the observation
// grid (Eq. 3 system matrix), both Legendre stages on the tensor cores
static int tc_apply(cr_plan* P, const void* x, void* y, int nrhs) {
  const Grid& g = P->obs;
  const int L = P->lmax;
  int rc = tc_begin(P, g, L, true, true);
  if (rc) return rc;
  const int64_t nlm = n_lm(L);
  for (int r0 = 0; r0 < nrhs; r0 += 16) {
    const int nr = std::min(16, nrhs - r0);
    const float2* xr = reinterpret_cast<const float2*>(x) + (int64_t)r0 * nlm;
    TcTail t;
    t.dl_out = P->d_bl32;
    t.dadd = P->d_sinv32;
    t.xadd = xr;
    t.out = reinterpret_cast<float2*>(y) + r0 * nlm;
    if ((rc = tc_sandwich(P, g, L, nr, xr, P->d_bl32, P->d_ninv32, t))) return rc;
  }
  return tc_end(P, "tensor-core apply: a completion wait gave up");
}

int cr_sht_synth(cr_plan* plan, int grid, const void* alm, void* map, int nrhs, int dtype) {
  if (!plan) return fail(CR_EINVAL, "cr_sht_synth: null plan");
  int L = 0;
  const Grid* g = grid_of(plan, grid, &L);
  if (!g) return fail(CR_EINVAL, "cr_sht_synth: unknown grid");
  if (nrhs >= 0 && dtype == CR_TC) {
    if (nrhs == 0) return CR_OK;
    if (check_ptr(alm, CR_F32) || check_ptr(map, CR_F32)) return CR_EINVAL;
    return tc_synth(plan, *g, L, alm, map, nrhs);
  }
  if (nrhs < 0 || (dtype != CR_F64 && dtype != CR_F32)) return fail(CR_EINVAL, "cr_sht_synth: nrhs/dtype");
  if (nrhs == 0) return CR_OK;
  if (check_ptr(alm, dtype) || check_ptr(map, dtype)) return CR_EINVAL;
  const size_t es = dtype == CR_F64 ? 8 : 4;
  for (int r = 0; r < nrhs; ++r) {
    const char* a = (const char*)alm + (size_t)r * n_lm(L) * 2 * es;
    char* m = (char*)map + (size_t)r * g->npix * es;
    int rc = dtype == CR_F64 ? do_synth<double>(plan, *g, L, a, m, nullptr) : do_synth<float>(plan, *g, L, a, m, nullptr);
    if (rc) return rc;
  }
  return CR_OK;
}

int cr_sht_adjoint(cr_plan* plan, int grid, const void* map, void* alm, int nrhs, int dtype) {
  if (!plan) return fail(CR_EINVAL, "cr_sht_adjoint: null plan");
  int L = 0;
  const Grid* g = grid_of(plan, grid, &L);
  if (!g) return fail(CR_EINVAL, "cr_sht_adjoint: unknown grid");
  if (nrhs >= 0 && dtype == CR_TC) {
    if (nrhs == 0) return CR_OK;
    if (check_ptr(alm, CR_F32) || check_ptr(map, CR_F32)) return CR_EINVAL;
    return tc_adjoint(plan, *g, L, map, alm, nrhs);
  }
  if (nrhs < 0 || (dtype != CR_F64 && dtype != CR_F32)) return fail(CR_EINVAL, "cr_sht_adjoint: nrhs/dtype");
  if (nrhs == 0) return CR_OK;
  if (check_ptr(alm, dtype) || check_ptr(map, dtype)) return CR_EINVAL;
  const size_t es = dtype == CR_F64 ? 8 : 4;
  for (int r = 0; r < nrhs; ++r) {
    const char* m = (const char*)map + (size_t)r * g->npix * es;
    char* a = (char*)alm + (size_t)r * n_lm(L) * 2 * es;
    int rc = dtype == CR_F64 ? do_adjoint<double>(plan, *g, L, m, a, nullptr, nullptr, nullptr, 0)
                             : do_adjoint<float>(plan, *g, L, m, a, nullptr, nullptr, nullptr, 0);
    if (rc) return rc;
  }
  return CR_OK;
}

int cr_apply_A(cr_plan* plan, int level, const void* x, void* y, int nrhs, int dtype) {
  if (!plan) return fail(CR_EINVAL, "cr_apply_A: null plan");
  if (!plan->has_op) return fail(CR_ESTATE, "cr_apply_A: plan was created without C_l");
  if (level != 0) return cr_level_apply(plan, level, x, y, dtype);
  if (nrhs >= 0 && dtype == CR_TC) {
    if (nrhs == 0) return CR_OK;
    if (check_ptr(x, CR_F32) || check_ptr(y, CR_F32)) return CR_EINVAL;
    if (x == y) return fail(CR_EINVAL, "cr_apply_A: x and y must not overlap");
    return tc_apply(plan, x, y, nrhs);
  }
  if (nrhs < 0 || (dtype != CR_F64 && dtype != CR_F32)) return fail(CR_EINVAL, "cr_apply_A: nrhs/dtype");
  if (nrhs == 0) return CR_OK;
  if (check_ptr(x, dtype) || check_ptr(y, dtype)) return CR_EINVAL;
  if (x == y) return fail(CR_EINVAL, "cr_apply_A: x and y must not overlap");
  const int L = plan->lmax;
  const size_t es = dtype == CR_F64 ? 8 : 4;
  if (dtype == CR_F64 && nrhs > 1 && !plan->fp64_df) {
    // several right-hand sides: the FP64 stages 8 at a time
    const int64_t nlm = n_lm(L);
    for (int r0 = 0; r0 < nrhs; r0 += 8) {
      int rc = do_sandwich_mr(plan, plan->obs, L, std::min(8, nrhs - r0), (const double2*)x + r0 * nlm,
                              (double2*)y + r0 * nlm, plan->d_bl, plan->d_ninv, plan->d_bl, plan->d_sinv, nullptr);
      if (rc) return rc;
    }
    return CR_OK;
  }
  for (int r = 0; r < nrhs; ++r) {
    const char* xr = (const char*)x + (size_t)r * n_lm(L) * 2 * es;
    char* yr = (char*)y + (size_t)r * n_lm(L) * 2 * es;
    int rc = dtype == CR_F64
                 ? do_sandwich<double>(plan, plan->obs, L, xr, yr, plan->d_bl, plan->d_ninv, plan->d_bl, plan->d_sinv,
                                       nullptr, nullptr)
                 : do_sandwich<float>(plan, plan->obs, L, xr, yr, plan->d_bl32, plan->d_ninv32, plan->d_bl32,
                                      plan->d_sinv32, nullptr, nullptr);
    if (rc) return rc;
  }
  return CR_OK;
}

int cr_plan_set_timing(cr_plan* plan, int enable) {
  if (!plan) return fail(CR_EINVAL, "cr_plan_set_timing: null plan");
  plan->timing.flush();
  plan->timing.acc.clear();
  plan->timing.enabled = enable != 0;
  return CR_OK;
}

int cr_plan_timing(cr_plan* plan, int i, char* name, int name_cap, double* ms, long* launches, double* work,
                   int* count) {
  if (!plan) return fail(CR_EINVAL, "cr_plan_timing: null plan");
  plan->timing.flush();
  if (count) *count = (int)plan->timing.acc.size();
  if (i < 0) return CR_OK;
  if (i >= (int)plan->timing.acc.size()) return fail(CR_EINVAL, "cr_plan_timing: index out of range");
  auto it = plan->timing.acc.begin();
  std::advance(it, i);
  if (name && name_cap > 0) {
    std::strncpy(name, it->first.c_str(), name_cap - 1);
    name[name_cap - 1] = 0;
  }
  if (ms) *ms = it->second.ms;
  if (launches) *launches = it->second.n;
  if (work) *work = it->second.work;
  return CR_OK;
}

int cr_plan_timing_exec(cr_plan* plan, int i, double* work_exec) {
  if (!plan || !work_exec) return fail(CR_EINVAL, "cr_plan_timing_exec: null argument");
  plan->timing.flush();
  if (i < 0 || i >= (int)plan->timing.acc.size()) return fail(CR_EINVAL, "cr_plan_timing_exec: index out of range");
  auto it = plan->timing.acc.begin();
  std::advance(it, i);
  *work_exec = it->second.work_exec;
  return CR_OK;
}

long cr_launch_count(void) { return launch_count(); }

}  // extern "C"
