// Allocation-free FP64 HEALPix synthesis (cr_sht_synth_noalloc).
//
// Some callers cannot call cudaMalloc at all: code that runs while a CUDA
// graph is being captured, code inside allocator callbacks or under a fixed
// device-memory budget owned by another framework, real-time loops that must
// never allocate.  Such callers cannot create a plan either.  This entry point
// needs no plan: every table (ring geometry, Legendre seeds and recurrence
// coefficients, azimuthal phases) is computed on the fly, and the only scratch
// -- the per-ring Legendre output F_m(ring) between the two stages -- lives in
// the file-scope device array below, sized for grids up to
// CR_NOALLOC_SCRATCH_BYTES.  The array belongs to every GPU that loads the
// library until the process exits; all calls share it and it keeps the
// contents of the last call.
#include <cuda.h>

#include <cmath>
#include <mutex>

#include "common.cuh"

#define CR_NOALLOC_SCRATCH_BYTES (16u << 20)

namespace cr {

static __device__ __align__(256) double2 g_noalloc_phase[CR_NOALLOC_SCRATCH_BYTES / sizeof(double2)];

// HEALPix ring i (1-based) of Nside N: z, sin(theta), pixels, shift s, first pixel.
__device__ static void hp_ring(int N, int i, double* z, double* sth, int* n, int* s, int64_t* off) {
  if (i < N || i > 3 * N) {
    const int ii = i < N ? i : 4 * N - i;
    const double omz = (double)ii * ii / (3.0 * N * N);
    *z = (i < N) ? 1.0 - omz : -(1.0 - omz);
    *sth = sqrt(omz * (2.0 - omz));
    *n = 4 * ii;
    *s = 1;
    *off = (i < N) ? 2LL * ii * (ii - 1) : 12LL * N * N - 2LL * ii * (ii + 1);
  } else {
    *z = 4.0 / 3.0 - 2.0 * i / (3.0 * N);
    *sth = sqrt((1.0 - *z) * (1.0 + *z));
    *n = 4 * N;
    *s = (i - N + 1) & 1;
    *off = 2LL * N * (N - 1) + (int64_t)(i - N) * 4 * N;
  }
}

// Legendre stage: F_m(+-z) = sum_l a_lm P~_lm(+-z) per ring pair, with the
// normalised recurrence P~_l = a_l (z P~_{l-1} - P~_{l-2} / a_{l-1}) evaluated
// in FP64 with its coefficients computed in place, and a seed
// log2 |P~_mm| = 1/2 [log2((2m+1)/(4 pi)) + sum_{k=1..m} log2(1 - 1/(2k))]
//               + m log2 sin(theta)
// carried as v 2^e to stay clear of underflow.  The product of (2k-1)/(2k) is
// summed term by term with log1p (each term at full relative precision, a
// fixed-order block reduction) rather than as a difference of two lgamma
// values, which would lose digits to cancellation at large m.
constexpr int NOALLOC_NT = 128;
__global__ void __launch_bounds__(NOALLOC_NT) noalloc_legendre_kernel(const double2* __restrict__ alm, int N, int L,
                                                                      double2* phase) {
  const int m = blockIdx.x;
  const int nring = 4 * N - 1, npairs = 2 * N;
  const int p = blockIdx.y * blockDim.x + threadIdx.x;
  __shared__ double s_part[NOALLOC_NT];
  {
    double t = 0.0;
    for (int k = 1 + (int)threadIdx.x; k <= m; k += NOALLOC_NT) t += log1p(-0.5 / k);
    s_part[threadIdx.x] = t;
    __syncthreads();
    for (int w = NOALLOC_NT / 2; w > 0; w >>= 1) {
      if ((int)threadIdx.x < w) s_part[threadIdx.x] += s_part[threadIdx.x + w];
      __syncthreads();
    }
  }
  if (p >= npairs) return;
  double z, sth;
  int n, s;
  int64_t off;
  hp_ring(N, p + 1, &z, &sth, &n, &s, &off);
  const double lgn = 0.5 * (log2((2.0 * m + 1.0) / (4.0 * M_PI)) + s_part[0] / log(2.0)) +
                     (m > 0 ? m * log2(sth) : 0.0);
  int e = (int)floor(lgn);
  double v1 = exp2(lgn - e);
  if (m & 1) v1 = -v1;
  double v0 = 0.0;  // P~_{l-2}, scaled like v1
  const int64_t o = (int64_t)m * (L + 1) - (int64_t)m * (m - 1) / 2;
  double2 E = make_double2(0.0, 0.0), O = make_double2(0.0, 0.0);
  double a_prev = 1.0;
  for (int l = m; l <= L; ++l) {
    double cur;
    if (l == m) {
      cur = v1;
    } else {
      const double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
      cur = (l == m + 1) ? a * z * v1 : a * (z * v1 - v0 / a_prev);
      a_prev = a;
      v0 = v1;
      v1 = cur;
      if (e < 0 && fabs(v1) > 0x1p200) {
        v0 *= 0x1p-200;
        v1 *= 0x1p-200;
        e += 200;
      }
    }
    const double pv = (e < -1000) ? 0.0 : ldexp(v1, e);
    double2 av = alm[o + (l - m)];
    if (m == 0) av.y = 0.0;
    if ((l - m) & 1) {
      O.x = fma(pv, av.x, O.x);
      O.y = fma(pv, av.y, O.y);
    } else {
      E.x = fma(pv, av.x, E.x);
      E.y = fma(pv, av.y, E.y);
    }
  }
  const int rn = p, rs = nring - 1 - p;
  phase[(int64_t)rn * (L + 1) + m] = make_double2(E.x + O.x, E.y + O.y);
  if (rs != rn) phase[(int64_t)rs * (L + 1) + m] = make_double2(E.x - O.x, E.y - O.y);
}

// Ring stage: map_j = Re F_0 + 2 sum_{m>0} Re(F_m e^{i m phi_j}),
// phi_j = pi (2 j + s) / n, by direct summation; e^{i m phi_j} is advanced by
// complex rotation and re-anchored exactly (integer-reduced argument) every 32 m.
__global__ void noalloc_ring_kernel(const double2* __restrict__ phase, int N, int L, double* map) {
  const int r = blockIdx.x;
  double z, sth;
  int n, s;
  int64_t off;
  hp_ring(N, r + 1, &z, &sth, &n, &s, &off);
  const double2* row = phase + (int64_t)r * (L + 1);
  __shared__ double2 sF[256];
  for (int j0 = 0; j0 < n; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    const int64_t u = 2LL * j + s;  // phi_j = pi u / n
    double sr, cr0;
    sincospi((double)u / n, &sr, &cr0);
    double acc = 0.0, c = 1.0, sn = 0.0;
    for (int m0 = 0; m0 <= L; m0 += 256) {
      __syncthreads();
      for (int t = threadIdx.x; t < 256 && m0 + t <= L; t += blockDim.x) sF[t] = row[m0 + t];
      __syncthreads();
      const int mend = min(L, m0 + 255);
      for (int m = m0; m <= mend; ++m) {
        if ((m & 31) == 0) {
          const int64_t arg = ((int64_t)m * u) % (2LL * n);
          sincospi((double)arg / n, &sn, &c);
        }
        const double2 F = sF[m - m0];
        const double w = (m == 0) ? 1.0 : 2.0;
        acc = fma(w, F.x * c - F.y * sn, acc);
        const double c2 = c * cr0 - sn * sr;
        sn = sn * cr0 + c * sr;
        c = c2;
      }
    }
    if (j < n) map[off + j] = acc;
  }
}

// Device address of the scratch array per device ordinal, with the unique id
// of the context it was resolved in: after a device reset the primary
// context (and the module holding the array) is rebuilt, the id changes, and
// the address is looked up again.
static std::mutex g_noalloc_mutex;
static double2* g_noalloc_addr[64] = {nullptr};
static unsigned long long g_noalloc_ctx[64] = {0};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current context (0 if none or if the
// CUDA driver cannot report it).  The CUDA driver API functions are reached
// through the runtime's entry-point query, so the library does not link
// libcuda.
static unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_cur, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess || q1 != cudaDriverEntryPointSuccess)
      get_cur = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess || q2 != cudaDriverEntryPointSuccess)
      get_id = nullptr;
  }
  if (!get_cur || !get_id) return 0;
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (get_cur(&c) != CUDA_SUCCESS || !c) return 0;
  if (get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

}  // namespace cr

using namespace cr;

extern "C" int cr_sht_synth_noalloc(int nside, int lmax, const void* alm, void* map, void* stream) {
  if (nside < 1 || (nside & (nside - 1)) || nside > 8192 || lmax < 0 || lmax > 16384)
    return fail(CR_EINVAL, "cr_sht_synth_noalloc: nside must be a power of two <= 8192 and 0 <= lmax <= 16384");
  const int nring = 4 * nside - 1;
  const double need = (double)nring * (lmax + 1) * sizeof(double2);
  if (need > (double)CR_NOALLOC_SCRATCH_BYTES)
    return fail(CR_EINVAL, "cr_sht_synth_noalloc: (4 nside - 1) (lmax + 1) complex doubles exceed the 16 MiB "
                           "static scratch");
  if (!alm || !map || ((uintptr_t)alm % 16) || ((uintptr_t)map % 8))
    return fail(CR_EINVAL, "cr_sht_synth_noalloc: null or misaligned buffer");
  int dev = 0;
  CR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(CR_EINVAL, "cr_sht_synth_noalloc: device index >= 64");
  double2* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    // Host code must not pass the symbol itself to a kernel: resolve its
    // device address once per device (and again if that device's context
    // was rebuilt), with that device current.  With no current context yet
    // the id reads 0, and the symbol lookup below creates the context.
    const unsigned long long ctx = current_ctx_id();
    if (!g_noalloc_addr[dev] || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
      cudaError_t e = cudaGetSymbolAddress((void**)&g_noalloc_addr[dev], g_noalloc_phase);
      if (e != cudaSuccess) {
        g_noalloc_addr[dev] = nullptr;
        return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
      }
      g_noalloc_ctx[dev] = current_ctx_id();
    }
    scratch = g_noalloc_addr[dev];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int npairs = 2 * nside;
  dim3 g1(lmax + 1, (npairs + NOALLOC_NT - 1) / NOALLOC_NT);
  { noalloc_legendre_kernel<<<g1, NOALLOC_NT, 0, st>>>((const double2*)alm, nside, lmax, scratch); count_launch(); }
  CR_CHECK_LAUNCH("noalloc_legendre_kernel");
  { noalloc_ring_kernel<<<nring, 256, 0, st>>>(scratch, nside, lmax, (double*)map); count_launch(); }
  CR_CHECK_LAUNCH("noalloc_ring_kernel");
  return CR_OK;
}
