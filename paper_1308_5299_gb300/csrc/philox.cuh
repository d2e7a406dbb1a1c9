// Philox4x32-10 normals shared by the right-hand-side generator and the
// gradient kernels (definition in draw.cu's header comment).
#pragma once
#include <stdint.h>

namespace cr {

struct U4 {
  uint32_t x[4];
};

__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                            uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
  U4 o;
  o.x[0] = c0;
  o.x[1] = c1;
  o.x[2] = c2;
  o.x[3] = c3;
  return o;
}

__device__ __forceinline__ double draw_normal(uint64_t seed, uint32_t stream, uint32_t rhs, uint64_t k) {
  const U4 x = philox4x32_10((uint32_t)(k >> 2), (uint32_t)(k >> 34), stream, rhs, (uint32_t)seed,
                             (uint32_t)(seed >> 32));
  const int slot = (int)(k & 3);
  const uint32_t a = slot < 2 ? x.x[0] : x.x[2];
  const uint32_t b = slot < 2 ? x.x[1] : x.x[3];
  const double ua = ((double)a + 0.5) * 0x1p-32;
  const double ub = ((double)b + 0.5) * 0x1p-32;
  const double r = sqrt(-2.0 * log(ua));
  double s, c;
  sincospi(2.0 * ub, &s, &c);
  return (slot & 1) ? r * s : r * c;
}

}  // namespace cr
