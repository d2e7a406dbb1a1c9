// HEALPix NESTED-scheme index arithmetic (Gorski et al. 2005), shared by
// host and device code: nested index -> (face, ix, iy) -> RING index, and the
// unit vector of continuous face coordinates.
#pragma once
#include <stdint.h>

#include <cmath>

namespace cr {

__host__ __device__ inline int64_t compress_bits(int64_t v) {
  int64_t out = 0;
  for (int b = 0; b < 31; ++b) out |= ((v >> (2 * b)) & 1) << b;
  return out;
}

__host__ __device__ inline void nest_xyf(int64_t nside, int64_t ipix, int* ix, int* iy, int* f) {
  const int64_t npf = nside * nside;
  *f = (int)(ipix / npf);
  const int64_t w = ipix % npf;
  *ix = (int)compress_bits(w);
  *iy = (int)compress_bits(w >> 1);
}

__host__ __device__ inline int64_t xyf_ring(int64_t N, int ix, int iy, int f) {
  const int jrll[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
  const int jpll[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};
  const int64_t jr = jrll[f] * N - ix - iy - 1;
  int64_t nr, s, start;
  if (jr < N) {
    nr = jr;
    s = 1;
    start = 2 * jr * (jr - 1);
  } else if (jr > 3 * N) {
    nr = 4 * N - jr;
    s = 1;
    start = 12 * N * N - 2 * nr * (nr + 1);
  } else {
    nr = N;
    s = (jr - N + 1) & 1;
    start = 2 * N * (N - 1) + (jr - N) * 4 * N;
  }
  int64_t j = (nr * jpll[f] + ix - iy - s) / 2;
  const int64_t M = 4 * nr;
  j = ((j % M) + M) % M;
  return start + j;
}

__host__ __device__ inline int64_t nest2ring(int64_t nside, int64_t ipix) {
  int ix, iy, f;
  nest_xyf(nside, ipix, &ix, &iy, &f);
  return xyf_ring(nside, ix, iy, f);
}

// Unit vector of continuous face coordinates (x, y) in [0, N]^2 of face f.
__host__ __device__ inline void face_vec(double N, int f, double x, double y, double* v) {
  const int jrll[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
  const int jpll[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};
  const double jr = jrll[f] * N - x - y;
  double z, nr;
  if (jr < N) {
    z = 1.0 - jr * jr / (3.0 * N * N);
    nr = jr;
  } else if (jr > 3.0 * N) {
    const double t = 4.0 * N - jr;
    z = -(1.0 - t * t / (3.0 * N * N));
    nr = t;
  } else {
    z = 4.0 / 3.0 - 2.0 * jr / (3.0 * N);
    nr = N;
  }
  const double phi = nr > 0 ? 0.25 * M_PI * (jpll[f] + (x - y) / nr) : 0.0;
  double omz;  // 1 - |z| exactly in the polar caps
  if (jr < N) omz = jr * jr / (3.0 * N * N);
  else if (jr > 3.0 * N) omz = (4.0 * N - jr) * (4.0 * N - jr) / (3.0 * N * N);
  else omz = 1.0 - fabs(z);
  const double st = sqrt(omz * (2.0 - omz));
  v[0] = st * cos(phi);
  v[1] = st * sin(phi);
  v[2] = z;
}

}  // namespace cr
