/*
 * Plain FP64 direct spherical-harmonic synthesis Y and adjoint synthesis Y^T
 * on an iso-latitude ring grid (HEALPix or Gauss-Legendre).
 *
 * TEST INFRASTRUCTURE ONLY (the oracle).  Nothing in the product library links
 * or calls this file; only tests/, the smoke check and the CPU baseline leg of
 * the benchmark load it.  It is written for obviousness, not speed: every ring
 * is handled on its own (no north/south symmetry), Legendre functions come
 * from the textbook three-term recurrence, and the azimuthal sums are direct
 * DFTs (no FFT, no aliasing/folding logic: e^{i m phi} is evaluated for every
 * pixel and every m).
 *
 * Definitions (Section 2.1, Eq. sh-synthesis; Section 3.3 normalised P~_lm):
 *   Y_lm(theta, phi) = P~_lm(cos theta) e^{i m phi}
 *   P~_lm(z) = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_lm(z), Condon-Shortley phase
 *   synthesis  map_i = sum_{l,m=-l..l} a_lm Y_lm(n_i)
 *             = sum_l [a_l0 P~_l0 + 2 Re sum_{m>0} a_lm P~_lm e^{i m phi_i}]
 *             (real field: a_{l,-m} = (-1)^m conj(a_lm))
 *   adjoint    a_lm = sum_i Y*_lm(n_i) y_i        (transpose of synthesis
 *             with respect to <a,b> = sum a_l0 b_l0 + 2 sum_{m>0} Re(a conj b))
 *
 * a_lm layout: complex (re, im interleaved), m-major, l = m..lmax contiguous;
 * index of (l, m) = off_m + (l - m) with off_m = m (lmax + 1) - m (m - 1) / 2.
 *
 * The seed P~_mm ~ sin^m(theta) underflows FP64 near the poles for large m.
 * Values are carried as v * 2^e (integer e <= 0), starting from the exact
 * log2 of the seed; v is renormalised by 2^-RESCALE whenever it exceeds
 * 2^RESCALE, and the true value is ldexp(v, e) (which is 0 below the FP64
 * range, where the contribution is negligible).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define RESCALE 200

static int64_t lm_off(int lmax, int m) { return (int64_t)m * (lmax + 1) - (int64_t)m * (m - 1) / 2; }

/* log2 of (2m+1)/(4 pi) * prod_{i=1..m} (2i-1)/(2i), for m = 0..lmax */
static void seed_log2_table(int lmax, double *t) {
  double acc = 0.0;
  for (int m = 0; m <= lmax; ++m) {
    if (m > 0) acc += log2((2.0 * m - 1.0) / (2.0 * m));
    t[m] = log2((2.0 * m + 1.0) / (4.0 * M_PI)) + acc;
  }
}

/* P~_lm(z) for l = m..lmax, written to out[l - m]. */
static void plm_column_t(int lmax, int m, double z, double sth, const double *seedtab, double *out) {
  double v0, v1; /* v0 = P_{l-2}, v1 = P_{l-1} (scaled) */
  int e;
  if (sth <= 0.0 && m > 0) {
    for (int l = m; l <= lmax; ++l) out[l - m] = 0.0;
    return;
  }
  double lg = 0.5 * seedtab[m] + (m > 0 ? m * log2(sth) : 0.0);
  e = (int)floor(lg);
  double vmm = exp2(lg - e);
  if (m & 1) vmm = -vmm;
  out[0] = ldexp(vmm, e);
  if (m == lmax) return;
  v0 = vmm;
  v1 = z * sqrt(2.0 * m + 3.0) * vmm;
  out[1] = ldexp(v1, e);
  double a_prev = sqrt(2.0 * m + 3.0); /* a_{m+1,m} */
  for (int l = m + 2; l <= lmax; ++l) {
    double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
    double v2 = a * (z * v1 - v0 / a_prev);
    v0 = v1;
    v1 = v2;
    a_prev = a;
    if (e < 0 && fabs(v1) > ldexp(1.0, RESCALE)) {
      v0 = ldexp(v0, -RESCALE);
      v1 = ldexp(v1, -RESCALE);
      e += RESCALE;
    }
    out[l - m] = ldexp(v1, e);
  }
}

/* Public: P~_lm(z) column, for tests. */
void oracle_plm(int lmax, int m, double z, double sth, double *out) {
  double *t = (double *)malloc(sizeof(double) * (lmax + 1));
  seed_log2_table(lmax, t);
  plm_column_t(lmax, m, z, sth, t, out);
  free(t);
}

/*
 * Synthesis.  alm: complex [n_lm]; map: real [npix].
 * Ring k: cos-colatitude z[k], sin-colatitude sth[k], nphi[k] pixels starting at
 * pixel offset off[k], azimuth of pixel j = phi0[k] + 2 pi j / nphi[k].
 */
void oracle_synth(int lmax, int nring, const double *z, const double *sth, const int64_t *nphi,
                  const int64_t *off, const double *phi0, const double *alm, double *map) {
  double *seedtab = (double *)malloc(sizeof(double) * (lmax + 1));
  seed_log2_table(lmax, seedtab);
#pragma omp parallel
  {
    double *col = (double *)malloc(sizeof(double) * (lmax + 1));
    double *F = (double *)malloc(sizeof(double) * 2 * (lmax + 1)); /* F_m, complex */
#pragma omp for schedule(dynamic, 1)
    for (int k = 0; k < nring; ++k) {
      /* Legendre stage: F_m = sum_l a_lm P~_lm(z_k) */
      for (int m = 0; m <= lmax; ++m) {
        plm_column_t(lmax, m, z[k], sth[k], seedtab, col);
        double fr = 0.0, fi = 0.0;
        const double *a = alm + 2 * lm_off(lmax, m);
        for (int l = m; l <= lmax; ++l) {
          fr += a[2 * (l - m)] * col[l - m];
          fi += a[2 * (l - m) + 1] * col[l - m];
        }
        F[2 * m] = fr;
        F[2 * m + 1] = fi;
      }
      /* Direct azimuthal sum: map_j = F_0 + 2 Re sum_{m>0} F_m e^{i m phi_j} */
      int64_t n = nphi[k];
      double *ct = (double *)malloc(sizeof(double) * n), *st = (double *)malloc(sizeof(double) * n);
      for (int64_t t = 0; t < n; ++t) {
        ct[t] = cos(2.0 * M_PI * (double)t / (double)n);
        st[t] = sin(2.0 * M_PI * (double)t / (double)n);
      }
      /* F_m <- F_m e^{i m phi0} once per m */
      for (int m = 0; m <= lmax; ++m) {
        double c0 = cos(m * phi0[k]), s0 = sin(m * phi0[k]);
        double fr = F[2 * m] * c0 - F[2 * m + 1] * s0, fi = F[2 * m] * s0 + F[2 * m + 1] * c0;
        F[2 * m] = fr;
        F[2 * m + 1] = fi;
      }
      for (int64_t j = 0; j < n; ++j) {
        double s = F[0];
        for (int m = 1; m <= lmax; ++m) {
          /* m phi_j = m phi0 + 2 pi (m j mod n) / n */
          int64_t t = ((int64_t)m * j) % n;
          s += 2.0 * (F[2 * m] * ct[t] - F[2 * m + 1] * st[t]);
        }
        map[off[k] + j] = s;
      }
      free(ct);
      free(st);
    }
    free(col);
    free(F);
  }
  free(seedtab);
}

/* Adjoint synthesis.  map: real [npix]; alm: complex [n_lm] (overwritten). */
void oracle_adjoint(int lmax, int nring, const double *z, const double *sth, const int64_t *nphi,
                    const int64_t *off, const double *phi0, const double *map, double *alm) {
  double *seedtab = (double *)malloc(sizeof(double) * (lmax + 1));
  seed_log2_table(lmax, seedtab);
  /* G[k][m] = sum_j y_kj e^{-i m phi_kj} */
  double *G = (double *)malloc(sizeof(double) * 2 * (size_t)nring * (lmax + 1));
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < nring; ++k) {
    int64_t n = nphi[k];
    double *ct = (double *)malloc(sizeof(double) * n), *st = (double *)malloc(sizeof(double) * n);
    for (int64_t t = 0; t < n; ++t) {
      ct[t] = cos(2.0 * M_PI * (double)t / (double)n);
      st[t] = sin(2.0 * M_PI * (double)t / (double)n);
    }
    for (int m = 0; m <= lmax; ++m) {
      double c0 = cos(m * phi0[k]), s0 = sin(m * phi0[k]);
      double gr = 0.0, gi = 0.0;
      for (int64_t j = 0; j < n; ++j) {
        int64_t t = ((int64_t)m * j) % n;
        double c = c0 * ct[t] - s0 * st[t], sn = s0 * ct[t] + c0 * st[t];
        double y = map[off[k] + j];
        gr += y * c;
        gi -= y * sn;
      }
      G[2 * ((size_t)k * (lmax + 1) + m)] = gr;
      G[2 * ((size_t)k * (lmax + 1) + m) + 1] = gi;
    }
    free(ct);
    free(st);
  }
  /* Legendre stage: a_lm = sum_k P~_lm(z_k) G[k][m] */
#pragma omp parallel
  {
    double *col = (double *)malloc(sizeof(double) * (lmax + 1));
#pragma omp for schedule(dynamic, 1)
    for (int m = 0; m <= lmax; ++m) {
      double *a = alm + 2 * lm_off(lmax, m);
      memset(a, 0, sizeof(double) * 2 * (lmax - m + 1));
      for (int k = 0; k < nring; ++k) {
        plm_column_t(lmax, m, z[k], sth[k], seedtab, col);
        double gr = G[2 * ((size_t)k * (lmax + 1) + m)], gi = G[2 * ((size_t)k * (lmax + 1) + m) + 1];
        for (int l = m; l <= lmax; ++l) {
          a[2 * (l - m)] += col[l - m] * gr;
          a[2 * (l - m) + 1] += col[l - m] * gi;
        }
      }
    }
    free(col);
  }
  free(G);
  free(seedtab);
}

/*
 * Ring sums for the explicit inverse-noise entries (Section 3.3, Eq. Ni-dense):
 * X[k][d] = sum_j xi_kj e^{-i d phi_kj}, d = 0..dmax (direct DFT).
 */
void oracle_ring_dft(int dmax, int nring, const int64_t *nphi, const int64_t *off, const double *phi0,
                     const double *map, double *X) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < nring; ++k) {
    for (int d = 0; d <= dmax; ++d) {
      double xr = 0.0, xi = 0.0;
      for (int64_t j = 0; j < nphi[k]; ++j) {
        double ph = d * (phi0[k] + 2.0 * M_PI * (double)j / (double)nphi[k]);
        xr += map[off[k] + j] * cos(ph);
        xi -= map[off[k] + j] * sin(ph);
      }
      X[2 * ((size_t)k * (dmax + 1) + d)] = xr;
      X[2 * ((size_t)k * (dmax + 1) + d) + 1] = xi;
    }
  }
}
