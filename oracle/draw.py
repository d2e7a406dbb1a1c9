"""Right-hand sides of the CR system (Section 2.3, Eq. system-explicit and
the constrained-realization construction it cites):

    b = B Y^T N^-1 d + S^-1/2 omega_1 + B Y^T N^-1/2 omega_2,

omega_1 ~ N(0, I) in the real orthonormal basis of the coefficients and
omega_2 ~ N(0, I) per pixel (N^-1/2 = 0 under the mask).  With d = 0 the
covariance of b is S^-1 + B Y^T N^-1 Y B = A, so x = A^-1 b has covariance
A^-1: the fluctuation part of a constrained realization.  Without the omega
terms b is the Wiener-filter right-hand side.

Oracle module -- test infrastructure only.

Random numbers: Philox4x32-10, the counter-based generator of Salmon, Moraes,
Dror and Shaw (2011), written here from its published definition: ten rounds
of (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1,
lo(M0 c0)) with the key bumped by the Weyl constants after every round.
Element k of stream s for right-hand side j uses counter (k >> 2, k >> 34, s, j)
and key (seed low, seed high) and takes slot k & 3 of the Box-Muller pairs
(x0, x1) -> slots 0, 1 and (x2, x3) -> slots 2, 3, with u = (x + 1/2) 2^-32:
z = sqrt(-2 ln u_a) (cos, sin)(2 pi u_b).
Streams: 3 = omega_1, 4 = omega_2.
Coefficient element k = 2 i + part (i the m-major storage index, part 0 real,
1 imaginary); m = 0 uses only the real part; pixel element k = pixel index.
"""
import math

import numpy as np

from . import sht

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF
STREAM_OMEGA1, STREAM_OMEGA2 = 3, 4


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on uint32 arrays (as uint64 for products)."""
    c = [np.asarray(v, dtype=np.uint64) & MASK for v in (c0, c1, c2, c3)]
    k0, k1 = int(k0) & MASK, int(k1) & MASK
    for _ in range(10):
        p0 = np.uint64(M0) * c[0]
        p1 = np.uint64(M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK)
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
        k0 = (k0 + W0) & MASK
        k1 = (k1 + W1) & MASK
    return c


def normals(seed, stream, n, rhs=0):
    """n standard normals of one stream (elements 0..n-1)."""
    k = np.arange(n, dtype=np.uint64)
    ctr = k >> np.uint64(2)
    x = philox4x32_10(ctr & np.uint64(MASK), ctr >> np.uint64(32), np.full_like(ctr, stream), np.full_like(ctr, rhs),
                      seed & MASK, (seed >> 32) & MASK)
    slot = (k & np.uint64(3)).astype(np.int64)
    a = np.where(slot < 2, x[0], x[2]).astype(np.float64)
    b = np.where(slot < 2, x[1], x[3]).astype(np.float64)
    ua = (a + 0.5) * 2.0 ** -32
    ub = (b + 0.5) * 2.0 ** -32
    r = np.sqrt(-2.0 * np.log(ua))
    return np.where(slot % 2 == 0, r * np.cos(2.0 * math.pi * ub), r * np.sin(2.0 * math.pi * ub))


def draw_rhs(prob, seed, d=None, fluct=True, rhs=0):
    """b of the module docstring for the problem ``prob`` (complex m >= 0
    coefficients of band limit prob.lmax)."""
    L = prob.lmax
    npix = prob.grid["npix"]
    mp = np.zeros(npix)
    if d is not None:
        mp += prob.ninv * np.asarray(d, dtype=np.float64)
    if fluct:
        mp += np.sqrt(np.maximum(prob.ninv, 0.0)) * normals(seed, STREAM_OMEGA2, npix, rhs)
    bl = prob.bl[prob.l]
    b = bl * sht.adjoint(mp, L, prob.grid)
    if fluct:
        n = sht.n_lm(L)
        w = normals(seed, STREAM_OMEGA1, 2 * n, rhs)
        a = np.where(prob.m == 0, w[0::2] + 0j, (w[0::2] + 1j * w[1::2]) / math.sqrt(2.0))
        act = prob.active
        b[act] += a[act] / np.sqrt(prob.cl[prob.l[act]])
    return prob.clean(b)


def rademacher(seed, stream, n, j=0):
    """n Rademacher signs of one stream for probe j: element k takes word
    k & 3 of Philox4x32-10 at counter (k >> 2, k >> 34, stream, j); + for an
    even word.  Streams: 5 = coefficient probes, 6 = pixel probes."""
    k = np.arange(n, dtype=np.uint64)
    ctr = k >> np.uint64(2)
    x = philox4x32_10(ctr & np.uint64(MASK), ctr >> np.uint64(32), np.full_like(ctr, stream), np.full_like(ctr, j),
                      seed & MASK, (seed >> 32) & MASK)
    slot = (k & np.uint64(3)).astype(np.int64)
    word = np.choose(slot, x)
    return np.where(word & np.uint64(1), -1.0, 1.0)
