"""Ring grids on the sphere (Section 2.1: HEALPix and Gauss-Legendre grids).

Oracle module -- test infrastructure only (see ``oracle/__init__``).

A grid is a dict of per-ring arrays, rings ordered north to south:
  z      cos(colatitude)
  sth    sin(colatitude), computed from the exact 1 - z where possible
  nphi   pixels on the ring (int64)
  off    index of the ring's first pixel in the map (int64)
  phi0   azimuth of the ring's first pixel; pixel j sits at phi0 + 2 pi j / nphi
  wgt    quadrature weight per pixel of the ring (pixel area for HEALPix)
HEALPix rings follow Gorski et al. (2005): for Nside N there are 4N-1 rings;
polar ring i (1 <= i < N, and its mirror 4N-i) has 4i pixels at
z = 1 - i^2/(3N^2) with phi = (pi / 2i)(j + 1/2); equatorial ring i
(N <= i <= 3N) has 4N pixels at z = 4/3 - 2i/(3N) with
phi = (pi / 2N)(j + s/2), s = (i - N + 1) mod 2.
"""
import numpy as np


def healpix_grid(nside):
    N = int(nside)
    rings = []
    for i in range(1, 4 * N):
        if i < N or i > 3 * N:
            ii = i if i < N else 4 * N - i
            one_minus_z = ii * ii / (3.0 * N * N)  # 1 - |z|
            z = 1.0 - one_minus_z
            sth = np.sqrt(one_minus_z * (2.0 - one_minus_z))
            if i > 3 * N:
                z = -z
            n = 4 * ii
            phi0 = np.pi / (4.0 * ii)
        else:
            z = 4.0 / 3.0 - 2.0 * i / (3.0 * N)
            sth = np.sqrt((1.0 - z) * (1.0 + z))
            n = 4 * N
            s = (i - N + 1) % 2
            phi0 = np.pi / (2.0 * N) * (s / 2.0)
        rings.append((z, sth, n, phi0))
    z = np.array([r[0] for r in rings])
    sth = np.array([r[1] for r in rings])
    nphi = np.array([r[2] for r in rings], dtype=np.int64)
    phi0 = np.array([r[3] for r in rings])
    off = np.concatenate([[0], np.cumsum(nphi)[:-1]]).astype(np.int64)
    npix = 12 * N * N
    wgt = np.full(len(z), 4.0 * np.pi / npix)
    return dict(kind="healpix", nside=N, z=z, sth=sth, nphi=nphi, off=off, phi0=phi0, wgt=wgt,
                npix=int(npix), nring=len(z))


def gl_grid(ntheta, nphi):
    """Gauss-Legendre grid: ntheta rings at the roots of P_ntheta, nphi
    equispaced pixels per ring starting at phi = 0; the pixel weight is the
    Gauss weight times 2 pi / nphi."""
    x, w = np.polynomial.legendre.leggauss(int(ntheta))
    order = np.argsort(-x)
    z = x[order]
    w = w[order]
    theta = np.arccos(z)
    sth = np.sin(theta)
    nphi_arr = np.full(len(z), int(nphi), dtype=np.int64)
    off = (np.arange(len(z)) * int(nphi)).astype(np.int64)
    return dict(kind="gl", z=z, sth=sth, nphi=nphi_arr, off=off, phi0=np.zeros(len(z)),
                wgt=w * 2.0 * np.pi / nphi, npix=int(ntheta) * int(nphi), nring=len(z))


def pixel_centres(grid):
    """(theta, phi) of every pixel, in map order."""
    th = np.repeat(np.arccos(np.clip(grid["z"], -1, 1)), grid["nphi"])
    ring = np.repeat(np.arange(grid["nring"]), grid["nphi"])
    j = np.arange(grid["npix"]) - grid["off"][ring]
    phi = grid["phi0"][ring] + 2.0 * np.pi * j / grid["nphi"][ring]
    return th, phi


def pixel_vectors(grid):
    th, phi = pixel_centres(grid)
    return np.stack([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)], axis=1)


def pixel_weights(grid):
    return np.repeat(grid["wgt"], grid["nphi"])
