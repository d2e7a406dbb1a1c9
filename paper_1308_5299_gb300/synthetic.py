"""Seeded synthetic inputs shaped like the paper's Planck-143 workload.

This module is shared by the tests, the benchmark and the oracle's test
cases.  It generates INPUT DATA only (power spectra, beams, noise and mask
maps, prior draws) and holds none of the solver's arithmetic: no spherical
harmonic transform, no operator, no solver.

The paper's inputs (the Planck 2013 143 GHz RMS map, beam, masks and the
LCDM spectrum, Section 4.1) are not available, so seeded stand-ins with the
same shapes are used:
  * C_l: 1e3 / (l(l+1)) uK^2 for l >= 2, optionally damped by
    exp(-l^2 / 2000^2), and C_0 = C_1 = C_2, the wide monopole/dipole prior of
    Section 4.1 (``low="zero"`` gives C_0 = C_1 = 0 instead, for tests of the
    inactive-multipole handling);
  * Gaussian beams b_l = exp(-l(l+1) sigma^2 / 2), sigma = FWHM / sqrt(8 ln 2);
    the pixel window is 1;
  * white noise with per-pixel RMS log-uniform in [lo, hi] uK, optionally
    modulated by exp(0.3 g), g a smooth unit-variance random field with a
    5-degree-FWHM Gaussian correlation (random-phase plane waves);
  * masks: a galactic cut |b| < b_cut (grid pole = galactic pole) plus random
    circular holes of a given radius with centres uniform on the sphere;
    masked pixels have N^-1 = 0;
  * prior draws x ~ N(0, S) in the real spherical-harmonic basis.
Random streams (numpy Philox bit generator keyed by (seed, stream)):
0 = RMS map, 1 = holes, 2 = x_true, 3 = omega_1, 4 = omega_2, 5 = modulation.

Coefficient storage everywhere in this project: complex, m >= 0, m-major with
l = m..lmax contiguous.
"""
import math

import numpy as np

BASE_SEED = 1308

# Workload presets (sizes, spectra, beams, noise and masks of the five
# configurations the solver is exercised on; see the paper's Section 4.1 for
# the Planck setup these imitate).  cl_low: "c2" is the paper's wide
# monopole/dipole prior C_0 = C_1 = C_2; "zero" conditions on l = 0, 1
# (C_0 = C_1 = 0), which the small FP64 cases use.
CONFIGS = {
    # plain FP64 method, small: Nside 32, lmax 95, no spectral damping
    "nside32_lmax95": dict(nside=32, lmax=95, damp=False, cl_low="zero", fwhm_arcmin=180.0, rms=(5.0, 50.0),
                           modulation=False, gal_cut_deg=20.0, holes=0, hole_radius_arcmin=0.0),
    # plain FP64 method, medium: Nside 256, lmax 767, modulated noise, 200 holes
    "nside256_lmax767": dict(nside=256, lmax=767, damp=True, cl_low="zero", fwhm_arcmin=20.0, rms=(2.0, 30.0),
                             modulation=True, gal_cut_deg=15.0, holes=200, hole_radius_arcmin=60.0),
    # Planck-143-shaped: Nside 2048, lmax 3000, 7.3' beam, 3000 holes of 5'
    "nside2048_lmax3000": dict(nside=2048, lmax=3000, damp=True, cl_low="c2", fwhm_arcmin=7.3, rms=(10.0, 60.0),
                               modulation=False, gal_cut_deg=10.0, holes=3000, hole_radius_arcmin=5.0),
    # batched mixed resolutions
    "nside1024_lmax2047": dict(nside=1024, lmax=2047, damp=True, cl_low="c2", fwhm_arcmin=7.3, rms=(10.0, 60.0),
                               modulation=False, gal_cut_deg=10.0, holes=3000, hole_radius_arcmin=5.0),
    "nside512_lmax1023": dict(nside=512, lmax=1023, damp=True, cl_low="c2", fwhm_arcmin=7.3, rms=(10.0, 60.0),
                              modulation=False, gal_cut_deg=10.0, holes=3000, hole_radius_arcmin=5.0),
    # tiny cases the dense oracle solves exactly
    "nside8_lmax23": dict(nside=8, lmax=23, damp=True, cl_low="c2", fwhm_arcmin=180.0, rms=(10.0, 60.0),
                          modulation=False, gal_cut_deg=10.0, holes=3, hole_radius_arcmin=300.0),
    "nside16_lmax47": dict(nside=16, lmax=47, damp=True, cl_low="zero", fwhm_arcmin=120.0, rms=(10.0, 60.0),
                           modulation=False, gal_cut_deg=10.0, holes=4, hole_radius_arcmin=300.0),
}


def rng(seed, stream):
    return np.random.Generator(np.random.Philox(key=[int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream)]))


def cl_spectrum(lmax, damp, low="c2"):
    """Prior spectrum.  With C_0 = C_1 = 0 every level's beam kernel
    sum_l (2l+1)/(4 pi) f_l b_l P_l loses its monopole and dipole and gets a
    negative floor over the whole sphere, so the pixel smoothers' block
    pattern misses a large part of A_hat; Section 4.1 sets C_0 = C_1 = C_2."""
    l = np.arange(lmax + 1, dtype=np.float64)
    cl = np.zeros(lmax + 1)
    cl[2:] = 1e3 / (l[2:] * (l[2:] + 1.0))
    if damp:
        cl *= np.exp(-(l * l) / (2000.0 ** 2))
    if low == "c2" and lmax >= 2:
        cl[0] = cl[1] = cl[2]
    elif low != "zero":
        raise ValueError("low must be 'c2' or 'zero'")
    return cl


def gaussian_beam(lmax, fwhm_arcmin):
    sigma = fwhm_arcmin / 60.0 * math.pi / 180.0 / math.sqrt(8.0 * math.log(2.0))
    l = np.arange(lmax + 1, dtype=np.float64)
    return np.exp(-0.5 * l * (l + 1.0) * sigma * sigma)


def healpix_ring_table(nside):
    """Per-ring (z, nphi, phi0, first pixel) of the HEALPix RING scheme, for
    placing masks and noise (Gorski et al. 2005 pixel centres)."""
    N = int(nside)
    i = np.arange(1, 4 * N, dtype=np.int64)
    north = i < N
    south = i > 3 * N
    ii = np.where(north, i, np.where(south, 4 * N - i, N))
    z = np.where(north | south, 1.0 - ii * ii / (3.0 * N * N), 0.0)
    z = np.where(south, -z, z)
    eq = ~(north | south)
    z = np.where(eq, 4.0 / 3.0 - 2.0 * i / (3.0 * N), z)
    nphi = np.where(eq, 4 * N, 4 * ii)
    s = (i - N + 1) % 2
    phi0 = np.where(eq, np.pi / (2.0 * N) * (s / 2.0), np.pi / (4.0 * ii))
    off = np.concatenate([[0], np.cumsum(nphi)[:-1]])
    return z, nphi, phi0, off


def _pixels_near(nside, vec, radius, table):
    """Indices of RING pixels whose centre lies within ``radius`` of unit
    vector ``vec``."""
    z, nphi, phi0, off = table
    th_c = math.acos(max(-1.0, min(1.0, vec[2])))
    ph_c = math.atan2(vec[1], vec[0])
    th = np.arccos(z)
    rings = np.nonzero(np.abs(th - th_c) <= radius + 1e-12)[0]
    out = []
    cosr = math.cos(radius)
    for k in rings:
        n = int(nphi[k])
        phi = phi0[k] + 2.0 * np.pi * np.arange(n) / n
        st = math.sin(th[k])
        cosd = st * math.sin(th_c) * np.cos(phi - ph_c) + z[k] * vec[2]
        sel = np.nonzero(cosd >= cosr)[0]
        out.append(off[k] + sel)
    return np.concatenate(out) if out else np.zeros(0, dtype=np.int64)


def smooth_field(nside, fwhm_deg, seed, table, nwaves=256):
    """Smooth, approximately Gaussian random field with unit variance and a
    Gaussian correlation of the given FWHM: a random-phase sum of 3-D plane
    waves cos(k . n + phi) restricted to the sphere, with wave vectors
    k ~ N(0, I / s^2), s = FWHM / sqrt(8 ln 2), so that
    E[f(n1) f(n2)] = exp(-|n1 - n2|^2 / (2 s^2)) ~ exp(-theta^2 / (2 s^2))."""
    z, nphi, phi0, off = table
    npix = 12 * nside * nside
    g = rng(seed, 5)
    s = math.radians(fwhm_deg) / math.sqrt(8.0 * math.log(2.0))
    k = g.normal(size=(nwaves, 3)) / s
    ph = g.uniform(0.0, 2.0 * np.pi, size=nwaves)
    th = np.repeat(np.arccos(z), nphi)
    ring = np.repeat(np.arange(len(z)), nphi)
    phi = phi0[ring] + 2.0 * np.pi * (np.arange(npix) - off[ring]) / nphi[ring]
    v = np.stack([np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi), np.cos(th)], axis=1)
    f = np.zeros(npix)
    for b0 in range(0, nwaves, 32):
        f += np.cos(v @ k[b0:b0 + 32].T + ph[b0:b0 + 32]).sum(axis=1)
    f *= math.sqrt(2.0 / nwaves)
    return f


def noise_rms(nside, lo, hi, seed=BASE_SEED, modulation=False, table=None):
    table = table or healpix_ring_table(nside)
    npix = 12 * nside * nside
    u = rng(seed, 0).uniform(size=npix)
    sig = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))
    if modulation:
        sig *= np.exp(0.3 * smooth_field(nside, 5.0, seed, table))
    return sig


def mask(nside, gal_cut_deg, holes, hole_radius_arcmin, seed=BASE_SEED, table=None):
    """1 = observed, 0 = masked."""
    table = table or healpix_ring_table(nside)
    z, nphi, phi0, off = table
    zpix = np.repeat(z, nphi)
    m = (np.abs(zpix) >= math.sin(math.radians(gal_cut_deg))).astype(np.float64)
    if holes:
        g = rng(seed, 1)
        c = g.normal(size=(holes, 3))
        c /= np.linalg.norm(c, axis=1, keepdims=True)
        r = math.radians(hole_radius_arcmin / 60.0)
        for h in range(holes):
            m[_pixels_near(nside, c[h], r, table)] = 0.0
    return m


def draw_prior(cl, seed=BASE_SEED, stream=2, index=0):
    """x ~ N(0, S): real-basis variance C_l per degree of freedom, i.e.
    x_l0 = sqrt(C_l) g, x_lm = sqrt(C_l / 2) (g1 + i g2) for m > 0."""
    lmax = len(cl) - 1
    g = rng(seed * 1000003 + index, stream)
    out = []
    for m in range(lmax + 1):
        c = np.sqrt(cl[m:])
        if m == 0:
            out.append(c * g.normal(size=lmax + 1) + 0j)
        else:
            re = g.normal(size=lmax + 1 - m)
            im = g.normal(size=lmax + 1 - m)
            out.append(c * (re + 1j * im) / math.sqrt(2.0))
    return np.concatenate(out)


def random_alm(lmax, seed, stream=7):
    """Unit-variance random coefficients (m = 0 real) for transform tests."""
    g = rng(seed, stream)
    n = (lmax + 1) * (lmax + 2) // 2
    a = g.normal(size=n) + 1j * g.normal(size=n)
    a[: lmax + 1] = a[: lmax + 1].real
    return a


def random_map(npix, seed, stream=8):
    return rng(seed, stream).normal(size=npix)


def problem_inputs(name, seed=BASE_SEED):
    """(cfg, cl, bl, ninv) for a named preset; ninv = mask / rms^2 (uK^-2)."""
    cfg = CONFIGS[name]
    nside, lmax = cfg["nside"], cfg["lmax"]
    table = healpix_ring_table(nside)
    cl = cl_spectrum(lmax, cfg["damp"], cfg["cl_low"])
    bl = gaussian_beam(lmax, cfg["fwhm_arcmin"])
    rms = noise_rms(nside, *cfg["rms"], seed=seed, modulation=cfg["modulation"], table=table)
    msk = mask(nside, cfg["gal_cut_deg"], cfg["holes"], cfg["hole_radius_arcmin"], seed=seed, table=table)
    ninv = msk / (rms * rms)
    return cfg, cl, bl, ninv
