"""The seeded synthetic inputs follow the stated recipe: the ring table the
masks and noise are placed with is the HEALPix ring scheme (against the
oracle's independent geometry), noise RMS is log-uniform in the configured
range, the galactic cut removes the band |b| < b_cut (sky fraction
sin b_cut) and the holes add about their area, the Gaussian beam halves at
FWHM / 2 in real space, the prior draw has variance C_l per real degree of
freedom, and every preset has the configured shapes with a valid N^-1."""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import geometry
from paper_1308_5299_gb300 import synthetic


@pytest.mark.parametrize("nside", [8, 64])
def test_ring_table_is_the_healpix_ring_scheme(nside):
    z, nphi, phi0, off = synthetic.healpix_ring_table(nside)
    g = geometry.healpix_grid(nside)
    np.testing.assert_allclose(z, g["z"], atol=1e-14)
    np.testing.assert_array_equal(nphi, g["nphi"])
    np.testing.assert_array_equal(off, g["off"])
    np.testing.assert_allclose(phi0, g["phi0"], atol=1e-14)


def test_noise_rms_log_uniform_in_range():
    lo, hi = 10.0, 60.0
    sig = synthetic.noise_rms(64, lo, hi)
    assert sig.min() >= lo and sig.max() <= hi
    u = (np.log(sig) - math.log(lo)) / (math.log(hi) - math.log(lo))
    # uniform on [0, 1]: mean 1/2, variance 1/12, quartiles at 1/4, 3/4
    n = u.size
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)
    assert abs(np.quantile(u, 0.25) - 0.25) < 0.01 and abs(np.quantile(u, 0.75) - 0.75) < 0.01


def test_mask_cut_fraction_and_holes():
    nside = 128
    npix = 12 * nside * nside
    m0 = synthetic.mask(nside, 15.0, 0, 0.0)
    # |b| < 15 deg removes the fraction sin(15 deg) of the sky (equal-area pixels)
    assert abs((1.0 - m0.mean()) - math.sin(math.radians(15.0))) < 0.01
    m1 = synthetic.mask(nside, 15.0, 200, 60.0)
    extra = (m0.sum() - m1.sum()) / npix
    # 200 holes of radius 1 deg, about a fraction (1 - sin 15 deg) outside the cut
    cap = 2.0 * math.pi * (1.0 - math.cos(math.radians(1.0))) / (4.0 * math.pi)
    expect = 200 * cap * (1.0 - math.sin(math.radians(15.0)))
    assert 0.6 * expect < extra < 1.2 * expect
    assert set(np.unique(m1)) <= {0.0, 1.0}


def test_gaussian_beam_halves_at_half_fwhm():
    fwhm = 180.0  # arcmin
    L = 600
    b = synthetic.gaussian_beam(L, fwhm)
    l = np.arange(L + 1)

    def profile(theta):
        return np.sum((2 * l + 1) / (4 * np.pi) * b * eval_legendre(l, math.cos(theta)))

    ratio = profile(math.radians(fwhm / 60.0 / 2.0)) / profile(0.0)
    assert abs(ratio - 0.5) < 0.01


def test_prior_draw_variance_is_cl():
    L = 40
    cl = synthetic.cl_spectrum(L, False, "c2")
    acc = np.zeros(L + 1)
    ndraw = 300
    for k in range(ndraw):
        x = synthetic.draw_prior(cl, index=k)
        off = 0
        for m in range(L + 1):
            n = L + 1 - m
            seg = x[off:off + n]
            # real-basis dofs: x_l0, sqrt2 Re x_lm, sqrt2 Im x_lm
            acc[m:] += seg.real ** 2 if m == 0 else 2.0 * np.abs(seg) ** 2
            off += n
    dof = 2 * np.arange(L + 1) + 1
    ratio = acc / (ndraw * dof * cl)
    # each l averages ndraw * (2l+1) chi-square(1) variables
    tol = 5.0 * np.sqrt(2.0 / (ndraw * dof))
    assert np.all(np.abs(ratio - 1.0) < tol)


@pytest.mark.parametrize("name", ["nside8_lmax23", "nside16_lmax47", "nside32_lmax95", "nside256_lmax767"])
def test_presets_shapes_and_valid_inverse_noise(name):
    cfg, cl, bl, ninv = synthetic.problem_inputs(name)
    assert cl.shape == bl.shape == (cfg["lmax"] + 1,)
    assert ninv.shape == (12 * cfg["nside"] ** 2,)
    assert np.all(np.isfinite(ninv)) and np.all(ninv >= 0)
    lo, hi = cfg["rms"]
    obs = ninv > 0
    # observed pixels: N^-1 = 1 / rms^2 within the configured range (modulation widens it)
    span = math.exp(0.3 * 6.0) if cfg["modulation"] else 1.0
    assert ninv[obs].min() >= 1.0 / (hi * span) ** 2 * (1 - 1e-12)
    assert ninv[obs].max() <= (span / lo) ** 2 * (1 + 1e-12)
    if cfg["cl_low"] == "zero":
        assert cl[0] == cl[1] == 0.0
    else:
        assert cl[0] == cl[1] == cl[2] > 0
