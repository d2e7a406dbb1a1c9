"""Pins for the oracle's grids and direct transforms, against things fixed
independently of the oracle: published grid definitions, closed-form Y_lm,
scipy / mpmath special functions, the addition theorem, exact quadrature and
the transpose identity (Section 2.1, Eq. sh-synthesis, Section 3.3)."""
import math
import os

import numpy as np
import pytest
import scipy.special as ss

from oracle import geometry, sht

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_healpix_ring_table_golden():
    g = geometry.healpix_grid(2)
    rows = np.loadtxt(os.path.join(GOLDEN, "healpix_nside2_rings.txt"))
    assert g["nring"] == len(rows)
    np.testing.assert_allclose(g["z"], rows[:, 1] / rows[:, 2], atol=1e-15)
    np.testing.assert_array_equal(g["nphi"], rows[:, 3].astype(int))
    np.testing.assert_allclose(g["phi0"] / np.pi, rows[:, 4], atol=1e-15)
    np.testing.assert_array_equal(g["off"], rows[:, 5].astype(int))


@pytest.mark.parametrize("nside", [1, 2, 4, 16, 64])
def test_healpix_counts_and_area(nside):
    g = geometry.healpix_grid(nside)
    assert g["npix"] == 12 * nside * nside == int(g["nphi"].sum())
    assert g["nring"] == 4 * nside - 1
    assert abs(g["wgt"] @ g["nphi"] - 4 * math.pi) < 1e-12
    # north/south mirror symmetry
    np.testing.assert_allclose(g["z"], -g["z"][::-1], atol=1e-15)
    np.testing.assert_allclose(g["sth"] ** 2 + g["z"] ** 2, 1.0, atol=1e-15)
    # equal-area rings: each polar cap holds N^2 * 2 pixels... total cap = 2N(N-1)
    assert int(g["nphi"][: nside - 1].sum()) == 2 * nside * (nside - 1)


def _textbook_plm(l, m, z):
    """Normalised P~_lm with Condon-Shortley phase for l <= 3 (standard
    tables of Y_lm)."""
    s = math.sqrt(1 - z * z)
    pi = math.pi
    tab = {
        (0, 0): math.sqrt(1 / (4 * pi)),
        (1, 0): math.sqrt(3 / (4 * pi)) * z,
        (1, 1): -math.sqrt(3 / (8 * pi)) * s,
        (2, 0): math.sqrt(5 / (16 * pi)) * (3 * z * z - 1),
        (2, 1): -math.sqrt(15 / (8 * pi)) * s * z,
        (2, 2): math.sqrt(15 / (32 * pi)) * s * s,
        (3, 0): math.sqrt(7 / (16 * pi)) * (5 * z ** 3 - 3 * z),
        (3, 1): -math.sqrt(21 / (64 * pi)) * s * (5 * z * z - 1),
        (3, 2): math.sqrt(105 / (32 * pi)) * s * s * z,
        (3, 3): -math.sqrt(35 / (64 * pi)) * s ** 3,
    }
    return tab[(l, m)]


@pytest.mark.parametrize("z", [-0.93, -0.2, 0.0, 0.41, 0.999])
def test_plm_closed_forms(z):
    for m in range(4):
        col = sht.plm(3, m, z)
        for l in range(m, 4):
            assert abs(col[l - m] - _textbook_plm(l, m, z)) < 1e-14


def test_plm_vs_scipy():
    for z in [-0.8, 0.05, 0.6, 0.97]:
        th = math.acos(z)
        for m in [0, 1, 7, 40, 120]:
            col = sht.plm(150, m, z)
            ref = ss.sph_legendre_p(np.arange(m, 151), m, th)
            assert np.max(np.abs(col - ref)) < 1e-12


def test_plm_high_degree_vs_mpmath():
    """High l and m, including seeds far below the FP64 range
    (sin^2000(theta) ~ 1e-310 at z = 0.7), against 40-digit mpmath."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    for (l, m, z) in [(3000, 2000, 0.7), (2500, 1700, 0.7), (3000, 10, 0.9999), (1200, 600, -0.3),
                      (3000, 2990, 0.05)]:
        col = sht.plm(l, m, z)
        zz = mpmath.mpf(z)
        norm = mpmath.sqrt((2 * l + 1) / (4 * mpmath.pi) * mpmath.factorial(l - m) / mpmath.factorial(l + m))
        ref = float(norm * mpmath.legenp(l, m, zz, type=2))
        assert abs(col[-1] - ref) <= 1e-11 * max(1.0, abs(ref)), (l, m, z, col[-1], ref)


@pytest.mark.parametrize("z", [0.9999999, 0.999, 0.5, 0.0])
def test_sum_rule_high_l(z):
    """Addition theorem at zero separation: sum_m |Y_lm|^2 = (2l+1)/(4 pi)."""
    L = 3000
    acc = np.zeros(L + 1)
    for m in range(L + 1):
        col = sht.plm(L, m, z)
        acc[m:] += (1.0 if m == 0 else 2.0) * col * col
    l = np.arange(L + 1)
    # FP64 three-term recurrence over 3000 steps: rounding accumulates to ~1e-11
    np.testing.assert_allclose(acc, (2 * l + 1) / (4 * math.pi), rtol=3e-11)


@pytest.mark.parametrize("nside,lmax", [(4, 10), (8, 20)])
def test_synth_unit_vs_scipy(nside, lmax):
    """Y applied to one unit coefficient equals 2 Re Y_lm (or Y_l0) at every
    HEALPix pixel centre, with scipy's spherical harmonics."""
    g = geometry.healpix_grid(nside)
    th, ph = geometry.pixel_centres(g)
    for (l, m) in [(0, 0), (3, 0), (5, 2), (lmax, 1), (lmax, lmax), (lmax - 3, lmax - 5)]:
        for c in (1.0, 1j):
            if m == 0 and c == 1j:
                continue
            a = np.zeros(sht.n_lm(lmax), dtype=np.complex128)
            a[sht.lm_index(lmax, l, m)] = c
            ref = ss.sph_harm_y(l, m, th, ph)
            ref = (ref.real if m == 0 else 2 * np.real(c * ref))
            np.testing.assert_allclose(sht.synth(a, lmax, g), ref, atol=1e-13)


@pytest.mark.parametrize("grid,lmax", [("hp8", 23), ("hp8", 40), ("hp4", 30), ("gl", 19)])
def test_adjoint_identity(grid, lmax):
    """<Y x, y> = <x, Y^T y> (Y^T is the transpose of Y), including band
    limits above what the grid resolves (aliasing in the polar caps)."""
    g = {"hp8": lambda: geometry.healpix_grid(8), "hp4": lambda: geometry.healpix_grid(4),
         "gl": lambda: geometry.gl_grid(20, 41)}[grid]()
    rs = np.random.default_rng(5)
    x = rs.normal(size=sht.n_lm(lmax)) + 1j * rs.normal(size=sht.n_lm(lmax))
    x[: lmax + 1] = x[: lmax + 1].real
    y = rs.normal(size=g["npix"])
    lhs = float(sht.synth(x, lmax, g) @ y)
    rhs = sht.alm_dot(x, sht.adjoint(y, lmax, g), lmax)
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.linalg.norm(y) * np.linalg.norm(x))


def test_gl_exact_roundtrip():
    """On a Gauss-Legendre grid with ntheta >= lmax+1 and nphi >= 2 lmax+1,
    Y^T W Y = I exactly (Eq. sh-analysis is exact quadrature there)."""
    L = 24
    g = geometry.gl_grid(L + 1, 2 * L + 1)
    rs = np.random.default_rng(1)
    a = rs.normal(size=sht.n_lm(L)) + 1j * rs.normal(size=sht.n_lm(L))
    a[: L + 1] = a[: L + 1].real
    back = sht.adjoint(geometry.pixel_weights(g) * sht.synth(a, L, g), L, g)
    assert np.max(np.abs(back - a)) < 1e-13


def test_monopole_adjoint():
    g = geometry.healpix_grid(8)
    a = sht.adjoint(np.ones(g["npix"]), 8, g)
    assert abs(a[0] - g["npix"] / math.sqrt(4 * math.pi)) < 1e-11


def test_addition_theorem_pair():
    """sum_m Y_lm(n1) Y*_lm(n2) = (2l+1)/(4 pi) P_l(n1.n2), through the
    oracle's P~_lm, at a random pair of directions."""
    L = 60
    z1, z2, dphi = 0.3, -0.45, 1.1
    acc = np.zeros(L + 1)
    for m in range(L + 1):
        p1 = sht.plm(L, m, z1)
        p2 = sht.plm(L, m, z2)
        acc[m:] += (1.0 if m == 0 else 2.0 * math.cos(m * dphi)) * p1 * p2
    cosg = z1 * z2 + math.sqrt(1 - z1 * z1) * math.sqrt(1 - z2 * z2) * math.cos(dphi)
    l = np.arange(L + 1)
    np.testing.assert_allclose(acc, (2 * l + 1) / (4 * math.pi) * ss.eval_legendre(l, cosg), atol=1e-13)
