"""Pins of the oracle's right-hand-side generator (oracle/draw.py): the
Philox4x32-10 normals have the moments and distribution of N(0, 1) and
independent streams, and the constrained-realization right-hand side with
d = 0 has covariance A (the defining property of the construction in
Section 2.3): a dropped term, a wrong sqrt(2) or a wrong N^-1/2 fails it."""
import math

import numpy as np
import scipy.stats

from oracle import draw, geometry, operators, sht


def test_normals_moments_and_distribution():
    z = draw.normals(1308, 3, 200000)
    assert abs(z.mean()) < 5.0 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 5.0 * math.sqrt(2.0 / z.size)
    assert scipy.stats.kstest(z, "norm").pvalue > 1e-4
    # fourth moment of N(0, 1) is 3
    assert abs(np.mean(z ** 4) - 3.0) < 0.1


def test_streams_seeds_and_rhs_are_independent():
    a = draw.normals(1308, 3, 50000)
    for other in (draw.normals(1308, 4, 50000), draw.normals(1309, 3, 50000), draw.normals(1308, 3, 50000, rhs=1)):
        assert abs(np.corrcoef(a, other)[0, 1]) < 5.0 / math.sqrt(a.size)
    assert np.array_equal(a, draw.normals(1308, 3, 50000))


def test_philox_is_a_bijection_on_a_small_domain():
    # each round is invertible for a fixed key, so distinct counters give
    # distinct outputs
    c = np.arange(4096, dtype=np.uint64)
    x = draw.philox4x32_10(c, np.zeros_like(c), np.zeros_like(c), np.zeros_like(c), 7, 9)
    keys = set(zip(*(v.tolist() for v in x)))
    assert len(keys) == c.size


def test_constrained_realization_rhs_covariance_is_A():
    nside, L = 4, 7
    g = geometry.healpix_grid(nside)
    cl = np.zeros(L + 1)
    cl[2:] = 1.0 / np.arange(2, L + 1) ** 2
    bl = np.exp(-0.02 * np.arange(L + 1) * np.arange(1, L + 2))
    rng = np.random.default_rng(5)
    ninv = rng.uniform(0.5, 2.0, size=g["npix"])
    ninv[: g["npix"] // 5] = 0.0
    prob = operators.Problem(L, cl, bl, ninv, g)
    act = operators.real_active_mask(prob)
    A = operators.dense_matrix(lambda v: operators.apply_A(prob, v), L, act)
    nd = 6000
    U = np.stack([sht.alm_to_real(draw.draw_rhs(prob, 77, rhs=j), L)[act] for j in range(nd)])
    Cov = U.T @ U / nd
    # entrywise standard error of a sample covariance: sqrt((A_ii A_jj + A_ij^2) / nd)
    dA = np.sqrt(np.outer(np.diag(A), np.diag(A)) + A ** 2) / math.sqrt(nd)
    z = (Cov - A) / dA
    assert np.max(np.abs(z)) < 5.5
    assert abs(np.mean(z)) < 0.2
