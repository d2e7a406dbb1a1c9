"""Pins for the oracle's system operator and solvers (Section 2.3, Eq.
system-explicit / cr-system; Section 2.4; Section 3.3, Eq. Ni-dense):
symmetry and definiteness, closed-form solutions, and two independent routes
to the explicit matrix (probing vs the ring formula)."""

import numpy as np

from oracle import geometry, operators, sht, solvers
from paper_1308_5299_gb300 import synthetic


def small_problem(nside=4, lmax=9, seed=3, cl0=False):
    g = geometry.healpix_grid(nside)
    rs = np.random.default_rng(seed)
    l = np.arange(lmax + 1)
    cl = 1.0 / (1.0 + l) ** 2
    if cl0:
        cl[:2] = 0.0
    bl = np.exp(-0.01 * l * (l + 1))
    ninv = rs.uniform(0.5, 2.0, size=g["npix"]) * (rs.uniform(size=g["npix"]) > 0.2)
    return operators.Problem(lmax, cl, bl, ninv, g)


def test_apply_A_symmetric_positive_definite():
    p = small_problem(cl0=True)
    act = operators.real_active_mask(p)
    A = operators.dense_matrix(lambda v: operators.apply_A(p, v), p.lmax, act)
    assert np.max(np.abs(A - A.T)) < 1e-12 * np.max(np.abs(A))
    w = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert w.min() > 0


def test_no_noise_gives_prior_solution():
    """N^-1 = 0 (fully masked sky): A = S^-1, so x = S b exactly."""
    p = small_problem()
    p.ninv[:] = 0.0
    rs = np.random.default_rng(0)
    b = p.clean(rs.normal(size=sht.n_lm(p.lmax)) + 1j * rs.normal(size=sht.n_lm(p.lmax)))
    x, _ = solvers.dense_solve(p, b)
    np.testing.assert_allclose(x, p.clean(b * p.cl[p.l]), atol=1e-13)


def test_gl_weighted_noise_is_diagonal():
    """On a Gauss-Legendre grid with N^-1_j = c w_j, Y^T N^-1 Y = c I, so A is
    diagonal: A x = (1/C_l + c b_l^2) x."""
    L = 16
    g = geometry.gl_grid(L + 1, 2 * L + 1)
    l = np.arange(L + 1)
    cl = 1.0 / (1.0 + l)
    bl = np.exp(-0.003 * l * (l + 1))
    c = 7.5
    p = operators.Problem(L, cl, bl, c * geometry.pixel_weights(g), g)
    rs = np.random.default_rng(2)
    x = p.clean(rs.normal(size=sht.n_lm(L)) + 1j * rs.normal(size=sht.n_lm(L)))
    y = operators.apply_A(p, x)
    np.testing.assert_allclose(y, x * (1.0 / cl[p.l] + c * bl[p.l] ** 2), rtol=1e-12, atol=1e-12)


def test_ring_formula_equals_probing():
    """Eq. Ni-dense (per-ring DFT of the inverse-noise map) reproduces every
    entry of Y^T N^-1 Y obtained by probing the direct transforms."""
    p = small_problem(nside=4, lmax=7)
    L = 7
    probe = operators.dense_matrix(lambda v: operators.apply_inv_noise_term(p, v, lmax=L), L)
    ring = operators.ring_formula_inv_noise(p, L)
    # Im(a_l0) is not a degree of freedom in either route
    assert np.max(np.abs(probe - ring)) < 1e-12 * np.max(np.abs(probe))


def test_dm0_diagonal_exact_for_m0():
    """The Delta m = 0 ring-formula diagonal is exact for m = 0 and misses
    only the Re X(2m) term for m > 0."""
    p = small_problem(nside=4, lmax=8)
    L = 8
    dm0 = operators.diag_inv_noise_dm0(p)
    M = operators.ring_formula_inv_noise(p, L)
    full = np.diag(M)
    np.testing.assert_allclose(dm0[: L + 1], full[: L + 1], rtol=1e-12)
    X = sht.ring_dft(p.ninv, p.grid, 2 * L)
    for m in range(1, L + 1):
        for lv in range(m, L + 1):
            pk = np.array([sht.plm(L, m, p.grid["z"][k], p.grid["sth"][k])[lv - m] for k in range(p.grid["nring"])])
            i = sht.lm_index(L, lv, m)
            re_part = full[L + 1 + 2 * (i - (L + 1))]
            exact = np.sum(pk * pk * (X[:, 0].real + X[:, 2 * m].real))
            assert abs(re_part - exact) < 1e-12 * abs(exact)
            assert abs(dm0[i] - np.sum(pk * pk * X[:, 0].real)) < 1e-12 * abs(exact)


def test_dense_solve_equals_cg():
    """Two independent routes to x* = A^-1 b agree (tiny Planck-shaped case)."""
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside8_lmax23")
    g = geometry.healpix_grid(cfg["nside"])
    p = operators.Problem(cfg["lmax"], cl, bl, ninv, g)
    x_true = synthetic.draw_prior(cl)
    b = operators.apply_A(p, x_true)
    xd, A = solvers.dense_solve(p, b)
    assert np.max(np.abs(xd - p.clean(x_true))) < 1e-9 * np.max(np.abs(x_true))
    diag = np.zeros(sht.n_lm(p.lmax))
    dm0 = operators.diag_inv_noise_dm0(p)
    diag[p.active] = 1.0 / (1.0 / cl[p.l[p.active]] + bl[p.l[p.active]] ** 2 * dm0[p.active])
    xc, it, rel = solvers.pcg(lambda v: operators.apply_A(p, v), b, diag, p.lmax, tol=1e-13)
    assert rel <= 1e-13
    assert np.max(np.abs(xc - xd)) < 1e-8 * np.max(np.abs(xd))


def test_restrict_prolong_transpose_and_coarse_operator():
    """I_h^H and its transpose (Eq. f_l): <I r, c> = <r, I^T c>, and the
    Galerkin product I A_h I^T equals A_H with the coarser filter."""
    p = small_problem(nside=4, lmax=10)
    Lh, LH = 10, 6
    l = np.arange(Lh + 1)
    fh = np.exp(-0.002 * l * l * (l + 1) ** 2 * 1e-2)
    fH = fh * np.exp(-0.05 * l * (l + 1))
    rs = np.random.default_rng(4)
    r = rs.normal(size=sht.n_lm(Lh)) + 1j * rs.normal(size=sht.n_lm(Lh))
    c = rs.normal(size=sht.n_lm(LH)) + 1j * rs.normal(size=sht.n_lm(LH))
    lhs = sht.alm_dot(operators.restrict(fh, fH, Lh, LH, r), c, LH)
    rhs = sht.alm_dot(r, operators.prolong(fh, fH, Lh, LH, c), Lh)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    c[: LH + 1] = c[: LH + 1].real
    c[0:2] = 0.0
    gal = operators.restrict(fh, fH, Lh, LH, operators.apply_A_level(p, fh, Lh, operators.prolong(fh, fH, Lh, LH, c)))
    direct = operators.apply_A_level(p, fH, LH, c)
    np.testing.assert_allclose(gal, direct, rtol=1e-11, atol=1e-12 * np.max(np.abs(direct)))
