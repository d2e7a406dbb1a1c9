"""Pins for the oracle's multi-level machinery (Sections 3.2-3.5): HEALPix
nested indexing and tiles, the addition theorem against explicit transforms,
ICC(0) against its defining properties, and the cycle's fixed point against
the dense solve."""

import numpy as np
import scipy.linalg
import pytest

from oracle import geometry, multilevel, operators, sht, solvers
from paper_1308_5299_gb300 import synthetic


@pytest.mark.parametrize("nside", [1, 2, 4, 16])
def test_nest2ring_is_bijection_with_matching_centres(nside):
    """NESTED -> RING maps every pixel once, and the nested pixel centre from
    the continuous face coordinates equals the RING-scheme centre."""
    n = 12 * nside * nside
    r = multilevel.nest2ring(nside, np.arange(n))
    assert sorted(r.tolist()) == list(range(n))
    ix, iy, f = multilevel.nest_to_xyf(nside, np.arange(n))
    v = multilevel.face_point(nside, f, ix + 0.5, iy + 0.5)
    vr = geometry.pixel_vectors(geometry.healpix_grid(nside))[r]
    assert np.max(np.abs(v - vr)) < 1e-12


def test_nest2ring_nside1_identity():
    assert multilevel.nest2ring(1, np.arange(12)).tolist() == list(range(12))


@pytest.mark.parametrize("nside_t", [2, 4, 8])
def test_tile_neighbourhoods(nside_t):
    """Vertex-sharing neighbourhoods: symmetric, 8 neighbours everywhere
    except around the 8 vertices where only three base faces meet, where
    each of the 3 tiles touching the vertex has 7 (24 tiles)."""
    nb = multilevel.tile_neighbours(nside_t)
    counts = np.array([len(x) - 1 for x in nb])
    for t, lst in enumerate(nb):
        assert t in lst
        for u in lst:
            assert t in nb[u]
    assert np.sum(counts == 7) == 24
    assert np.all((counts == 8) | (counts == 7))
    col = multilevel.greedy_colours(nb)
    for t, lst in enumerate(nb):
        for u in lst:
            if u != t:
                assert col[u] != col[t]


def test_addition_theorem_equals_transforms():
    """g(theta) of Eq. addition-theorem equals Y diag(g_l) Y^T between pixel
    pairs computed with the direct transforms (Eq. Dhat)."""
    nside, L = 4, 12
    g = geometry.healpix_grid(nside)
    gl = np.exp(-0.02 * np.arange(L + 1)) * (1 + np.arange(L + 1))
    l, m = sht.lm_arrays(L)
    for j in [0, 17, 100]:
        e = np.zeros(g["npix"])
        e[j] = 1.0
        col = sht.synth(gl[l] * sht.adjoint(e, L, g), L, g)
        v = geometry.pixel_vectors(g)
        ref = multilevel.coupling(gl, v @ v[j])
        np.testing.assert_allclose(col, ref, atol=1e-13 * np.max(np.abs(ref)))


def test_icc0_properties():
    """ICC(0) with a full pattern is the Cholesky factor; with a sparse
    pattern L L^T reproduces A on the pattern and L vanishes off it."""
    rs = np.random.default_rng(0)
    n = 40
    X = rs.normal(size=(n, n))
    A = X @ X.T + n * np.eye(n)
    full = np.ones((n, n), dtype=bool)
    np.testing.assert_allclose(multilevel.icc0(A, full), np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)
    pat = np.abs(np.subtract.outer(np.arange(n), np.arange(n))) <= 3
    pat |= (np.add.outer(np.arange(n), np.arange(n)) % 7 == 0)
    Lf = multilevel.icc0(A, pat)
    assert Lf is not None
    assert np.all(Lf[~pat] == 0.0)
    LL = Lf @ Lf.T
    np.testing.assert_allclose(LL[pat], A[pat], rtol=1e-12, atol=1e-10)


def test_block_icc_equals_elementwise():
    """The tile-block elimination is the element-wise ICC(0) on the same
    block pattern."""
    rs = np.random.default_rng(2)
    bs, nt = 5, 7
    nb = np.eye(nt, dtype=bool)
    for i, j in [(0, 1), (1, 2), (2, 5), (3, 4), (4, 6), (0, 6), (5, 6)]:
        nb[i, j] = nb[j, i] = True
    pat = np.kron(nb, np.ones((bs, bs), dtype=bool))
    X = rs.normal(size=(nt * bs, nt * bs))
    A = np.where(pat, X @ X.T, 0.0) + 8.0 * np.eye(nt * bs)
    e = multilevel.icc0(A, pat)
    b = multilevel.icc0_blocks(A, bs, nb)
    assert e is not None and b is not None
    np.testing.assert_allclose(b, e, rtol=1e-11, atol=1e-12)


def test_block_jacobi_is_exact_for_block_diagonal_and_a_preconditioner():
    """The additive Schwarz (block Jacobi) smoother: for a block-diagonal SPD
    matrix it is the exact inverse; for a coupled SPD matrix it is SPD and
    solves the tile blocks exactly (the residual of its result vanishes on
    each block's own rows of A_pp x = r_p)."""
    rs = np.random.default_rng(5)
    bs, nt = 6, 5
    n = bs * nt
    blocks = []
    for _ in range(nt):
        X = rs.normal(size=(bs, bs))
        blocks.append(X @ X.T + bs * np.eye(bs))
    A = scipy.linalg.block_diag(*blocks)
    r = rs.normal(size=n)
    np.testing.assert_allclose(multilevel.block_jacobi_apply(A, bs, 0.0, r), np.linalg.solve(A, r), rtol=1e-12)
    # with coupling: M = blockdiag(A)^-1 is symmetric positive definite
    Y = rs.normal(size=(n, n))
    A2 = A + 0.1 * (Y @ Y.T)
    M = np.column_stack([multilevel.block_jacobi_apply(A2, bs, 0.3, e) for e in np.eye(n)])
    np.testing.assert_allclose(M, M.T, atol=1e-12)
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0
    z = multilevel.block_jacobi_apply(A2, bs, 0.3, r)
    for p0 in range(0, n, bs):
        sl = slice(p0, p0 + bs)
        np.testing.assert_allclose((A2[sl, sl] + 0.3 * np.eye(bs)) @ z[sl], r[sl], rtol=1e-10, atol=1e-12)


def test_ridge_search_bracket():
    """The search returns 1.5 x the smallest working ridge: ICC(0) fails just
    below the found alpha and succeeds at it."""
    rs = np.random.default_rng(1)
    n = 30
    X = rs.normal(size=(n, n))
    A = X @ X.T - 5.0 * np.eye(n)  # indefinite
    pat = np.abs(np.subtract.outer(np.arange(n), np.arange(n))) <= 4
    used, Lf = multilevel.ridge_search(A, pat, factor=1.5)
    alpha = used / 1.5
    amax = np.max(np.abs(A))
    assert multilevel.icc0(A + alpha * np.eye(n), pat) is not None
    assert multilevel.icc0(A + alpha * 0.95 * np.eye(n), pat) is None
    assert Lf is not None


def test_filters_match_paper_constraints():
    """q_2570 = 0.1 (Nside_h 1024) and q_1536 = 0.1 (Nside_h 512), Eq.
    fourth-power-beam; the Planck level table of Table cycle-cost."""
    t = multilevel.level_table(2048, 3000)
    lv = t["levels"]
    assert [x["nside_h"] for x in lv] == [1024, 512, 256, 128, 64, 32]
    assert [x["lmax_h"] for x in lv][:2] == [3000, 2048]
    assert abs(lv[0]["fl"][2570] - 0.1) < 1e-12
    assert abs(lv[1]["fl"][1536] / lv[0]["fl"][1536] - 0.1) < 1e-12
    assert t["bottom"]["lmax_h"] == 40
    assert [x["n_rec"] for x in lv] == [2, 2, 2, 2, 2, 1]
    for a, b in zip(lv[:-1], lv[1:]):
        assert np.all(b["fl"] <= a["fl"] + 1e-15)


@pytest.mark.slow
def test_multilevel_fixed_point_equals_dense_solve():
    """CR-Solve converges to x* = A^-1 b of the dense oracle (Nside 16: one
    pixel level at Nside_h 8 plus the dense bottom)."""
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside16_lmax47")
    g = geometry.healpix_grid(cfg["nside"])
    prob = operators.Problem(cfg["lmax"], cl, bl, ninv, g)
    x_true = synthetic.draw_prior(cl, index=1)
    b = operators.apply_A(prob, x_true)
    H = multilevel.Hierarchy(prob, table=multilevel.level_table(cfg["nside"], cfg["lmax"], first=8))
    assert len(H.pix) == 1
    x, hist = H.solve(b, eps=1e-20, max_cycles=45, x_true=prob.clean(x_true))
    errs = [h[1] for h in hist]
    assert all(b2 < b1 for b1, b2 in zip(errs[:-1], errs[1:]))
    assert errs[-1] < 1e-8 * errs[0]
    assert np.max(np.abs(x - prob.clean(x_true))) < 1e-7 * np.max(np.abs(x_true))


def test_first_level_rule_matches_planck_table():
    """The default first pixel level reproduces the paper's Planck choice
    (lmax 3000 -> Nside_h 1024, Section 3.2) and scales with lmax elsewhere."""
    assert multilevel.first_level_nside(2048, 3000) == 1024
    assert multilevel.first_level_nside(32, 95) == 32
    assert multilevel.first_level_nside(256, 767) == 256
    assert multilevel.first_level_nside(1024, 2047) == 512
    assert multilevel.first_level_nside(8, 23) == 8
    t = multilevel.level_table(256, 767)
    assert [lv["nside_h"] for lv in t["levels"]] == [256, 128, 64, 32, 16, 8]
