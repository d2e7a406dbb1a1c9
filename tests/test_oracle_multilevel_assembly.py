"""Pins for the parts of the oracle's multi-level solver that its fixed point
cannot see: the pixel smoother's assembled matrix (Section 3.5, Eqs. Dhat
and Bhat), the CR-Cycle's control structure (Fig. code:mg, Table
cycle-cost) and the smoother's lambda_max estimate.

- D_hat and B_hat are checked against columns of Y_h diag(f^2/C) Y_h^T and
  Y_obs diag(f b) Y_h^T probed with the direct transforms, inside a tile
  pattern built here from face coordinates and pixel-centre matching (no
  nested-index arithmetic shared with the oracle), and zero outside it.
- The cycle's visit counts, smoother applications and operator applications
  on non-zero vectors are checked against the numbers Table cycle-cost
  prints for the paper's Planck level table.
- The cycle from x = 0 is a symmetric linear map of b (pre- and
  post-smoothing with the same symmetric smoother), which fails when either
  smoothing step is dropped or altered.
"""
import math

import numpy as np
import pytest

from oracle import geometry, multilevel, operators, sht
from paper_1308_5299_gb300 import synthetic


def _match_pixels(vecs, grid):
    """RING index of the grid pixel whose centre coincides with each vector."""
    ref = geometry.pixel_vectors(grid)
    # nearest centre by dot product; the match must be exact to rounding
    idx = np.argmax(vecs @ ref.T, axis=1)
    assert np.max(np.linalg.norm(ref[idx] - vecs, axis=1)) < 1e-10
    return idx


def _tile_of_ring_pixels(nside, nside_t):
    """Tile (NESTED pixel of the Nside_t grid) of every RING pixel of the
    Nside grid: tile t = (face f, tx, ty) holds the pixels with face
    coordinates (tx r + i, ty r + j), r = nside / nside_t; their centres come
    from the continuous face coordinates and are matched to ring centres."""
    r = nside // nside_t
    g = geometry.healpix_grid(nside)
    out = -np.ones(g["npix"], dtype=np.int64)
    nt = 12 * nside_t * nside_t
    tx, ty, tf = multilevel.nest_to_xyf(nside_t, np.arange(nt))
    ii, jj = np.meshgrid(np.arange(r), np.arange(r), indexing="ij")
    for t in range(nt):
        x = tx[t] * r + ii.ravel() + 0.5
        y = ty[t] * r + jj.ravel() + 0.5
        v = multilevel.face_point(nside, np.full(x.shape, tf[t]), x, y)
        out[_match_pixels(v, g)] = t
    assert np.all(out >= 0)
    return out


@pytest.mark.slow
def test_pixel_level_assembly_equals_probed_transforms():
    """PixelLevel's D_hat, B_hat and A_hat at Nside_obs 16 / Nside_h 8 equal
    the probed transforms on the tile pattern and vanish off it."""
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside16_lmax47")
    gobs = geometry.healpix_grid(cfg["nside"])
    prob = operators.Problem(cfg["lmax"], cl, bl, ninv, gobs)
    table = multilevel.level_table(cfg["nside"], cfg["lmax"], first=8)
    lev = table["levels"][0]
    pl = multilevel.PixelLevel(prob, lev)
    nh, Lh, fl = lev["nside_h"], lev["lmax_h"], lev["fl"]
    gh = geometry.healpix_grid(nh)
    nt_side = nh // 8

    # tiles of level and observation pixels, built independently
    tile_h = _tile_of_ring_pixels(nh, nt_side)
    tile_o = _tile_of_ring_pixels(cfg["nside"], nt_side)
    assert np.all(np.bincount(tile_h) == 64)
    # the oracle's tile order: pixel a of the level vector is ring pixel perm[a]
    np.testing.assert_array_equal(pl.tile_of, tile_h[pl.perm])
    nb = multilevel.tile_neighbours(nt_side)
    ntile = len(nb)
    nbm = np.zeros((ntile, ntile), dtype=bool)
    for t in range(ntile):
        nbm[t, nb[t]] = True

    # probed full matrices (RING order): D = Y_h diag(f^2/C) Y_h^T,
    # B = Y_obs diag(f b) Y_h^T, one level pixel per column
    l, m = sht.lm_arrays(Lh)
    act = cl[l] > 0
    gD = np.where(act, fl[l] ** 2 / np.where(act, cl[l], 1.0), 0.0)
    gB = np.where(act, fl[l] * bl[l], 0.0)
    npx = gh["npix"]
    Dfull = np.zeros((npx, npx))
    Bfull = np.zeros((gobs["npix"], npx))
    for j in range(npx):
        e = np.zeros(npx)
        e[j] = 1.0
        a = sht.adjoint(e, Lh, gh)
        Dfull[:, j] = sht.synth(gD * a, Lh, gh)
        Bfull[:, j] = sht.synth(gB * a, Lh, gobs)

    perm = pl.perm
    dpat = nbm[np.ix_(tile_h[perm], tile_h[perm])]
    Dref = np.where(dpat, Dfull[np.ix_(perm, perm)], 0.0)
    scale = np.max(np.abs(Dref))
    np.testing.assert_allclose(pl.Dhat, Dref, rtol=0, atol=1e-11 * scale)
    assert np.all(pl.Dhat[~dpat] == 0.0)

    bpat = nbm[np.ix_(tile_o, tile_h[perm])]
    Bref = np.where(bpat, Bfull[:, perm], 0.0)
    np.testing.assert_allclose(pl.Bhat, Bref, rtol=0, atol=1e-11 * np.max(np.abs(Bref)))
    assert np.all(pl.Bhat[~bpat] == 0.0)

    # A_hat = D_hat + B_hat^T N^-1 B_hat on the pattern, zero off it
    Aref = np.where(dpat, Dref + Bref.T @ (ninv[:, None] * Bref), 0.0)
    np.testing.assert_allclose(pl.Ahat, Aref, rtol=0, atol=1e-11 * np.max(np.abs(Aref)))
    assert np.all(pl.Ahat[~dpat] == 0.0)


class _CountingHierarchy(multilevel.Hierarchy):
    """The oracle's CR-Cycle on stand-in operators (A_h = 1.1 I, smoothers
    0.3 I, an inexact bottom solve 0.7 I, so that no residual vanishes by
    accident) that record every call by level, with small band limits per
    level; the n_rec values come from the level table."""

    def __init__(self, table, lmax):
        self.table = table
        self.levels = table["levels"]
        H = len(self.levels)
        self._lm = [lmax - h for h in range(H + 2)]
        self.events = []

    def lmax_h(self, h):
        return self._lm[h]

    def apply_A(self, h, x):
        self.events.append(("A", h, bool(np.any(x != 0))))
        return 1.1 * x

    def smooth(self, h, r):
        self.events.append(("M", h, True))
        return 0.3 * r

    def restrict(self, h, r):
        self.events.append(("R", h, True))
        return _truncate(r, self._lm[h], self._lm[h + 1])

    def prolong(self, h, c):
        self.events.append(("P", h, True))
        return _pad(c, self._lm[h + 1], self._lm[h])

    def bottom_solve(self, b):
        self.events.append(("B", len(self.levels) + 1, True))
        return 0.7 * b


def _truncate(x, L, LH):
    l, m = sht.lm_arrays(L)
    return x[l <= LH].copy()


def _pad(c, LH, L):
    l, m = sht.lm_arrays(L)
    out = np.zeros(sht.n_lm(L), dtype=np.complex128)
    out[l <= LH] = c
    return out


def test_cycle_structure_matches_table_cycle_cost():
    """One CR-Cycle from the top with the Planck level table visits the
    levels 1, 1, 2, 4, 8, 16, 32 times and the dense bottom 32 times, smooths
    twice and restricts and prolongs once per visit (M_hat 2, 4, ..., 64 and
    Y_h 4 per visit), and applies A_h to non-zero vectors 3 times at the top
    and 2, 5, 10, 20, 40, 80 times on the pixel levels -- Table cycle-cost's
    Y_obs column of 6, 4, 10, 20, 40, 80, 160 transforms (two per A_h): a
    level's first visit starts from c = 0, so its pre-smoothing residual
    needs no operator application."""
    table = multilevel.level_table(2048, 3000)
    H = len(table["levels"])
    hier = _CountingHierarchy(table, lmax=12)
    x0 = np.ones(sht.n_lm(12), dtype=np.complex128)  # the top starts from a non-zero iterate
    b = np.arange(sht.n_lm(12)).astype(np.complex128)
    hier.cycle(0, x0, b)
    ev = hier.events
    visits = [sum(1 for e in ev if e[0] == "R" and e[1] == h) for h in range(H + 1)]
    assert visits == [1, 1, 2, 4, 8, 16, 32]                   # Table cycle-cost, "visits"
    assert sum(1 for e in ev if e[0] == "B") == 32              # lmax=40 (dense): 32 solves
    smooths = [sum(1 for e in ev if e[0] == "M" and e[1] == h) for h in range(H + 1)]
    assert smooths == [2, 2, 4, 8, 16, 32, 64]                  # M_hat column (2 x 11, 4 x 2.3, ...)
    prol = [sum(1 for e in ev if e[0] == "P" and e[1] == h) for h in range(H + 1)]
    assert prol == visits
    a_nonzero = [sum(1 for e in ev if e[0] == "A" and e[1] == h and e[2]) for h in range(H + 1)]
    assert [2 * a for a in a_nonzero] == [6, 4, 10, 20, 40, 80, 160]  # Y_obs column
    a_all = [sum(1 for e in ev if e[0] == "A" and e[1] == h) for h in range(H + 1)]
    assert a_all == [3 * v for v in visits]
    # order within the top visit: A, M, A, R, (recursion), P, A, M
    top = [e[0] for e in ev if e[1] == 0]
    assert top == ["A", "M", "A", "R", "P", "A", "M"]


@pytest.mark.slow
def test_cycle_from_zero_is_symmetric():
    """With x = 0 the CR-Cycle is a linear map b -> B b; pre- and
    post-smoothing with the same symmetric smoothers make B symmetric in the
    real inner product: <B u, v> = <u, B v> (Nside 16, one pixel level plus
    the dense bottom).  B is also positive definite on these vectors."""
    cfg, cl, bl, ninv = synthetic.problem_inputs("nside16_lmax47")
    g = geometry.healpix_grid(cfg["nside"])
    prob = operators.Problem(cfg["lmax"], cl, bl, ninv, g)
    H = multilevel.Hierarchy(prob, table=multilevel.level_table(cfg["nside"], cfg["lmax"], first=8))
    L = prob.lmax
    u = prob.clean(synthetic.random_alm(L, seed=3))
    v = prob.clean(synthetic.random_alm(L, seed=4))
    z = np.zeros_like(u)
    Bu = H.cycle(0, z, u)
    Bv = H.cycle(0, z, v)
    lhs = sht.alm_dot(Bu, v, L)
    rhs = sht.alm_dot(u, Bv, L)
    assert abs(lhs - rhs) < 1e-10 * math.sqrt(sht.alm_dot(Bu, Bu, L) * sht.alm_dot(v, v, L))
    assert sht.alm_dot(Bu, u, L) > 0 and sht.alm_dot(Bv, v, L) > 0


class _PowerStub(multilevel.Hierarchy):
    """smoother_lambda_max on explicit matrices: A_h and S_h act on the real
    parts of a band-limit-1 coefficient vector (three coefficients)."""

    def __init__(self, A, S):
        self.A, self.S = A, S

    def lmax_h(self, h):
        return 1

    def apply_A(self, h, x):
        return self.A @ x.real + 0j

    def smooth(self, h, r):
        return self.S @ r.real + 0j


def test_smoother_lambda_max_power_iteration():
    """The Rayleigh-quotient power iteration returns the largest eigenvalue
    of S A for symmetric positive definite S and A (at an eigenvector the
    quotient is the eigenvalue in any inner product)."""
    rs = np.random.default_rng(8)
    X = rs.normal(size=(3, 3))
    A = X @ X.T + 3 * np.eye(3)
    Y = rs.normal(size=(3, 3))
    S = Y @ Y.T + 0.5 * np.eye(3)
    lam = _PowerStub(A, S).smoother_lambda_max(1, iters=60)
    ref = np.max(np.linalg.eigvals(S @ A).real)
    assert abs(lam - ref) < 1e-8 * ref
