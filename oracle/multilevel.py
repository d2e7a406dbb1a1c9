"""The multi-level CR solver of Sections 3.2-3.5 and Fig. code:mg, written
out step by step in FP64 for small grids (observation Nside <= 32).

Oracle module -- test infrastructure only.  It exists to check the GPU's
level operators, restriction, smoothers and cycle row by row; the answer of
the solve itself is defined by ``solvers`` (x* = A^-1 b).

Level structure (Section 3.2; readings for configurations other than the
paper's Planck setup are listed in the design notes):
  level 0      spherical-harmonic top level at lmax, filter 1, diagonal error
               smoother diag(A)^-1 applied through the high-pass 1 - f^1;
  levels 1..H  spherical-harmonic levels (lmax_h, cumulative filter f^h) each
               with a sibling HEALPix pixel grid Nside_h and a block-sparse
               incomplete-Cholesky error smoother M_h ~ (Y_h A_h Y_h^T)^-1;
  bottom       A_H restricted to l <= l_dense, solved by dense Cholesky.
Restriction I_h^H = diag(f^H / f^h) truncated at lmax_H (Eq. f_l);
interpolation is its transpose.

Pixel smoother (Section 3.5): tiles are the pixels of the HEALPix grid at
Nside_h / k, each holding its k^2 NESTED children; a tile couples to itself
and to the tiles it shares a vertex with.  D_hat (Eq. Dhat) and B_hat
(Eq. Bhat) are evaluated inside that pattern with the addition theorem
(Eq. addition-theorem), B_hat^T N^-1 B_hat is formed without fill-in, D_hat
is added, and an ICC(0) factorisation is taken in a multicolour tile order
(greedy colouring in nested tile order; colour-major, then tile index), with
the binary ridge search of Section 3.5 (smallest alpha that lets the
factorisation succeed, used times 1.5).
"""
import math

import numpy as np
import scipy.linalg

from . import geometry, operators, sht

# ---------------------------------------------------------------------------
# level table and filters (Section 3.3, Eq. fourth-power-beam; Section 3.4)


def q_filter(lmax, ell_star, value=0.1):
    """q_l = exp(-l^2 (l+1)^2 lambda) with lambda fixed by q_{ell*} = value."""
    l = np.arange(lmax + 1, dtype=np.float64)
    lam = -math.log(value) / (ell_star ** 2 * (ell_star + 1.0) ** 2)
    return np.exp(-(l * l) * (l + 1.0) ** 2 * lam)


def gauss_filter(lmax, nside_h):
    """Gaussian with FWHM of 2 pixel widths of the Nside_h grid."""
    fwhm = 2.0 * math.sqrt(4.0 * math.pi / (12.0 * nside_h * nside_h))
    s = fwhm / math.sqrt(8.0 * math.log(2.0))
    l = np.arange(lmax + 1, dtype=np.float64)
    return np.exp(-0.5 * l * (l + 1.0) * s * s)


def first_level_nside(nside, lmax, k=8):
    """Nside of the first pixel level outside the paper's Planck table: the
    power of two nearest lmax / 2.93 (the table's 3000 / 1024), so that the
    top level's high-pass 1 - f^1 covers the same share of the band, clipped
    to [k, nside]."""
    e = math.log2(max(1.0, lmax / 2.93))
    nh = 1 << max(0, int(math.floor(e + 0.5)))
    return max(min(nh, nside), k)


def level_table(nside, lmax, k=8, planck=None, first=None):
    """Levels for an observation grid of Nside ``nside`` and band limit
    ``lmax``.  Returns dict(top, levels[list], bottom).  Each pixel level:
    nside_h, lmax_h, fl (cumulative filter, length lmax+1, zero above
    lmax_h), n_rec (recursions into the next level)."""
    if planck is None:
        planck = (nside == 2048 and lmax == 3000)
    levels = []
    if planck:
        spec = [(1024, 3000), (512, 2048), (256, 1280), (128, 768), (64, 384), (32, 224)]
    else:
        spec = []
        nh = first_level_nside(nside, lmax, k) if first is None else first
        while nh >= k:
            if not spec:
                lh = lmax
            elif len(spec) == 1:
                lh = min(lmax, 4 * nh)
            else:
                lh = min(spec[-1][1], 6 * nh)
            spec.append((nh, lh))
            nh //= 2
    prev = np.ones(lmax + 1)
    for i, (nh, lh) in enumerate(spec):
        if i == 0:
            f = q_filter(lmax, 2.51 * nh if not planck else 2570.0)
        elif i == 1:
            f = prev * q_filter(lmax, 3.0 * nh if not planck else 1536.0)
        else:
            f = np.minimum(gauss_filter(lmax, nh), prev)
        f = f.copy()
        f[lh + 1:] = 0.0
        f[f < 1e-8] = 0.0
        # band limit: last l with a nonzero filter
        nz = np.nonzero(f > 0)[0]
        lh = int(min(lh, nz[-1])) if len(nz) else 0
        f[lh + 1:] = 0.0
        levels.append(dict(nside_h=nh, lmax_h=lh, fl=f, n_rec=2))
        prev = f
    if levels:
        levels[-1]["n_rec"] = 1
        ld = min(40, levels[-1]["lmax_h"] // 2)
        fb = levels[-1]["fl"].copy()
    else:
        ld = min(40, lmax)
        fb = np.ones(lmax + 1)
    fb[ld + 1:] = 0.0
    top = dict(lmax_h=lmax, fl=np.ones(lmax + 1), n_rec=1)
    bottom = dict(lmax_h=ld, fl=fb)
    return dict(top=top, levels=levels, bottom=bottom, k=k)


# ---------------------------------------------------------------------------
# HEALPix nested scheme and tiles (Gorski et al. 2005)

JRLL = np.array([2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4])
JPLL = np.array([1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7])


def _compress_bits(v):
    """Keep the even-position bits of v, packed."""
    out = np.zeros_like(v)
    for b in range(31):
        out |= ((v >> (2 * b)) & 1) << b
    return out


def nest_to_xyf(nside, ipix):
    ipix = np.asarray(ipix, dtype=np.int64)
    f = ipix // (nside * nside)
    w = ipix % (nside * nside)
    return _compress_bits(w), _compress_bits(w >> 1), f


def nest2ring(nside, ipix):
    """RING index of NESTED pixels: face (f, ix, iy) -> ring jr = jrll N -
    ix - iy - 1 (1-based) and position j = (nr jpll + ix - iy - s) / 2 mod
    4 nr, nr the ring's quarter length, s its half-pixel shift."""
    N = nside
    ix, iy, f = nest_to_xyf(N, ipix)
    jr = JRLL[f] * N - ix - iy - 1
    nr = np.where(jr < N, jr, np.where(jr > 3 * N, 4 * N - jr, N))
    s = np.where((jr < N) | (jr > 3 * N), 1, (jr - N + 1) % 2)
    j = (nr * JPLL[f] + ix - iy - s) // 2
    j = np.mod(j, 4 * nr)
    start = np.where(jr < N, 2 * jr * (jr - 1),
                     np.where(jr > 3 * N, 12 * N * N - 2 * nr * (nr + 1), 2 * N * (N - 1) + (jr - N) * 4 * N))
    return start + j


def face_point(nside, f, x, y):
    """Unit vector of continuous face coordinates (x, y) in [0, N]^2 of face f."""
    N = float(nside)
    jr = JRLL[f] * N - x - y
    with np.errstate(divide="ignore", invalid="ignore"):
        z = np.where(jr < N, 1.0 - jr * jr / (3 * N * N),
                     np.where(jr > 3 * N, -(1.0 - (4 * N - jr) ** 2 / (3 * N * N)), 4.0 / 3.0 - 2.0 * jr / (3 * N)))
        nr = np.where(jr < N, jr, np.where(jr > 3 * N, 4 * N - jr, N))
        phi = np.where(nr > 0, 0.25 * np.pi * (JPLL[f] + (x - y) / np.where(nr > 0, nr, 1.0)), 0.0)
    st = np.sqrt(np.maximum(0.0, (1.0 - z) * (1.0 + z)))
    return np.stack([st * np.cos(phi), st * np.sin(phi), z], axis=-1)


def vertex_keys(nside, f, x, y):
    """Exact integer identity of lattice points (x, y) of face f: the ring
    coordinate jr = jrll N - x - y and the azimuth numerator
    (jpll nr + x - y) mod 8 nr (nr the ring's quarter length; 0 at the
    poles), the same for every face that contains the point."""
    N = nside
    jr = JRLL[f] * N - x - y
    nr = np.where(jr < N, jr, np.where(jr > 3 * N, 4 * N - jr, N))
    num = np.where(nr > 0, np.mod(JPLL[f] * nr + x - y, np.maximum(8 * nr, 1)), 0)
    return jr, num


def tile_neighbours(nside_t):
    """Neighbour lists of the tiles (pixels of the Nside_t grid, NESTED
    index): tiles sharing at least one vertex."""
    nt = 12 * nside_t * nside_t
    ix, iy, f = nest_to_xyf(nside_t, np.arange(nt))
    keys = {}
    for dx, dy in [(0, 0), (1, 0), (0, 1), (1, 1)]:
        jr, num = vertex_keys(nside_t, f, ix + dx, iy + dy)
        for t in range(nt):
            keys.setdefault((int(jr[t]), int(num[t])), set()).add(t)
    nb = [set() for _ in range(nt)]
    for s in keys.values():
        for t in s:
            nb[t] |= s
    return [sorted(x) for x in nb]  # includes the tile itself


def greedy_colours(nb):
    col = -np.ones(len(nb), dtype=np.int64)
    for t in range(len(nb)):
        used = {col[u] for u in nb[t] if col[u] >= 0}
        c = 0
        while c in used:
            c += 1
        col[t] = c
    return col


def tile_order(nb):
    col = greedy_colours(nb)
    order = np.lexsort((np.arange(len(nb)), col))  # colour-major, then index
    return order, col


# ---------------------------------------------------------------------------
# addition theorem (Eq. addition-theorem)


def coupling(gl, cos_theta, lmin=0):
    """g(theta) = sum_l (2l+1)/(4 pi) g_l P_l(cos theta) by the Legendre
    recurrence, for an array of cos(theta)."""
    x = np.asarray(cos_theta, dtype=np.float64)
    L = len(gl) - 1
    p0 = np.ones_like(x)
    out = np.zeros_like(x)
    if lmin <= 0:
        out += gl[0] / (4 * math.pi) * p0
    if L >= 1:
        p1 = x.copy()
        if lmin <= 1:
            out += 3.0 * gl[1] / (4 * math.pi) * p1
        for l in range(2, L + 1):
            p2 = ((2 * l - 1) * x * p1 - (l - 1) * p0) / l
            p0, p1 = p1, p2
            if l >= lmin and gl[l] != 0.0:
                out += (2 * l + 1) * gl[l] / (4 * math.pi) * p1
    return out


# ---------------------------------------------------------------------------
# incomplete Cholesky


def icc0(A, pattern):
    """Zero-fill-in incomplete Cholesky: ordinary in-place Cholesky, but
    every update outside ``pattern`` (boolean, symmetric) is dropped.
    Returns the lower factor, or None if a pivot is not positive."""
    n = A.shape[0]
    Lf = np.where(pattern, A, 0.0)
    Lf = np.tril(Lf)
    for j in range(n):
        d = Lf[j, j] - Lf[j, :j] @ Lf[j, :j]
        if not (d > 0.0) or not np.isfinite(d):
            return None
        Lf[j, j] = math.sqrt(d)
        col = (Lf[j + 1:, j] - Lf[j + 1:, :j] @ Lf[j, :j]) / Lf[j, j]
        Lf[j + 1:, j] = np.where(pattern[j + 1:, j], col, 0.0)
    return Lf


def block_jacobi_apply(A, bs, alpha, r):
    """Additive Schwarz smoother without overlap (block Jacobi): the tiles
    (consecutive groups of bs rows, elimination order) are the subdomains,
    each solved exactly, r -> sum_p R_p^T (A_pp + alpha I)^-1 R_p r, with
    A_pp the tile's diagonal block.  The domain-decomposition alternative to
    the multicolour ICC(0) that Section 3.5 names for a fully parallel apply;
    the ridge alpha plays the same role as in the ICC factorisation."""
    n = A.shape[0]
    out = np.zeros(n)
    for p0 in range(0, n, bs):
        sl = slice(p0, p0 + bs)
        Ap = A[sl, sl] + alpha * np.eye(min(bs, n - p0))
        out[sl] = scipy.linalg.cho_solve(scipy.linalg.cho_factor(Ap, lower=True), r[sl])
    return out


def icc0_blocks(A, bs, nbmat):
    """The same zero-fill-in incomplete Cholesky as ``icc0`` for a pattern
    made of dense bs x bs tile blocks (nbmat[i, j]: tiles i and j coupled,
    tiles in elimination order).  Block form of the same elimination:
    L_jj = chol(A_jj - sum_k L_jk L_jk^T), L_ij = (A_ij - sum_k L_ik L_jk^T)
    L_jj^-T over earlier tiles k coupled to both.  Returns None on a
    non-positive pivot."""
    nt = nbmat.shape[0]
    Lb = {}
    for j in range(nt):
        S = A[j * bs:(j + 1) * bs, j * bs:(j + 1) * bs].copy()
        for k in range(j):
            if nbmat[j, k]:
                S -= Lb[(j, k)] @ Lb[(j, k)].T
        try:
            Ljj = np.linalg.cholesky(S)
        except np.linalg.LinAlgError:
            return None
        if not np.all(np.isfinite(Ljj)):
            return None
        Lb[(j, j)] = Ljj
        for i in range(j + 1, nt):
            if not nbmat[i, j]:
                continue
            S = A[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs].copy()
            for k in range(j):
                if nbmat[i, k] and nbmat[j, k]:
                    S -= Lb[(i, k)] @ Lb[(j, k)].T
            Lb[(i, j)] = scipy.linalg.solve_triangular(Ljj, S.T, lower=True).T
    Lf = np.zeros_like(A)
    for (i, j), blk in Lb.items():
        Lf[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = blk
    return Lf


def ridge_search(A, pattern, factor=1.5, bisections=30, icc=None):
    """Smallest ridge alpha (in units of max|A|, searched in log space on
    [1e-12, 1]) that lets ICC(0) succeed; returns (alpha_used, L) with the
    final factorisation taken at factor * alpha (Section 3.5)."""
    f = icc or (lambda M: icc0(M, pattern))
    amax = float(np.max(np.abs(A)))
    eye = np.eye(A.shape[0])
    if f(A) is not None:
        alpha = 0.0
    else:
        lo, hi = math.log(1e-12), 0.0
        if f(A + amax * eye) is None:
            raise RuntimeError("ICC fails even with alpha = max|A|")
        for _ in range(bisections):
            mid = 0.5 * (lo + hi)
            if f(A + amax * math.exp(mid) * eye) is None:
                lo = mid
            else:
                hi = mid
        alpha = amax * math.exp(hi)
    Lf = f(A + factor * alpha * eye)
    return factor * alpha, Lf


# ---------------------------------------------------------------------------
# the hierarchy


class PixelLevel:
    """Pixel grid, tile pattern, explicit A_hat in the pattern and its ICC
    factor for one level."""

    def __init__(self, prob, lev, k=8, ridge_factor=1.5, alpha=None):
        nh, lh, fl = lev["nside_h"], lev["lmax_h"], lev["fl"]
        self.nside_h, self.lmax_h, self.fl = nh, lh, fl
        self.grid = geometry.healpix_grid(nh)
        nt_side = nh // k
        self.nb = tile_neighbours(nt_side)
        self.order, self.colour = tile_order(self.nb)
        ntile = len(self.nb)
        kk = k * k
        # level pixels in tile order: tile t (in colour order) holds NESTED
        # pixels t*k^2 .. t*k^2+k^2-1 of the Nside_h grid
        nest = (self.order[:, None] * kk + np.arange(kk)[None, :]).ravel()
        self.perm = nest2ring(nh, nest)  # ring index of each tile-ordered pixel
        self.tile_of = np.repeat(self.order, kk)  # nested tile index of each tile-ordered pixel
        pos = np.empty(ntile, dtype=np.int64)
        pos[self.order] = np.arange(ntile)
        nbmat = np.zeros((ntile, ntile), dtype=bool)
        for t in range(ntile):
            nbmat[t, self.nb[t]] = True
        self.pattern = nbmat[np.ix_(self.tile_of, self.tile_of)]
        # pixel vectors in tile order
        vh = geometry.pixel_vectors(self.grid)[self.perm]
        cl = prob.cl[: lh + 1]
        act = cl > 0
        gD = np.where(act, fl[: lh + 1] ** 2 / np.where(act, cl, 1.0), 0.0)
        gB = np.where(act, fl[: lh + 1] * prob.bl[: lh + 1], 0.0)
        cosv = np.clip(vh @ vh.T, -1.0, 1.0)
        D = np.zeros_like(cosv)
        D[self.pattern] = coupling(gD, cosv[self.pattern])
        # B_hat on the observation grid: obs pixel o couples to level pixel j
        # when the tile containing o neighbours the tile of j
        obs = prob.grid
        nobs = obs["npix"]
        ratio = obs["nside"] // nt_side
        ring_of_nest = nest2ring(obs["nside"], np.arange(nobs))
        obs_tile = np.empty(nobs, dtype=np.int64)
        obs_tile[ring_of_nest] = np.arange(nobs) // (ratio * ratio)
        vo = geometry.pixel_vectors(obs)
        Bm = np.zeros((nobs, len(self.perm)))
        bpat = nbmat[np.ix_(obs_tile, self.tile_of)]
        cob = np.clip(vo @ vh.T, -1.0, 1.0)
        Bm[bpat] = coupling(gB, cob[bpat])
        BNB = Bm.T @ (prob.ninv[:, None] * Bm)
        self.Ahat = np.where(self.pattern, D + BNB, 0.0)
        self.Ahat = 0.5 * (self.Ahat + self.Ahat.T)
        self.nbmat_ord = nbmat[np.ix_(self.order, self.order)]
        icc = lambda M: icc0_blocks(M, kk, self.nbmat_ord)
        if alpha is None:
            self.alpha, self.L = ridge_search(self.Ahat, self.pattern, ridge_factor, icc=icc)
        else:
            self.alpha = alpha
            self.L = icc(self.Ahat + alpha * np.eye(len(self.perm)))
        self.Dhat, self.Bhat = D, Bm

    def apply_M(self, r_pix):
        """M_hat r for a RING-ordered level map r: (L L^T)^-1 in tile order."""
        rt = r_pix[self.perm]
        y = scipy.linalg.solve_triangular(self.L, rt, lower=True)
        c = scipy.linalg.solve_triangular(self.L.T, y, lower=False)
        out = np.zeros(self.grid["npix"])
        out[self.perm] = c
        return out

    def apply_M_schwarz(self, r_pix, alpha):
        """Block-Jacobi (additive Schwarz) smoother of the same A_hat for a
        RING-ordered level map, ridge alpha on every tile block."""
        out = np.zeros(self.grid["npix"])
        out[self.perm] = block_jacobi_apply(self.Ahat, 64, alpha, r_pix[self.perm])
        return out

    def smooth_schwarz(self, r, alpha, prob):
        """Y_h^T M Y_h r with the block-Jacobi M (level's active mask)."""
        Lh = self.lmax_h
        c = sht.adjoint(self.apply_M_schwarz(sht.synth(r, Lh, self.grid), alpha), Lh, self.grid)
        l, m = sht.lm_arrays(Lh)
        c[prob.cl[l] <= 0] = 0.0
        c[m == 0] = c[m == 0].real
        return c


class Hierarchy:
    def __init__(self, prob, table=None, k=8, ridge_factor=1.5, alphas=None, lambda_target=None):
        """lambda_target: if given (and alphas is None), each level's ridge is
        raised after the search until the power-iteration estimate of
        lambda_max(S_h A_h) is at most this value."""
        self.prob = prob
        self.table = table or level_table(prob.grid["nside"], prob.lmax, k=k)
        self.levels = self.table["levels"]
        self.pix = [PixelLevel(prob, lev, k, ridge_factor, None if alphas is None else alphas[i])
                    for i, lev in enumerate(self.levels)]
        L = prob.lmax
        # top-level diagonal smoother: H (diag A)^-1 with H = 1 - f^1
        dm0 = operators.diag_inv_noise_dm0(prob)
        l = prob.l
        with np.errstate(divide="ignore"):
            sinv = np.where(prob.active, 1.0 / np.where(prob.active, prob.cl[l], 1.0), 0.0)
        self.diagA = sinv + prob.bl[l] ** 2 * dm0
        f1 = self.levels[0]["fl"] if self.levels else np.zeros(L + 1)
        self.highpass = 1.0 - f1[l]
        # bottom dense block
        bt = self.table["bottom"]
        self.ld, self.fb = bt["lmax_h"], bt["fl"]
        act_d = operators.real_active_mask(prob, self.ld)
        Ad = operators.dense_matrix(lambda v: operators.apply_A_level(prob, self.fb, self.ld, v), self.ld, act_d)
        self.act_d = act_d
        self.Abottom = 0.5 * (Ad + Ad.T)
        self.chol_bottom = scipy.linalg.cho_factor(self.Abottom, lower=True)
        self.lambda_max = [None] * len(self.pix)
        if lambda_target is not None and alphas is None:
            for h in range(1, len(self.pix) + 1):
                pl = self.pix[h - 1]
                for _ in range(24):
                    lam = self.smoother_lambda_max(h)
                    self.lambda_max[h - 1] = lam
                    if lam <= lambda_target:
                        break
                    a = pl.alpha if pl.alpha > 0 else 1e-6 * np.max(np.abs(pl.Ahat))
                    a *= max(2.0, lam / lambda_target)
                    pl.alpha = a
                    pl.L = icc0_blocks(pl.Ahat + a * np.eye(len(pl.perm)), 64, pl.nbmat_ord)

    def smoother_lambda_max(self, h, iters=12, seed=0):
        """Rayleigh-quotient power iteration for lambda_max(S_h A_h) in the
        A_h inner product."""
        L = self.lmax_h(h)
        rs = np.random.default_rng(seed)
        v = rs.uniform(-1, 1, size=sht.n_lm(L)) + 1j * rs.uniform(-1, 1, size=sht.n_lm(L))
        lam = 0.0
        for _ in range(iters):
            av = self.apply_A(h, v)
            w = self.smooth(h, av)
            lam = sht.alm_dot(w, av, L) / sht.alm_dot(v, av, L)
            v = w / np.sqrt(sht.alm_dot(w, w, L))
        return lam

    # level h: 0 = top, 1..H = pixel levels, H+1 = bottom
    def fl(self, h):
        if h == 0:
            return self.table["top"]["fl"]
        if h <= len(self.levels):
            return self.levels[h - 1]["fl"]
        return self.fb

    def lmax_h(self, h):
        if h == 0:
            return self.prob.lmax
        if h <= len(self.levels):
            return self.levels[h - 1]["lmax_h"]
        return self.ld

    def apply_A(self, h, x):
        if h == 0:
            return operators.apply_A(self.prob, x)
        return operators.apply_A_level(self.prob, self.fl(h), self.lmax_h(h), x)

    def restrict(self, h, r):
        return operators.restrict(self.fl(h), self.fl(h + 1), self.lmax_h(h), self.lmax_h(h + 1), r)

    def prolong(self, h, c):
        return operators.prolong(self.fl(h), self.fl(h + 1), self.lmax_h(h), self.lmax_h(h + 1), c)

    def smooth(self, h, r):
        """Correction of one error-smoothing step on level h for residual r."""
        if h == 0:
            return np.where(self.diagA != 0, self.highpass * r / np.where(self.diagA != 0, self.diagA, 1.0), 0.0)
        pl = self.pix[h - 1]
        Lh = pl.lmax_h
        rp = sht.synth(r, Lh, pl.grid)
        cp = pl.apply_M(rp)
        c = sht.adjoint(cp, Lh, pl.grid)
        l, m = sht.lm_arrays(Lh)
        c[self.prob.cl[l] <= 0] = 0.0
        c[m == 0] = c[m == 0].real
        return c

    def bottom_solve(self, b):
        u = sht.alm_to_real(b, self.ld)[self.act_d]
        x = np.zeros((self.ld + 1) ** 2)
        x[self.act_d] = scipy.linalg.cho_solve(self.chol_bottom, u)
        return sht.real_to_alm(x, self.ld)

    def n_rec(self, h):
        if h == 0:
            return self.table["top"]["n_rec"]
        return self.levels[h - 1]["n_rec"]

    def cycle(self, h, x, b):
        """CR-Cycle of Fig. code:mg (the top level uses the diagonal smoother)."""
        H = len(self.levels)
        if h == H + 1:
            return self.bottom_solve(b)
        x = x + self.smooth(h, b - self.apply_A(h, x))
        rH = self.restrict(h, b - self.apply_A(h, x))
        c = np.zeros(sht.n_lm(self.lmax_h(h + 1)), dtype=np.complex128)
        for _ in range(self.n_rec(h)):
            c = self.cycle(h + 1, c, rH)
        x = x + self.prolong(h, c)
        x = x + self.smooth(h, b - self.apply_A(h, x))
        return x

    def solve(self, b, eps=1e-12, max_cycles=50, x_true=None):
        """CR-Solve: repeat cycles until r^T S^-1 r < eps b^T S^-1 b.
        Returns (x, history of (relres, err))."""
        prob = self.prob
        l = prob.l
        with np.errstate(divide="ignore"):
            sinv = np.where(prob.active, 1.0 / np.where(prob.active, prob.cl[l], 1.0), 0.0)
        bsb = sht.alm_dot(b, sinv * b, prob.lmax)
        x = np.zeros_like(b)
        hist = []
        for _ in range(max_cycles):
            x = self.cycle(0, x, b)
            r = b - operators.apply_A(prob, x)
            rel = sht.alm_dot(r, sinv * r, prob.lmax) / bsb
            err = None
            if x_true is not None:
                e = x - x_true
                err = float(np.sqrt(sht.alm_dot(e, sinv * e, prob.lmax)))
            hist.append((math.sqrt(rel), err))
            if rel < eps:
                break
        return x, hist
