"""The constrained-realization system and its level operators, written out
plainly in FP64 on top of the direct SHT.

Oracle module -- test infrastructure only.

  A   = S^-1 + B Y^T N^-1 Y B                     (Section 2.3, Eq. system-explicit)
  A_h = F_h A F_h = D_h + B_h Y^T N^-1 Y B_h       (Section 3.2, Eq. A_h)
        D_h = (f_h)^2 / C_l,  B_h = f_h b_l p_l,  band limit lmax_h
  b   = B Y^T N^-1 d (+ fluctuation terms)         (Eq. cr-system)

Reading (documented): coefficients with C_l = 0 are not unknowns -- their rows
and columns are removed (x_l = 0 there, the C_l -> 0 limit); Im(a_l0) is not
a degree of freedom and is kept at zero.
"""
import numpy as np

from . import sht


class Problem:
    """One CR system: band limit, prior C_l, beam*pixel window b_l p_l, the
    inverse-noise map (0 under the mask) on ``grid``."""

    def __init__(self, lmax, cl, bl, ninv, grid):
        self.lmax = int(lmax)
        self.cl = np.asarray(cl, dtype=np.float64)
        self.bl = np.asarray(bl, dtype=np.float64)
        self.ninv = np.asarray(ninv, dtype=np.float64)
        self.grid = grid
        assert self.cl.shape == (self.lmax + 1,) and self.bl.shape == (self.lmax + 1,)
        assert self.ninv.shape == (grid["npix"],)
        self.l, self.m = sht.lm_arrays(self.lmax)
        self.active = self.cl[self.l] > 0

    def clean(self, x):
        """Zero the non-degrees of freedom: C_l = 0 rows and Im(a_l0)."""
        x = np.array(x, dtype=np.complex128)
        x[~self.active] = 0.0
        x[self.m == 0] = x[self.m == 0].real
        return x


def apply_inv_noise_term(prob, x, lmax=None, gl=None):
    """Y^T N^-1 Y x on the observation grid, for a band limit ``lmax``
    (default the problem's)."""
    L = prob.lmax if lmax is None else lmax
    mp = sht.synth(x, L, prob.grid)
    mp *= prob.ninv
    return sht.adjoint(mp, L, prob.grid)


def apply_A(prob, x):
    """A x = S^-1 x + B Y^T N^-1 Y B x  (Eq. system-explicit)."""
    x = prob.clean(x)
    bl = prob.bl[prob.l]
    y = bl * apply_inv_noise_term(prob, bl * x)
    y[prob.active] += x[prob.active] / prob.cl[prob.l[prob.active]]
    return prob.clean(y)


def level_coeffs(prob, fl, lmax_h):
    """Diagonals of the level operator for filter f_l (length >= lmax_h+1):
    D_h = f^2 / C_l and B_h = f b_l p_l, on the lmax_h layout (Eq. A_h)."""
    l, m = sht.lm_arrays(lmax_h)
    f = np.asarray(fl, dtype=np.float64)[: lmax_h + 1]
    cl = prob.cl[: lmax_h + 1]
    with np.errstate(divide="ignore"):
        d = np.where(cl > 0, f * f / np.where(cl > 0, cl, 1.0), 0.0)
    bh = f * prob.bl[: lmax_h + 1]
    active = cl[l] > 0
    return d[l], bh[l], active, l, m


def apply_A_level(prob, fl, lmax_h, x):
    """A_h x = D_h x + B_h Y^T N^-1 Y B_h x at band limit lmax_h (Eq. A_h)."""
    d, bh, active, l, m = level_coeffs(prob, fl, lmax_h)
    x = np.array(x, dtype=np.complex128)
    x[~active] = 0.0
    x[m == 0] = x[m == 0].real
    y = bh * apply_inv_noise_term(prob, bh * x, lmax=lmax_h)
    y += d * x
    y[~active] = 0.0
    y[m == 0] = y[m == 0].real
    return y


def restrict(fl_h, fl_H, lmax_h, lmax_H, x):
    """I_h^H: diagonal f_H / f_h for l <= lmax_H, dropped above (Eq. f_l)."""
    lh, mh = sht.lm_arrays(lmax_h)
    keep = lh <= lmax_H
    ratio = np.asarray(fl_H)[lh] / np.asarray(fl_h)[lh]
    return (x * np.where(keep, ratio, 0.0))[keep]


def prolong(fl_h, fl_H, lmax_h, lmax_H, c):
    """(I_h^H)^T: the transpose of ``restrict`` (zero-padded above lmax_H)."""
    lh, mh = sht.lm_arrays(lmax_h)
    keep = lh <= lmax_H
    out = np.zeros(sht.n_lm(lmax_h), dtype=np.complex128)
    out[keep] = c * (np.asarray(fl_H)[lh[keep]] / np.asarray(fl_h)[lh[keep]])
    return out


def dense_matrix(apply_fn, lmax, active=None):
    """Real-basis matrix of a linear map on m>=0 coefficient vectors, by
    applying it to every real unit vector (probing).  Rows/columns of
    inactive coefficients are dropped when ``active`` (bool per real dof) is
    given."""
    n = (lmax + 1) ** 2
    M = np.zeros((n, n))
    for i in range(n):
        u = np.zeros(n)
        u[i] = 1.0
        M[:, i] = sht.alm_to_real(apply_fn(sht.real_to_alm(u, lmax)), lmax)
    if active is not None:
        M = M[np.ix_(active, active)]
    return M


def real_active_mask(prob, lmax=None):
    """Boolean mask over real dofs (alm_to_real order) of active unknowns."""
    L = prob.lmax if lmax is None else lmax
    l, m = sht.lm_arrays(L)
    act = prob.cl[l] > 0
    return sht.alm_to_real(act.astype(np.complex128) * (1 + 1j), L) != 0


def ring_formula_inv_noise(prob, lmax_d):
    """Real-basis matrix of Y^T N^-1 Y restricted to l <= lmax_d, from the
    ring formula of Section 3.3 (Eq. Ni-dense):
      sum_k P~_l1m1(z_k) P~_l2m2(z_k) sum_j xi_kj e^{i(m1-m2) phi_kj}
    extended to real fields: in m>=0 storage
      (Y^T N Y a)_{l1 m1} = sum_k P1 sum_{l2,m2} (w_m2/2) P2
                            [a_{l2m2} X_k(m1-m2) + conj(a_{l2m2}) X_k(m1+m2)],
    X_k(d) = sum_j xi_kj e^{-i d phi_kj}, X_k(-d) = conj X_k(d), w_0=1, w_m=2.
    An independent route to the same numbers as probing ``apply_A``."""
    g = prob.grid
    L = lmax_d
    X = sht.ring_dft(prob.ninv, g, 2 * L)  # [k, d]

    def Xd(d):
        return X[:, d] if d >= 0 else np.conj(X[:, -d])

    P = {m: np.stack([sht.plm(L, m, g["z"][k], g["sth"][k]) for k in range(g["nring"])], axis=1)
         for m in range(L + 1)}  # P[m][l-m, k]
    n = (L + 1) ** 2
    M = np.zeros((n, n))
    r2 = np.sqrt(2.0)
    # column index of real dof for (l, m, part)
    def col_index(l, m, part):
        if m == 0:
            return l
        base = L + 1 + 2 * (sht.lm_offset(L, m) - (L + 1) + (l - m))
        return base + part

    for m1 in range(L + 1):
        for m2 in range(L + 1):
            T1 = (P[m1] * Xd(m1 - m2)[None, :]) @ P[m2].T  # [l1, l2]
            T2 = (P[m1] * Xd(m1 + m2)[None, :]) @ P[m2].T
            for i2, l2 in enumerate(range(m2, L + 1)):
                parts = [(0, 1.0 + 0j)] if m2 == 0 else [(0, 1.0 / r2 + 0j), (1, 1j / r2)]
                for part, a in parts:
                    # y_{l1 m1} = (w_m2/2)[a T1 + conj(a) T2]
                    w = 0.5 if m2 == 0 else 1.0
                    y = w * (a * T1[:, i2] + np.conj(a) * T2[:, i2])
                    c = col_index(l2, m2, part)
                    for i1, l1 in enumerate(range(m1, L + 1)):
                        if m1 == 0:
                            M[col_index(l1, 0, 0), c] = y[i1].real
                        else:
                            M[col_index(l1, m1, 0), c] = r2 * y[i1].real
                            M[col_index(l1, m1, 1), c] = r2 * y[i1].imag
    return M


def diag_inv_noise_dm0(prob, lmax=None):
    """Approximate diagonal of Y^T N^-1 Y: the Delta m = 0 term of the ring
    formula, sum_k P~_lm(z_k)^2 sum_j xi_kj (Sections 3.2-3.3; used for the
    top-level diagonal smoother)."""
    g = prob.grid
    L = prob.lmax if lmax is None else lmax
    ring_sum = np.add.reduceat(prob.ninv, g["off"])
    out = np.zeros(sht.n_lm(L))
    for m in range(L + 1):
        acc = np.zeros(L - m + 1)
        for k in range(g["nring"]):
            p = sht.plm(L, m, g["z"][k], g["sth"][k])
            acc += p * p * ring_sum[k]
        out[sht.lm_offset(L, m): sht.lm_offset(L, m) + L - m + 1] = acc
    return out
