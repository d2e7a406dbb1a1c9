"""Gradients of a constrained realization and of the Wiener-filter data term
with respect to C_l and the inverse-noise map, for the system of Section 2.3
(Eq. system-explicit), by dense linear algebra at tiny sizes.

Oracle module -- test infrastructure only.

Realization: x = A^-1 b with b = B Y^T (N^-1 d + N^-1/2 w2) + S^-1/2 w1
(``draw.draw_rhs``).  For a loss L(x) = <w, x> (real inner product) the
adjoint vector is lambda = A^-1 w and, differentiating A x = b,
  dL/dC_l = C_l^-2 <lambda, x>_l - 1/2 C_l^-3/2 <lambda, a1>_l,
  dL/dn_i = -(Y B lambda)_i (Y B x)_i + (Y B lambda)_i (d_i + w2_i / (2 sqrt n_i)),
with a1 the complex-storage w1 and <.,.>_l the inner product restricted to
multipole l.

Log-determinant term: -1/2 ln det M with ln det M = ln det N + ln det S +
ln det A (over the observed pixels, N = diag(1/n)), so
  d/dC_l = -1/2 ((2l+1)/C_l - C_l^-2 tr(P_l A^-1 P_l)),
  d/dn_i = -1/2 (-1/n_i + (Y B A^-1 B Y^T)_ii)     (n_i > 0),
exactly from the dense A^-1, or by Hutchinson's estimator with the
Rademacher probes of ``draw.rademacher`` (the estimator the GPU runs).

Wiener-filter data term: with M = N + Y B S B Y^T (pixel covariance of the
data over observed pixels), d^T M^-1 d = d^T N^-1 d - b^T A^-1 b,
b = B Y^T N^-1 d (Woodbury), so
  D = -1/2 (d^T N^-1 d - b^T xh),   xh = A^-1 b,
  dD/dC_l = 1/2 C_l^-2 <xh, xh>_l,  dD/dn_i = -1/2 (d_i - (Y B xh)_i)^2.
"""
import math

import numpy as np
import scipy.linalg

from . import draw, operators, sht


def _dense(prob):
    act = operators.real_active_mask(prob)
    A = operators.dense_matrix(lambda v: operators.apply_A(prob, v), prob.lmax, act)
    return 0.5 * (A + A.T), act


def solve_dense(prob, b, A=None, act=None):
    if A is None:
        A, act = _dense(prob)
    u = sht.alm_to_real(prob.clean(b), prob.lmax)[act]
    x = np.zeros((prob.lmax + 1) ** 2)
    x[act] = scipy.linalg.cho_solve(scipy.linalg.cho_factor(A, lower=True), u)
    return sht.real_to_alm(x, prob.lmax)


def per_l_dot(u, v, L):
    """<u, v>_l for every l (real inner product restricted to multipole l)."""
    l, m = sht.lm_arrays(L)
    w = np.where(m == 0, 1.0, 2.0)
    t = w * (u.real * v.real + np.where(m == 0, 0.0, u.imag * v.imag))
    return np.bincount(l, weights=t, minlength=L + 1)


def prior_normals(prob, seed, rhs=0):
    """w1 in complex storage (w_l0, (w_re + i w_im) / sqrt2)."""
    n = sht.n_lm(prob.lmax)
    w = draw.normals(seed, draw.STREAM_OMEGA1, 2 * n, rhs)
    return np.where(prob.m == 0, w[0::2] + 0j, (w[0::2] + 1j * w[1::2]) / math.sqrt(2.0))


def realization_loss(prob, seed, d, w, rhs=0):
    b = draw.draw_rhs(prob, seed, d, fluct=True, rhs=rhs)
    x = solve_dense(prob, b)
    return sht.alm_dot(w, x, prob.lmax), x


def realization_grad(prob, seed, d, w, rhs=0):
    """(dL/dC_l [lmax+1], dL/dn [npix], x) for L = <w, x>."""
    A, act = _dense(prob)
    L = prob.lmax
    b = draw.draw_rhs(prob, seed, d, fluct=True, rhs=rhs)
    x = solve_dense(prob, b, A, act)
    lam = solve_dense(prob, prob.clean(w), A, act)
    cl = prob.cl
    with np.errstate(divide="ignore"):
        si = np.where(cl > 0, 1.0 / np.where(cl > 0, cl, 1.0), 0.0)
    a1 = prior_normals(prob, seed, rhs)
    gcl = si ** 2 * per_l_dot(lam, x, L) - 0.5 * si ** 1.5 * per_l_dot(lam, a1, L)
    bl = prob.bl[prob.l]
    p = sht.synth(bl * lam, L, prob.grid)
    q = sht.synth(bl * x, L, prob.grid)
    w2 = draw.normals(seed, draw.STREAM_OMEGA2, prob.grid["npix"], rhs)
    n = prob.ninv
    dd = np.zeros(prob.grid["npix"]) if d is None else np.asarray(d, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        fl = np.where(n > 0, w2 / (2.0 * np.sqrt(np.where(n > 0, n, 1.0))), 0.0)
    gn = -p * q + p * (dd + fl)
    return gcl, gn, x


def wf_data_term(prob, d):
    """(D, dD/dC_l, dD/dn, xh)."""
    A, act = _dense(prob)
    L = prob.lmax
    bl = prob.bl[prob.l]
    b = prob.clean(bl * sht.adjoint(prob.ninv * d, L, prob.grid))
    xh = solve_dense(prob, b, A, act)
    D = -0.5 * (np.sum(prob.ninv * d * d) - sht.alm_dot(b, xh, L))
    cl = prob.cl
    with np.errstate(divide="ignore"):
        si = np.where(cl > 0, 1.0 / np.where(cl > 0, cl, 1.0), 0.0)
    gcl = 0.5 * si ** 2 * per_l_dot(xh, xh, L)
    q = sht.synth(bl * xh, L, prob.grid)
    gn = -0.5 * (d - q) ** 2
    return D, gcl, gn, xh


def wf_data_term_pixel(prob, d):
    """-1/2 d^T M^-1 d over the observed pixels with M = N + Y B S B Y^T
    formed densely (the left side of the Woodbury identity)."""
    L = prob.lmax
    obs = np.nonzero(prob.ninv > 0)[0]
    npix = prob.grid["npix"]
    # columns of Y B S^1/2 in the real basis
    act = operators.real_active_mask(prob)
    nd = int(act.sum())
    cols = np.zeros((npix, nd))
    idx = np.nonzero(act)[0]
    l_of_real = np.concatenate([np.arange(L + 1)] + [np.repeat(np.arange(m, L + 1), 2) for m in range(1, L + 1)])
    for j, k in enumerate(idx):
        u = np.zeros((L + 1) ** 2)
        u[k] = 1.0
        a = sht.real_to_alm(u, L)
        lk = l_of_real[k]
        cols[:, j] = sht.synth(prob.bl[prob.l] * a, L, prob.grid) * math.sqrt(prob.cl[lk])
    K = cols[obs] @ cols[obs].T
    M = np.diag(1.0 / prob.ninv[obs]) + K
    return -0.5 * d[obs] @ np.linalg.solve(M, d[obs])


def _ainv_dense(prob):
    A, act = _dense(prob)
    return np.linalg.inv(A), act


def logdet_grad_exact(prob):
    """(d/dC_l, d/dn) of -1/2 ln det M, traces from the dense inverse."""
    L = prob.lmax
    Ainv, act = _ainv_dense(prob)
    l_real = np.concatenate([np.arange(L + 1)] + [np.repeat(np.arange(m, L + 1), 2) for m in range(1, L + 1)])
    la = l_real[act]
    tr = np.bincount(la, weights=np.diag(Ainv), minlength=L + 1)
    nu = np.bincount(la, minlength=L + 1).astype(np.float64)
    cl = prob.cl
    with np.errstate(divide="ignore", invalid="ignore"):
        gcl = np.where(cl > 0, -0.5 * (nu / np.where(cl > 0, cl, 1.0) - tr / np.where(cl > 0, cl, 1.0) ** 2), 0.0)
    # (Y B A^-1 B Y^T)_ii: columns of Y B in the real basis
    npix = prob.grid["npix"]
    idx = np.nonzero(act)[0]
    YB = np.zeros((npix, idx.size))
    for j, k in enumerate(idx):
        u = np.zeros((L + 1) ** 2)
        u[k] = 1.0
        YB[:, j] = sht.synth(prob.bl[prob.l] * sht.real_to_alm(u, L), L, prob.grid)
    diag = np.einsum("ij,jk,ik->i", YB, Ainv, YB)
    n = prob.ninv
    with np.errstate(divide="ignore"):
        gn = np.where(n > 0, -0.5 * (-1.0 / np.where(n > 0, n, 1.0) + diag), 0.0)
    return gcl, gn


def logdet_grad_hutchinson(prob, seed, nprobe):
    """The same gradient with both traces by Hutchinson over nprobe probes."""
    L = prob.lmax
    cl, n = prob.cl, prob.ninv
    nlm = sht.n_lm(L)
    A, act = _dense(prob)
    trs = np.zeros(L + 1)
    dg = np.zeros(prob.grid["npix"])
    bl = prob.bl[prob.l]
    for j in range(nprobe):
        zr = draw.rademacher(seed, 5, 2 * nlm, j)
        z = np.where(prob.m == 0, zr[0::2] + 0j, (zr[0::2] + 1j * zr[1::2]) / math.sqrt(2.0))
        z = prob.clean(z)
        trs += per_l_dot(z, solve_dense(prob, z, A, act), L)
        w = np.where(n > 0, draw.rademacher(seed, 6, prob.grid["npix"], j), 0.0)
        bw = prob.clean(bl * sht.adjoint(w, L, prob.grid))
        dg += sht.synth(bl * solve_dense(prob, bw, A, act), L, prob.grid) * w
    trs /= nprobe
    dg /= nprobe
    l = np.arange(L + 1)
    nu = np.where(cl > 0, 2 * l + 1.0, 0.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        gcl = np.where(cl > 0, -0.5 * (nu / np.where(cl > 0, cl, 1.0) - trs / np.where(cl > 0, cl, 1.0) ** 2), 0.0)
        gn = np.where(n > 0, -0.5 * (-1.0 / np.where(n > 0, n, 1.0) + dg), 0.0)
    return gcl, gn


def logdet_M(prob):
    """ln det M over the observed pixels, M = N + Y B S B Y^T, formed densely."""
    L = prob.lmax
    obs = np.nonzero(prob.ninv > 0)[0]
    act = operators.real_active_mask(prob)
    l_real = np.concatenate([np.arange(L + 1)] + [np.repeat(np.arange(m, L + 1), 2) for m in range(1, L + 1)])
    cols = []
    for k in np.nonzero(act)[0]:
        u = np.zeros((L + 1) ** 2)
        u[k] = 1.0
        cols.append(sht.synth(prob.bl[prob.l] * sht.real_to_alm(u, L), L, prob.grid)[obs] * math.sqrt(prob.cl[l_real[k]]))
    K = np.stack(cols, axis=1)
    M = np.diag(1.0 / prob.ninv[obs]) + K @ K.T
    return np.linalg.slogdet(M)[1]
