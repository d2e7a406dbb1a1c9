"""Pins of the oracle's gradient formulas (oracle/gradients.py) against
finite differences of its own dense solve at Nside 4, and of the
Wiener-filter data term against the pixel-space covariance M = N + Y B S B
Y^T formed densely (the Woodbury identity).  A dropped term or a wrong sign
in any of the formulas fails one of these."""
import numpy as np
import pytest

from oracle import geometry, gradients, operators, sht


def small_problem(cl0=0.0):
    nside, L = 4, 8
    g = geometry.healpix_grid(nside)
    l = np.arange(L + 1.0)
    cl = np.zeros(L + 1)
    cl[2:] = 5.0 / (l[2:] * (l[2:] + 1))
    cl[0] = cl[1] = cl0
    bl = np.exp(-0.01 * l * (l + 1))
    rng = np.random.default_rng(3)
    ninv = rng.uniform(0.5, 3.0, size=g["npix"])
    ninv[rng.random(g["npix"]) < 0.15] = 0.0
    return operators.Problem(L, cl, bl, ninv, g), rng


def rebuild(prob, cl=None, ninv=None):
    return operators.Problem(prob.lmax, prob.cl if cl is None else cl, prob.bl,
                             prob.ninv if ninv is None else ninv, prob.grid)


@pytest.mark.parametrize("cl0", [0.0, 0.3])
def test_realization_gradient_matches_finite_differences(cl0):
    prob, rng = small_problem(cl0)
    d = rng.normal(size=prob.grid["npix"]) * 2.0
    w = sht.random_alm(prob.lmax, 9) if hasattr(sht, "random_alm") else None
    if w is None:
        w = rng.normal(size=sht.n_lm(prob.lmax)) + 1j * rng.normal(size=sht.n_lm(prob.lmax))
    w = prob.clean(w)
    seed = 4242
    gcl, gn, _ = gradients.realization_grad(prob, seed, d, w)
    for l in [0, 2, 5, 8]:
        if prob.cl[l] <= 0:
            assert gcl[l] == 0.0
            continue
        h = 1e-5 * prob.cl[l]
        cp, cm = prob.cl.copy(), prob.cl.copy()
        cp[l] += h
        cm[l] -= h
        fd = (gradients.realization_loss(rebuild(prob, cl=cp), seed, d, w)[0]
              - gradients.realization_loss(rebuild(prob, cl=cm), seed, d, w)[0]) / (2 * h)
        assert abs(fd - gcl[l]) < 1e-6 * max(1.0, abs(fd)), (l, fd, gcl[l])
    for i in np.nonzero(prob.ninv > 0)[0][:4]:
        h = 1e-5 * prob.ninv[i]
        npl, nmi = prob.ninv.copy(), prob.ninv.copy()
        npl[i] += h
        nmi[i] -= h
        fd = (gradients.realization_loss(rebuild(prob, ninv=npl), seed, d, w)[0]
              - gradients.realization_loss(rebuild(prob, ninv=nmi), seed, d, w)[0]) / (2 * h)
        assert abs(fd - gn[i]) < 1e-6 * max(1.0, abs(fd)), (i, fd, gn[i])


def test_wf_data_term_woodbury_and_gradient():
    prob, rng = small_problem(0.3)
    d = rng.normal(size=prob.grid["npix"]) * 2.0
    D, gcl, gn, _ = gradients.wf_data_term(prob, d)
    assert abs(D - gradients.wf_data_term_pixel(prob, d)) < 1e-9 * abs(D)
    for l in [0, 1, 4, 8]:
        h = 1e-5 * prob.cl[l]
        cp, cm = prob.cl.copy(), prob.cl.copy()
        cp[l] += h
        cm[l] -= h
        fd = (gradients.wf_data_term(rebuild(prob, cl=cp), d)[0] - gradients.wf_data_term(rebuild(prob, cl=cm), d)[0]) / (2 * h)
        assert abs(fd - gcl[l]) < 1e-6 * max(1.0, abs(fd)), (l, fd, gcl[l])
    for i in np.nonzero(prob.ninv > 0)[0][:4]:
        h = 1e-5 * prob.ninv[i]
        npl, nmi = prob.ninv.copy(), prob.ninv.copy()
        npl[i] += h
        nmi[i] -= h
        fd = (gradients.wf_data_term(rebuild(prob, ninv=npl), d)[0]
              - gradients.wf_data_term(rebuild(prob, ninv=nmi), d)[0]) / (2 * h)
        assert abs(fd - gn[i]) < 1e-6 * max(1.0, abs(fd)), (i, fd, gn[i])


def test_logdet_gradient_matches_finite_differences_of_dense_logdet():
    prob, rng = small_problem(0.3)
    gcl, gn = gradients.logdet_grad_exact(prob)
    f = lambda p: -0.5 * gradients.logdet_M(p)
    for l in [0, 1, 3, 8]:
        h = 1e-5 * prob.cl[l]
        cp, cm = prob.cl.copy(), prob.cl.copy()
        cp[l] += h
        cm[l] -= h
        fd = (f(rebuild(prob, cl=cp)) - f(rebuild(prob, cl=cm))) / (2 * h)
        assert abs(fd - gcl[l]) < 1e-6 * max(1.0, abs(fd)), (l, fd, gcl[l])
    for i in np.nonzero(prob.ninv > 0)[0][:4]:
        h = 1e-5 * prob.ninv[i]
        npl, nmi = prob.ninv.copy(), prob.ninv.copy()
        npl[i] += h
        nmi[i] -= h
        fd = (f(rebuild(prob, ninv=npl)) - f(rebuild(prob, ninv=nmi))) / (2 * h)
        assert abs(fd - gn[i]) < 1e-6 * max(1.0, abs(fd)), (i, fd, gn[i])


def test_hutchinson_estimate_converges_to_exact_trace():
    prob, rng = small_problem(0.3)
    gcl, gn = gradients.logdet_grad_exact(prob)
    hcl, hn = gradients.logdet_grad_hutchinson(prob, 31, 400)
    act = prob.cl > 0
    assert np.max(np.abs(hcl - gcl)[act] / np.abs(gcl[act])) < 0.1
    obs = prob.ninv > 0
    assert np.linalg.norm((hn - gn)[obs]) < 0.1 * np.linalg.norm(gn[obs])
