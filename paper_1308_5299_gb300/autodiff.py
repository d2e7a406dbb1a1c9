"""Differentiable constrained realizations and Wiener-filter data term
(torch.autograd.Function over the C ABI; argument marshalling only).

realization(cl, ninv, ...): x = A^-1 b with A = S^-1 + B Y^T N^-1 Y B and the
constrained-realization right-hand side b = B Y^T (N^-1 d + N^-1/2 w2) +
S^-1/2 w1 of cr_draw (Section 2.3).  Forward: cr_draw + CR-Solve.  Backward:
A is symmetric, so lambda = A^-1 g is the same CR-Solve on the loss gradient,
followed by the contractions cr_grad_cl / cr_grad_ninv:
  dL/dC_l = C_l^-2 <lambda, x>_l - 1/2 C_l^-3/2 <lambda, w1>_l,
  dL/dn_i = -(Y B lambda)_i (Y B x)_i + (Y B lambda)_i (d_i + w2_i / (2 sqrt n_i)).

wf_data_term(cl, ninv, d): D = -1/2 (d^T N^-1 d - b^T A^-1 b), b = B Y^T N^-1 d
(the data part of the Wiener-filter log-likelihood, by the Woodbury
identity), with dD/dC_l = 1/2 C_l^-2 <xh, xh>_l and dD/dn_i =
-1/2 (d_i - (Y B xh)_i)^2, xh = A^-1 b.

wf_loglike_grad(cl, ninv, d, nprobe): the gradient of the whole Wiener-filter
log-likelihood -1/2 d^T M^-1 d - 1/2 ln det M, M = N + Y B S B Y^T: the data
term above plus the log-determinant term (determinant lemma ln det M =
ln det N + ln det S + ln det A)
  d/dC_l = -1/2 ((2l+1)/C_l - C_l^-2 tr_l A^-1),
  d/dn_i = -1/2 (-1/n_i + (Y B A^-1 B Y^T)_ii),
with both traces estimated by Hutchinson over nprobe Rademacher probes
(cr_probe), each needing one more solve.

Complex gradients follow torch's convention G = dL/dRe x + i dL/dIm x; the
library's adjoint right-hand side g satisfies dL = <g, dx> in its real inner
product, so g = G at m = 0 and G / 2 at m > 0 (a convention conversion).
"""
import numpy as np
import torch

from . import binding


def _m_weights(lmax, device):
    m = np.concatenate([np.full(lmax + 1 - mm, mm) for mm in range(lmax + 1)])
    return torch.from_numpy(np.where(m == 0, 1.0, 0.5)).to(device)


def _plan(cl, ninv, bl, nside, levels, stream):
    return binding.Plan(len(bl) - 1, nside=nside, cl=cl.detach().cpu().numpy().astype(np.float64),
                        bl=np.asarray(bl, dtype=np.float64), ninv=ninv.detach().contiguous(), levels=levels,
                        stream=stream)


class _Realization(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cl, ninv, bl, nside, d, seed, nrhs, solve_kw):
        plan = _plan(cl, ninv, bl, nside, "default", None)
        nlm = binding.n_lm(plan.lmax)
        b = torch.empty((nrhs, nlm), dtype=torch.complex128, device=ninv.device)
        plan.draw(seed, b, d=d, fluct=True)
        x = torch.empty_like(b)
        plan.solve(b, x, **solve_kw)
        ctx.plan, ctx.seed, ctx.nrhs, ctx.solve_kw = plan, seed, nrhs, solve_kw
        ctx.d = d
        ctx.save_for_backward(x)
        ctx.cl_dev = cl.device
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        plan = ctx.plan
        g = (gx.contiguous() * _m_weights(plan.lmax, gx.device)).contiguous()
        lam = torch.empty_like(g)
        plan.solve(g, lam, **ctx.solve_kw)
        gcl = torch.zeros(plan.lmax + 1, dtype=torch.float64, device=x.device)
        gn = torch.zeros(plan.npix, dtype=torch.float64, device=x.device)
        for j in range(ctx.nrhs):
            dj = None if ctx.d is None else ctx.d[j].contiguous()
            plan.grad_cl(lam[j].contiguous(), x[j].contiguous(), 1.0, -0.5, ctx.seed, j, out=gcl, accumulate=True)
            plan.grad_ninv(lam[j].contiguous(), x[j].contiguous(), dj, -1.0, 1.0, 0.5, 0.0, ctx.seed, j, out=gn,
                           accumulate=True)
        return gcl.to(ctx.cl_dev), gn, None, None, None, None, None, None


class _WFData(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cl, ninv, bl, nside, d, solve_kw):
        plan = _plan(cl, ninv, bl, nside, "default", None)
        nlm = binding.n_lm(plan.lmax)
        b = torch.empty(nlm, dtype=torch.complex128, device=ninv.device)
        plan.draw(0, b, d=d, fluct=False)
        xh = torch.empty_like(b)
        plan.solve(b, xh, **solve_kw)
        val = -0.5 * (plan.map_wdot(d, d) - plan.alm_dot(b, xh))
        ctx.plan, ctx.d = plan, d
        ctx.save_for_backward(xh)
        ctx.cl_dev = cl.device
        return torch.tensor(val, dtype=torch.float64, device=ninv.device)

    @staticmethod
    def backward(ctx, gD):
        (xh,) = ctx.saved_tensors
        plan = ctx.plan
        s = float(gD)
        gcl = plan.grad_cl(xh, xh, 0.5 * s, 0.0)
        gn = plan.grad_ninv(xh, xh, ctx.d, -0.5 * s, s, 0.0, -0.5 * s)
        return gcl.to(ctx.cl_dev), gn, None, None, None, None


DEFAULT_SOLVE = dict(eps=1e-24, max_cycles=80, mode=binding.CR_MIXED | binding.CR_PCG)


def realization(cl, ninv, bl, nside, d=None, seed=0, nrhs=1, solve_kw=None):
    """Constrained realizations x [nrhs, N_lm] (complex128, CUDA),
    differentiable with respect to cl (float64 [lmax+1]) and ninv (float64
    CUDA [npix]).  d: float64 CUDA [nrhs, npix] data or None."""
    return _Realization.apply(cl, ninv, bl, nside, d, seed, nrhs, dict(DEFAULT_SOLVE, **(solve_kw or {})))


def wf_data_term(cl, ninv, bl, nside, d, solve_kw=None):
    """Wiener-filter data term D (scalar), differentiable in cl and ninv."""
    return _WFData.apply(cl, ninv, bl, nside, d, dict(DEFAULT_SOLVE, **(solve_kw or {})))


def wf_loglike_grad(cl, ninv, bl, nside, d, nprobe=8, seed=0, solve_kw=None):
    """(D, dL/dC_l, dL/dn): the Wiener-filter data term D and the gradient of
    the whole log-likelihood (data term exact, log-determinant term by
    Hutchinson over nprobe probes).  cl float64 [lmax+1], ninv and d float64
    CUDA [npix]; returns CUDA tensors."""
    kw = dict(DEFAULT_SOLVE, **(solve_kw or {}))
    plan = _plan(cl, ninv, bl, nside, "default", None)
    nlm = binding.n_lm(plan.lmax)
    dev = ninv.device
    b = torch.empty(nlm, dtype=torch.complex128, device=dev)
    plan.draw(0, b, d=d, fluct=False)
    xh = torch.empty_like(b)
    plan.solve(b, xh, **kw)
    D = -0.5 * (plan.map_wdot(d, d) - plan.alm_dot(b, xh))
    gcl = plan.grad_cl(xh, xh, 0.5, 0.0, kappa=-0.5)
    gn = plan.grad_ninv(xh, xh, d, -0.5, 1.0, 0.0, -0.5, kappa=0.5)
    z = torch.empty(nlm, dtype=torch.complex128, device=dev)
    lam = torch.empty_like(z)
    w = torch.empty(plan.npix, dtype=torch.float64, device=dev)
    bw = torch.empty_like(z)
    for j in range(nprobe):
        plan.probe(seed, binding.CR_PROBE_ALM, j, z)
        plan.solve(z, lam, **kw)
        plan.grad_cl(z, lam, 0.5 / nprobe, 0.0, out=gcl, accumulate=True)
        plan.probe(seed, binding.CR_PROBE_MAP, j, w)
        plan.draw(0, bw, d=w, fluct=False, plain=True)
        plan.solve(bw, lam, **kw)
        plan.grad_ninv(lam, None, w, 0.0, -0.5 / nprobe, 0.0, 0.0, out=gn, accumulate=True)
    return D, gcl, gn
