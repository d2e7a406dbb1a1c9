"""Convergence diagnostics of the multi-level solver, computed through the
library's calls:

- error_by_scale (Fig. errors-by-scale, Section 5): the relative error
  ||x_true,l - x_l|| / ||x_true,l|| per multipole l after each W-cycle;
- smoother_only (Fig. smoother, Section 2.4): repeated error smoothing on one
  pixel level, x_h += S_h (b_h - A_h x_h), whose error falls only in part of
  the spectrum and then stagnates -- the observation behind the multi-level
  algorithm;
- filter_curves (Section 3.3, Fig. of the level filters): the cumulative
  filters f^h_l of every level.

The solves, smoothing steps and level operators run on the GPU; the per-l
norms of their results are evaluated here on the host (analysis of the
output, not a step of the solver).
"""
import numpy as np
import torch

from . import binding


def per_l_norm(alm, lmax):
    """sqrt(sum_m w_m |a_lm|^2) per l (w_0 = 1, w_m>0 = 2: the norm of the
    real field's l component) for complex m-major coefficients a[n_lm]."""
    a = np.asarray(alm)
    out = np.zeros(lmax + 1)
    off = 0
    for m in range(lmax + 1):
        n = lmax + 1 - m
        p = np.abs(a[off:off + n]) ** 2
        out[m:] += (1.0 if m == 0 else 2.0) * p
        off += n
    return np.sqrt(out)


def _rel_by_l(x, x_true, lmax):
    num = per_l_norm(x - x_true, lmax)
    den = per_l_norm(x_true, lmax)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(den > 0, num / den, np.nan)


def error_by_scale(plan, b, x_true, cycles, mode=binding.CR_MIXED):
    """[cycles][lmax+1] relative error per l after 1..cycles fixed W-cycles
    (stationary solve of b, host copies of the iterates)."""
    xt = x_true.detach().cpu().numpy()
    x = torch.empty_like(b)
    rows = []
    for k in range(1, cycles + 1):
        plan.solve(b, x, eps=0.0, max_cycles=k, mode=mode | binding.CR_FIXED, check=False)
        rows.append(_rel_by_l(x.cpu().numpy(), xt, plan.lmax))
    return np.array(rows)


def smoother_only(plan, h, x_true_h, iters):
    """Repeated error smoothing on pixel level h against a known level
    solution: b_h = A_h x_true_h, x_h = 0, then x_h += S_h (b_h - A_h x_h).
    Returns (relative residual per iteration, [iters][lmax_h+1] relative
    error per l)."""
    L = plan.level(h)["lmax_h"]
    b = torch.empty_like(x_true_h)
    plan.apply_A(x_true_h, b, level=h)
    x = torch.zeros_like(b)
    r = torch.empty_like(b)
    c = torch.empty_like(b)
    bn = float(torch.linalg.vector_norm(b))
    res, rows = [], []
    xt = x_true_h.detach().cpu().numpy()
    for _ in range(iters):
        plan.apply_A(x, r, level=h)
        r = b - r
        res.append(float(torch.linalg.vector_norm(r)) / bn)
        plan.smooth(h, r, c)
        x += c
        rows.append(_rel_by_l(x.cpu().numpy(), xt, L))
    return np.array(res), np.array(rows)


def filter_curves(plan):
    """{h: f^h_l} for the pixel levels h = 1..H and the bottom level H + 1."""
    return {h: plan.level(h)["fl"] for h in range(1, plan.nlevels() + 2)}
