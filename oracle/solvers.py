"""Reference solvers for A x = b.

Oracle module -- test infrastructure only.

The method iterates toward the exact solution of A x = b (Section 2.3), so the
oracle defines the answer as x* = A^-1 b, computed two independent ways:
  * ``dense_solve``: form A by probing and Cholesky-solve (tiny sizes);
  * ``pcg``: plain diagonal-preconditioned conjugate gradients (Section 2.4,
    the baseline the paper compares against), run to a tight residual.
"""
import numpy as np
import scipy.linalg

from . import operators, sht


def dense_solve(prob, b, apply_fn=None):
    """x = A^-1 b with A formed densely by probing (real basis), Cholesky."""
    L = prob.lmax
    f = apply_fn or (lambda v: operators.apply_A(prob, v))
    act = operators.real_active_mask(prob)
    A = operators.dense_matrix(f, L, act)
    ub = sht.alm_to_real(prob.clean(b), L)[act]
    c = scipy.linalg.cho_factor(0.5 * (A + A.T), lower=True)
    u = np.zeros((L + 1) ** 2)
    u[act] = scipy.linalg.cho_solve(c, ub)
    return sht.real_to_alm(u, L), A


def pcg(apply_fn, b, precond_diag, lmax, tol=1e-12, maxiter=20000, x0=None, callback=None):
    """Preconditioned CG in the real inner product of m>=0 coefficient
    vectors; stops when ||r|| <= tol ||b||.  ``precond_diag`` multiplies the
    residual (zero entries mark non-unknowns).  Returns (x, iterations,
    relative residual)."""
    dot = lambda u, v: sht.alm_dot(u, v, lmax)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_fn(x) if x0 is not None else b.copy()
    z = precond_diag * r
    p = z.copy()
    rz = dot(r, z)
    bn = np.sqrt(dot(b, b))
    it = 0
    rel = np.sqrt(dot(r, r)) / bn
    while rel > tol and it < maxiter:
        Ap = apply_fn(p)
        alpha = rz / dot(p, Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        z = precond_diag * r
        rz_new = dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
        rel = np.sqrt(dot(r, r)) / bn
        if callback is not None:
            callback(it, x, rel)
    return x, it, rel
