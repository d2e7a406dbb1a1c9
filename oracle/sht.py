"""Direct FP64 spherical-harmonic synthesis ``Y`` and adjoint synthesis ``Y^T``
(Section 2.1, Eq. sh-synthesis; the adjoint is the transpose of ``Y``, not
analysis).  Thin ctypes front of ``sht_direct.c``.

Oracle module -- test infrastructure only.

a_lm storage: complex128, m-major, l = m..lmax contiguous, index
``lm_index(lmax, l, m) = m(lmax+1) - m(m-1)/2 + (l - m)``.  Real fields are
represented by m >= 0 coefficients; Im(a_l0) is not a degree of freedom.
The real inner product that makes ``Y^T`` the transpose of ``Y`` is
``<a, b> = sum_l a_l0 b_l0 + 2 sum_{m>0} Re(a_lm conj(b_lm))``.
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int64)
        _lib.oracle_synth.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ip, ip, dp, dp, dp]
        _lib.oracle_adjoint.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ip, ip, dp, dp, dp]
        _lib.oracle_plm.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
        _lib.oracle_ring_dft.argtypes = [ctypes.c_int, ctypes.c_int, ip, ip, dp, dp, dp]
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def n_lm(lmax):
    return (lmax + 1) * (lmax + 2) // 2


def lm_offset(lmax, m):
    return m * (lmax + 1) - m * (m - 1) // 2


def lm_index(lmax, l, m):
    return lm_offset(lmax, m) + (l - m)


def lm_arrays(lmax):
    """(l, m) of every stored coefficient, in storage order."""
    ls, ms = [], []
    for m in range(lmax + 1):
        ls.append(np.arange(m, lmax + 1))
        ms.append(np.full(lmax + 1 - m, m))
    return np.concatenate(ls), np.concatenate(ms)


def _ring_args(grid, rings=None):
    z = np.ascontiguousarray(grid["z"], dtype=np.float64)
    sth = np.ascontiguousarray(grid["sth"], dtype=np.float64)
    nphi = np.ascontiguousarray(grid["nphi"], dtype=np.int64)
    off = np.ascontiguousarray(grid["off"], dtype=np.int64)
    phi0 = np.ascontiguousarray(grid["phi0"], dtype=np.float64)
    if rings is not None:
        z, sth, nphi, off, phi0 = (np.ascontiguousarray(a[rings]) for a in (z, sth, nphi, off, phi0))
    return z, sth, nphi, off, phi0


def synth(alm, lmax, grid, rings=None):
    """map = Y a.  With ``rings`` (an index array) only those rings are
    computed; other pixels are left at zero."""
    alm = np.ascontiguousarray(alm, dtype=np.complex128)
    assert alm.shape == (n_lm(lmax),)
    z, sth, nphi, off, phi0 = _ring_args(grid, rings)
    out = np.zeros(grid["npix"])
    lib().oracle_synth(lmax, len(z), _dp(z), _dp(sth), _ip(nphi), _ip(off), _dp(phi0),
                       _dp(alm.view(np.float64)), _dp(out))
    return out


def adjoint(m, lmax, grid, rings=None):
    """a = Y^T map (adjoint synthesis, no quadrature weights).  With ``rings``
    only those rings contribute."""
    m = np.ascontiguousarray(m, dtype=np.float64)
    assert m.shape == (grid["npix"],)
    z, sth, nphi, off, phi0 = _ring_args(grid, rings)
    out = np.zeros(n_lm(lmax), dtype=np.complex128)
    lib().oracle_adjoint(lmax, len(z), _dp(z), _dp(sth), _ip(nphi), _ip(off), _dp(phi0), _dp(m),
                         _dp(out.view(np.float64)))
    return out


def plm(lmax, m, z, sth=None):
    """Normalised associated Legendre P~_lm(z) for l = m..lmax (Section 3.3),
    Condon-Shortley phase included."""
    if sth is None:
        sth = np.sqrt((1.0 - z) * (1.0 + z))
    out = np.zeros(lmax - m + 1)
    lib().oracle_plm(lmax, m, float(z), float(sth), _dp(out))
    return out


def ring_dft(map_, grid, dmax):
    """X[k, d] = sum_j map_kj e^{-i d phi_kj} for d = 0..dmax (direct DFT)."""
    map_ = np.ascontiguousarray(map_, dtype=np.float64)
    _, _, nphi, off, phi0 = _ring_args(grid)
    out = np.zeros((grid["nring"], dmax + 1), dtype=np.complex128)
    lib().oracle_ring_dft(dmax, grid["nring"], _ip(nphi), _ip(off), _dp(phi0), _dp(map_),
                          _dp(out.view(np.float64)))
    return out


def alm_dot(a, b, lmax):
    """Real inner product of two m>=0 coefficient vectors."""
    _, ms = lm_arrays(lmax)
    w = np.where(ms == 0, 1.0, 2.0)
    return float(np.sum(w * (a.real * b.real + a.imag * b.imag)))


def alm_to_real(a, lmax):
    """Real degree-of-freedom vector u with <a,b> = u_a . u_b:
    [a_l0 (l=0..lmax) | sqrt2 Re a_lm, sqrt2 Im a_lm for m>=1 in storage order]."""
    n0 = lmax + 1
    r2 = np.sqrt(2.0)
    rest = a[n0:]
    u = np.empty((lmax + 1) ** 2)
    u[:n0] = a[:n0].real
    u[n0::2] = r2 * rest.real
    u[n0 + 1::2] = r2 * rest.imag
    return u


def real_to_alm(u, lmax):
    n0 = lmax + 1
    r2 = np.sqrt(2.0)
    a = np.zeros(n_lm(lmax), dtype=np.complex128)
    a[:n0] = u[:n0]
    a[n0:] = (u[n0::2] + 1j * u[n0 + 1::2]) / r2
    return a
