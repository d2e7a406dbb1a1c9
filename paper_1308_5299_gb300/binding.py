"""Thin ctypes binding over the C ABI in ``include/cr.h``.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libcrgb300.so``.  Tensors must be CUDA tensors (torch supplies
device memory and streams); there is no CPU fallback -- if the shared library
is missing or a call fails, a ``CRError`` is raised.

Coefficient vectors are complex tensors (complex128 for CR_F64, complex64 for
CR_F32) in the library's layout (m >= 0, m-major, l contiguous); maps are
real tensors in RING order.  A leading batch dimension is the nrhs of a call.
"""
import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcrgb300.so")

CR_OK = 0
CR_F64, CR_F32 = 0, 1
CR_GRID_HEALPIX, CR_GRID_GL = 0, 1
CR_OBS = 0

ERRORS = {-1: "CR_EINVAL", -2: "CR_ENOMEM", -3: "CR_ECUDA", -4: "CR_EICC", -5: "CR_EDIVERGED",
          -6: "CR_EMAXITER", -7: "CR_ENONFINITE", -8: "CR_ESTATE", -9: "CR_EIO"}


class CRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class cr_params(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_int),
        ("grid_kind", ctypes.c_int),
        ("nside", ctypes.c_int),
        ("gl_ntheta", ctypes.c_int),
        ("gl_nphi", ctypes.c_int),
        ("lmax", ctypes.c_int),
        ("cl", ctypes.POINTER(ctypes.c_double)),
        ("bl", ctypes.POINTER(ctypes.c_double)),
        ("ninv", ctypes.c_void_p),
        ("stream", ctypes.c_void_p),
    ]


_lib = None

# exported entry points and their ctypes signatures (the names of include/cr.h)
_SIGS = {
    "cr_last_error": ([], ctypes.c_char_p),
    "cr_plan_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(cr_params)], ctypes.c_int),
    "cr_plan_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "cr_plan_sizes": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int),
                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "cr_sht_synth": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int],
                     ctypes.c_int),
    "cr_sht_adjoint": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int],
                       ctypes.c_int),
    "cr_apply_A": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int],
                   ctypes.c_int),
    "cr_sht_synth_noalloc": ([ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
                             ctypes.c_int),
    "cr_plan_set_timing": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "cr_plan_timing": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_char_p, ctypes.c_int,
                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_long),
                        ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
}


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise CRError(-3, "CUDA library %s not built (run __graft_entry__.build())" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(rc):
    if rc != CR_OK:
        raise CRError(rc, lib().cr_last_error().decode())


def _dtype_code(t):
    if t.dtype in (torch.complex128, torch.float64):
        return CR_F64
    if t.dtype in (torch.complex64, torch.float32):
        return CR_F32
    raise TypeError("unsupported dtype %s" % t.dtype)


def _dev(t):
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("tensors must be contiguous CUDA tensors")
    return ctypes.c_void_p(t.data_ptr())


def n_lm(lmax):
    return (lmax + 1) * (lmax + 2) // 2


def sht_synth_noalloc(nside, lmax, alm, out, stream=None):
    """FP64 synthesis with no plan and no allocation (``cr_sht_synth_noalloc``):
    for callers that cannot allocate device memory.  ``alm`` complex128 and
    ``out`` float64 CUDA tensors."""
    if alm.dtype != torch.complex128 or out.dtype != torch.float64:
        raise TypeError("sht_synth_noalloc is FP64 only")
    if alm.numel() != n_lm(lmax) or out.numel() != 12 * nside * nside:
        raise ValueError("sht_synth_noalloc: sizes")
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(lib().cr_sht_synth_noalloc(int(nside), int(lmax), _dev(alm), _dev(out), ctypes.c_void_p(st.cuda_stream)))
    return out


class Plan:
    """One CR system / transform plan (``cr_plan_create``)."""

    def __init__(self, lmax, nside=None, gl=None, cl=None, bl=None, ninv=None, stream=None):
        p = cr_params()
        p.struct_size = ctypes.sizeof(cr_params)
        if gl is not None:
            p.grid_kind = CR_GRID_GL
            p.gl_ntheta, p.gl_nphi = int(gl[0]), int(gl[1])
        else:
            p.grid_kind = CR_GRID_HEALPIX
            p.nside = int(nside)
        p.lmax = int(lmax)
        self._keep = []
        if cl is not None:
            cl = np.ascontiguousarray(cl, dtype=np.float64)
            self._keep.append(cl)
            p.cl = cl.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if bl is not None:
            bl = np.ascontiguousarray(bl, dtype=np.float64)
            self._keep.append(bl)
            p.bl = bl.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if ninv is not None:
            if not (ninv.is_cuda and ninv.dtype == torch.float64):
                raise ValueError("ninv must be a float64 CUDA tensor")
            ninv = ninv.contiguous()
            self._keep.append(ninv)
            p.ninv = ninv.data_ptr()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        p.stream = self.stream.cuda_stream
        h = ctypes.c_void_p()
        _check(lib().cr_plan_create(ctypes.byref(h), ctypes.byref(p)))
        self._h = h
        self.lmax = int(lmax)
        self._keep = []

    def close(self):
        if getattr(self, "_h", None):
            lib().cr_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sizes(self, grid=CR_OBS):
        npix, nring, lmax, nlm = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        _check(lib().cr_plan_sizes(self._h, grid, ctypes.byref(npix), ctypes.byref(nring), ctypes.byref(lmax),
                                   ctypes.byref(nlm)))
        return dict(npix=npix.value, nring=nring.value, lmax=lmax.value, nlm=nlm.value)

    @staticmethod
    def _nrhs(t, per):
        if t.numel() % per:
            raise ValueError("tensor size %d is not a multiple of %d" % (t.numel(), per))
        return t.numel() // per

    def sht_synth(self, alm, out, grid=CR_OBS):
        s = self.sizes(grid)
        nrhs = self._nrhs(alm, s["nlm"])
        if out.numel() != nrhs * s["npix"] or _dtype_code(alm) != _dtype_code(out):
            raise ValueError("sht_synth: output shape/dtype")
        _check(lib().cr_sht_synth(self._h, grid, _dev(alm), _dev(out), nrhs, _dtype_code(alm)))
        return out

    def sht_adjoint(self, map_, out, grid=CR_OBS):
        s = self.sizes(grid)
        nrhs = self._nrhs(map_, s["npix"])
        if out.numel() != nrhs * s["nlm"] or _dtype_code(map_) != _dtype_code(out):
            raise ValueError("sht_adjoint: output shape/dtype")
        _check(lib().cr_sht_adjoint(self._h, grid, _dev(map_), _dev(out), nrhs, _dtype_code(map_)))
        return out

    def set_timing(self, enable=True):
        _check(lib().cr_plan_set_timing(self._h, 1 if enable else 0))

    def timing(self):
        """{stage name: (total ms, launches)} since timing was enabled."""
        cnt = ctypes.c_int()
        _check(lib().cr_plan_timing(self._h, -1, None, 0, None, None, ctypes.byref(cnt)))
        out = {}
        for i in range(cnt.value):
            buf = ctypes.create_string_buffer(64)
            ms, n = ctypes.c_double(), ctypes.c_long()
            _check(lib().cr_plan_timing(self._h, i, buf, 64, ctypes.byref(ms), ctypes.byref(n), None))
            out[buf.value.decode()] = (ms.value, n.value)
        return out

    def apply_A(self, x, out, level=0):
        nrhs = self._nrhs(x, n_lm(self.lmax)) if level == 0 else x.numel() // max(1, out.numel())
        _check(lib().cr_apply_A(self._h, level, _dev(x), _dev(out), nrhs, _dtype_code(x)))
        return out
