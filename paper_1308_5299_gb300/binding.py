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
CR_F64, CR_F32, CR_MIXED, CR_PCG, CR_FIXED, CR_CG = 0, 1, 2, 4, 8, 16
CR_DRAW_FLUCT, CR_DRAW_PLAIN = 1, 2
CR_TC = 3
CR_TC_CYCLES = 32
CR_TC_TOP_F32 = 64
CR_TC_SPLIT = 128
CR_PROBE_ALM, CR_PROBE_MAP = 0, 1
CR_GRID_HEALPIX, CR_GRID_GL = 0, 1
CR_OBS = 0

ERRORS = {-1: "CR_EINVAL", -2: "CR_ENOMEM", -3: "CR_ECUDA", -4: "CR_EICC", -5: "CR_EDIVERGED",
          -6: "CR_EMAXITER", -7: "CR_ENONFINITE", -8: "CR_ESTATE", -9: "CR_EIO"}
(CR_EINVAL, CR_ENOMEM, CR_ECUDA, CR_EICC, CR_EDIVERGED, CR_EMAXITER, CR_ENONFINITE, CR_ESTATE,
 CR_EIO) = range(-1, -10, -1)


class CRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


class cr_level_spec(ctypes.Structure):
    _fields_ = [("nside_h", ctypes.c_int), ("lmax_h", ctypes.c_int), ("n_rec", ctypes.c_int),
                ("fl", ctypes.POINTER(ctypes.c_double))]


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
        ("nlevels", ctypes.c_int),
        ("levels", ctypes.POINTER(cr_level_spec)),
        ("lmax_dense", ctypes.c_int),
        ("ridge_factor", ctypes.c_double),
        ("ridge_bisections", ctypes.c_int),
        ("ridge_alpha", ctypes.POINTER(ctypes.c_double)),
        ("ridge_lambda_target", ctypes.c_double),
        ("gl_downgrade", ctypes.c_int),
        ("fp64_df", ctypes.c_int),
        ("defer_precompute", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("smoother", ctypes.c_int),
        ("smoother_sweep", ctypes.c_int),
        ("tc_split", ctypes.c_int),
    ]


_lib = None

# exported entry points and their ctypes signatures (the names of include/cr.h)
_SIGS = {
    "cr_last_error": ([], ctypes.c_char_p),
    "cr_plan_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(cr_params)], ctypes.c_int),
    "cr_plan_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "cr_plan_update_cl": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "cr_save": ([ctypes.c_void_p, ctypes.c_char_p], ctypes.c_int),
    "cr_plan_autotune": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "cr_tune_set": ([ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                     ctypes.c_int], ctypes.c_int),
    "cr_tune_entry": ([ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)],
                      ctypes.c_int),
    "cr_load": ([ctypes.c_void_p, ctypes.c_char_p], ctypes.c_int),
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
    "cr_launch_count": ([], ctypes.c_long),
    "cr_tc_selftest": ([ctypes.c_int, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "cr_plan_nlevels": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "cr_batch_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                         ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                         ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "cr_batch_run": ([ctypes.c_void_p], ctypes.c_int),
    "cr_batch_nodes": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
                       ctypes.c_int),
    "cr_batch_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "cr_grad_cl": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                    ctypes.c_double, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "cr_grad_ninv": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                      ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                      ctypes.c_int, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "cr_probe": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "cr_map_wdot": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)],
                    ctypes.c_int),
    "cr_alm_dot": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                    ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "cr_draw": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int],
                ctypes.c_int),
    "cr_plan_level_grid": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "cr_plan_level": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                       ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "cr_level_apply": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "cr_restrict": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "cr_prolong_add": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "cr_smooth": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "cr_pixel_smoother": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int],
                          ctypes.c_int),
    "cr_bottom_solve": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "cr_bottom_matrix": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)],
                         ctypes.c_int),
    "cr_wcycle": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "cr_solve": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                  ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                  ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "cr_plan_timing_exec": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "cr_tc_selftest_mn": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "cr_probe_fma_peak": ([ctypes.c_int, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "cr_plan_timing": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_char_p, ctypes.c_int,
                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_long),
                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
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


def tc_selftest(K=64):
    """Largest |difference| of a 128 x 32 x K tcgen05 BF16 tile against the CUDA cores (cr_tc_selftest)."""
    e = ctypes.c_float()
    _check(lib().cr_tc_selftest(int(K), ctypes.byref(e)))
    return e.value


def tc_selftest_mn(K=64, swap=0):
    """Largest |difference| of the MN-major tcgen05 tile against the CUDA
    cores (cr_tc_selftest_mn)."""
    e = ctypes.c_float()
    _check(lib().cr_tc_selftest_mn(int(K), int(swap), ctypes.byref(e)))
    return e.value


def fma_peak(kind):
    """Measured FMA-pipe peak in TFLOP/s on the current device: kind 'f32',
    'f32x2' (packed pairs) or 'f64' (cr_probe_fma_peak)."""
    k = {"f32": 0, "f32x2": 1, "f64": 2}[kind]
    t = ctypes.c_double()
    _check(lib().cr_probe_fma_peak(k, ctypes.byref(t)))
    return t.value


def launch_count():
    """Kernels launched by the library so far in this process."""
    return int(lib().cr_launch_count())


def tune_table():
    """The autotuner's cached choices: one dict per (grid, band limit,
    precision, stage).  Legendre stages (precision "f32"/"f64", stage
    "synthesis"/"adjoint"): the chosen pairs per thread and m tile (1: one m
    per CTA, 2: m and L - m per CTA) and the measured ms of 2, 4, 8 (and,
    for the FP32 adjoint, 16) pairs per thread with m tile 1 (``ms``) and 2
    (``ms_m_tile2``).  The batched tensor-core synthesis (precision "bf16",
    stage "tc_synthesis"): the chosen stage-shape variant (0: K 32 per
    parity, 2 stages; 1: K 32, 3 stages; 2: K 16, 3 stages) and the measured
    ms of each."""
    out = []
    i = 0
    while True:
        nring, lmax, nb, stage, rp, mt = (ctypes.c_int() for _ in range(6))
        npix = ctypes.c_int64()
        ms = (ctypes.c_double * 8)()
        if lib().cr_tune_entry(i, ctypes.byref(nring), ctypes.byref(npix), ctypes.byref(lmax), ctypes.byref(nb),
                               ctypes.byref(stage), ctypes.byref(rp), ctypes.byref(mt), ms) != 0:
            return out
        if nb.value == 2:
            out.append(dict(nring=nring.value, npix=npix.value, lmax=lmax.value, precision="bf16",
                            stage="tc_synthesis", variant=rp.value,
                            ms={k: ms[k] for k in range(3) if ms[k] >= 0}))
        else:
            out.append(dict(nring=nring.value, npix=npix.value, lmax=lmax.value,
                            precision="f64" if nb.value == 8 else "f32",
                            stage="synthesis" if stage.value == 0 else "adjoint", pairs_per_thread=rp.value,
                            m_tile=mt.value,
                            ms={k: ms[i2] for i2, k in enumerate((2, 4, 8, 16)) if ms[i2] >= 0},
                            ms_m_tile2={k: ms[4 + i2] for i2, k in enumerate((2, 4, 8, 16)) if ms[4 + i2] >= 0}))
        i += 1


def tune_set(nring, npix, lmax, precision, stage, pairs_per_thread, m_tile=1):
    """Pin one autotuner choice (``cr_tune_set``): precision "f32"/"f64" with
    stage "synthesis"/"adjoint", the pairs per thread and the m tile (1 or
    2), or precision "bf16" with stage "tc_synthesis" and the shape variant
    (0, 1, 2)."""
    nb = {"f64": 8, "f32": 4, "bf16": 2}[precision]
    st = {"synthesis": 0, "adjoint": 1, "tc_synthesis": 2}[stage]
    _check(lib().cr_tune_set(int(nring), int(npix), int(lmax), nb, st, int(pairs_per_thread), int(m_tile)))


def _tc_code(code, tensor_cores, what):
    if not tensor_cores:
        return code
    if code != CR_F32:
        raise TypeError("tensor-core %s takes complex64 / float32 data" % what)
    return CR_TC


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

    def __init__(self, lmax, nside=None, gl=None, cl=None, bl=None, ninv=None, stream=None, levels=None,
                 lmax_dense=-1, ridge_factor=0.0, ridge_bisections=0, ridge_alpha=None, ridge_lambda_target=0.0,
                 gl_downgrade=0, fp64_df=False, defer_precompute=False, autotune=False, smoother="icc",
                 smoother_sweep="auto", tc_split=False):
        """levels: None (transforms and A only), "default" (the library's level
        table), or a list of dicts with nside_h, lmax_h, n_rec and fl
        (cumulative filter, length lmax+1).  gl_downgrade: 0 auto, 1 every
        pixel level, -1 off (Gauss-Legendre grids for the levels'
        inverse-noise term).  defer_precompute: skip the C_l-dependent
        precompute (then ``load`` a checkpoint or ``update_cl``).
        smoother_sweep: "auto", "per_colour" or "cooperative" (how the ICC(0)
        triangular sweeps are launched; the same operator).  tc_split: the
        tensor-core contractions with hi + lo BF16 operands (three MMAs)."""
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
        if levels is None:
            p.nlevels = 0
        elif isinstance(levels, str) and levels == "default":
            p.nlevels = -1
        else:
            arr = (cr_level_spec * len(levels))()
            for i, lv in enumerate(levels):
                f = np.ascontiguousarray(lv["fl"], dtype=np.float64)
                self._keep.append(f)
                arr[i].nside_h = int(lv["nside_h"])
                arr[i].lmax_h = int(lv["lmax_h"])
                arr[i].n_rec = int(lv["n_rec"])
                arr[i].fl = f.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            self._keep.append(arr)
            p.nlevels = len(levels)
            p.levels = arr
        p.lmax_dense = int(lmax_dense)
        p.ridge_factor = float(ridge_factor)
        p.ridge_bisections = int(ridge_bisections)
        p.ridge_lambda_target = float(ridge_lambda_target)
        p.gl_downgrade = int(gl_downgrade)
        p.fp64_df = int(bool(fp64_df))
        p.defer_precompute = int(bool(defer_precompute))
        p.autotune = int(bool(autotune))
        if smoother not in ("icc", "schwarz"):
            raise ValueError("smoother: 'icc' (multicolour block ICC(0)) or 'schwarz' (block Jacobi)")
        p.smoother = 0 if smoother == "icc" else 1
        p.smoother_sweep = {"auto": 0, "per_colour": 1, "cooperative": 2}[smoother_sweep]
        p.tc_split = int(bool(tc_split))
        if ridge_alpha is not None:
            ra = np.ascontiguousarray(ridge_alpha, dtype=np.float64)
            self._keep.append(ra)
            p.ridge_alpha = ra.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        h = ctypes.c_void_p()
        _check(lib().cr_plan_create(ctypes.byref(h), ctypes.byref(p)))
        self._h = h
        self.lmax = int(lmax)
        self._keep = []
        self.npix = self.sizes()["npix"]

    def autotune(self):
        """Time the Legendre kernels' ring-block choices on this plan's grids
        and keep the fastest (``cr_plan_autotune``); returns tune_table()."""
        n = ctypes.c_int()
        _check(lib().cr_plan_autotune(self._h, ctypes.byref(n)))
        return tune_table()

    def update_cl(self, cl):
        """Replace the prior C_l and redo the C_l-dependent precompute
        (``cr_plan_update_cl``)."""
        cl = np.ascontiguousarray(cl, dtype=np.float64)
        if cl.shape != (self.lmax + 1,):
            raise ValueError("update_cl: C_l must have lmax + 1 entries")
        _check(lib().cr_plan_update_cl(self._h, cl.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def save(self, path):
        """Write the precompute checkpoint (``cr_save``)."""
        _check(lib().cr_save(self._h, os.fsencode(path)))

    def load(self, path):
        """Read a precompute checkpoint made for the same inputs (``cr_load``)."""
        _check(lib().cr_load(self._h, os.fsencode(path)))

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

    def sht_synth(self, alm, out, grid=CR_OBS, tensor_cores=False):
        """map = Y alm for every right-hand side; tensor_cores=True (complex64
        / float32 data): batched Legendre contraction on the tensor cores
        (CR_TC, BF16 operands, FP32 accumulation)."""
        s = self.sizes(grid)
        nrhs = self._nrhs(alm, s["nlm"])
        if out.numel() != nrhs * s["npix"] or _dtype_code(alm) != _dtype_code(out):
            raise ValueError("sht_synth: output shape/dtype")
        code = _dtype_code(alm)
        code = _tc_code(code, tensor_cores, "synthesis")
        _check(lib().cr_sht_synth(self._h, grid, _dev(alm), _dev(out), nrhs, code))
        return out

    def sht_adjoint(self, map_, out, grid=CR_OBS, tensor_cores=False):
        """alm = Y^T map for every right-hand side; tensor_cores=True (float32
        / complex64 data): batched Legendre contraction on the tensor cores
        (CR_TC)."""
        s = self.sizes(grid)
        nrhs = self._nrhs(map_, s["npix"])
        if out.numel() != nrhs * s["nlm"] or _dtype_code(map_) != _dtype_code(out):
            raise ValueError("sht_adjoint: output shape/dtype")
        code = _tc_code(_dtype_code(map_), tensor_cores, "adjoint")
        _check(lib().cr_sht_adjoint(self._h, grid, _dev(map_), _dev(out), nrhs, code))
        return out

    def set_timing(self, enable=True):
        _check(lib().cr_plan_set_timing(self._h, 1 if enable else 0))

    def timing(self):
        """{stage name: (total ms, scopes, algorithmic work)} since timing was
        enabled."""
        cnt = ctypes.c_int()
        _check(lib().cr_plan_timing(self._h, -1, None, 0, None, None, None, ctypes.byref(cnt)))
        out = {}
        for i in range(cnt.value):
            buf = ctypes.create_string_buffer(64)
            ms, n, w = ctypes.c_double(), ctypes.c_long(), ctypes.c_double()
            _check(lib().cr_plan_timing(self._h, i, buf, 64, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(w),
                                        None))
            out[buf.value.decode()] = (ms.value, n.value, w.value)
        return out

    def timing_exec(self):
        """{stage name: executed work} since timing was enabled: for the
        Legendre stages the flops of the terms past the start tables."""
        cnt = ctypes.c_int()
        _check(lib().cr_plan_timing(self._h, -1, None, 0, None, None, None, ctypes.byref(cnt)))
        out = {}
        for i in range(cnt.value):
            buf = ctypes.create_string_buffer(64)
            w = ctypes.c_double()
            _check(lib().cr_plan_timing(self._h, i, buf, 64, None, None, None, None))
            _check(lib().cr_plan_timing_exec(self._h, i, ctypes.byref(w)))
            out[buf.value.decode()] = w.value
        return out

    # ---- multi-level solver -------------------------------------------------
    def nlevels(self):
        h = ctypes.c_int()
        _check(lib().cr_plan_nlevels(self._h, ctypes.byref(h)))
        return h.value

    def level(self, h):
        """dict(nside_h, lmax_h, n_rec, fl, ridge) of level h (0 = top,
        1..H pixel levels, H+1 bottom)."""
        ns, lm, nr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        fl = np.zeros(self.lmax + 1)
        ridge, lam = ctypes.c_double(), ctypes.c_double()
        _check(lib().cr_plan_level(self._h, h, ctypes.byref(ns), ctypes.byref(lm), ctypes.byref(nr),
                                   fl.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(ridge),
                                   ctypes.byref(lam)))
        return dict(nside_h=ns.value, lmax_h=lm.value, n_rec=nr.value, fl=fl, ridge=ridge.value, lambda_max=lam.value)

    def draw(self, seed, b, d=None, fluct=True, plain=False):
        """Right-hand side b = B Y^T N^-1 d (+ S^-1/2 w1 + B Y^T N^-1/2 w2 with
        fluct) for every right-hand side j of b ([nrhs, N_lm] complex128);
        d: float64 CUDA map(s) [nrhs, npix] or None."""
        nrhs = self._nrhs(b, n_lm(self.lmax))
        if d is not None and not (d.is_cuda and d.dtype == torch.float64):
            raise ValueError("d must be a float64 CUDA tensor")
        _check(lib().cr_draw(self._h, int(seed) & 0xFFFFFFFFFFFFFFFF, None if d is None else _dev(d), _dev(b), nrhs,
                             (CR_DRAW_FLUCT if fluct else 0) | (CR_DRAW_PLAIN if plain else 0)))
        return b

    def grad_cl(self, u, v, alpha, beta, seed=0, rhs=0, out=None, kappa=0.0, accumulate=False):
        """out[l] (+)= alpha C_l^-2 <u, v>_l + beta C_l^-3/2 <u, w1>_l + kappa (2l+1)/C_l (cr_grad_cl)."""
        if out is None:
            out = torch.empty(self.lmax + 1, dtype=torch.float64, device=u.device)
        _check(lib().cr_grad_cl(self._h, _dev(u), None if v is None else _dev(v), float(alpha), float(beta),
                                float(kappa), int(seed) & 0xFFFFFFFFFFFFFFFF, int(rhs), int(bool(accumulate)),
                                _dev(out)))
        return out

    def grad_ninv(self, u, v, d, alpha, gamma, delta, eps, seed=0, rhs=0, out=None, kappa=0.0, accumulate=False):
        """out_i (+)= alpha p_i q_i + p_i (gamma d_i + delta w2_i / sqrt n_i) + eps d_i^2 + kappa / n_i,
        p = Y B u, q = Y B v (cr_grad_ninv)."""
        if out is None:
            out = torch.empty(self.npix, dtype=torch.float64, device=u.device)
        _check(lib().cr_grad_ninv(self._h, _dev(u), None if v is None else _dev(v), None if d is None else _dev(d),
                                  float(alpha), float(gamma), float(delta), float(eps), float(kappa),
                                  int(seed) & 0xFFFFFFFFFFFFFFFF, int(rhs), int(bool(accumulate)), _dev(out)))
        return out

    def probe(self, seed, kind, j, out):
        """Rademacher probe j (cr_probe): kind CR_PROBE_ALM -> complex [N_lm], CR_PROBE_MAP -> map [npix]."""
        _check(lib().cr_probe(self._h, int(seed) & 0xFFFFFFFFFFFFFFFF, int(kind), int(j), _dev(out)))
        return out

    def map_wdot(self, a, b):
        out = ctypes.c_double()
        _check(lib().cr_map_wdot(self._h, _dev(a), _dev(b), ctypes.byref(out)))
        return out.value

    def alm_dot(self, u, v, weighted=False):
        out = ctypes.c_double()
        _check(lib().cr_alm_dot(self._h, _dev(u), _dev(v), int(bool(weighted)), ctypes.byref(out)))
        return out.value

    def level_grid(self, h):
        """(kind, nring, npix) of the grid on which pixel level h applies its
        inverse-noise term: kind "healpix" (observation grid) or "gl"."""
        k, nr, npx = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        _check(lib().cr_plan_level_grid(self._h, h, ctypes.byref(k), ctypes.byref(nr), ctypes.byref(npx)))
        return ("gl" if k.value == CR_GRID_GL else "healpix", nr.value, npx.value)

    def level_apply(self, h, x, out):
        _check(lib().cr_level_apply(self._h, h, _dev(x), _dev(out), _dtype_code(x)))
        return out

    def restrict(self, h, r, out):
        _check(lib().cr_restrict(self._h, h, _dev(r), _dev(out), _dtype_code(r)))
        return out

    def prolong_add(self, h, c, x):
        _check(lib().cr_prolong_add(self._h, h, _dev(c), _dev(x), _dtype_code(c)))
        return x

    def smooth(self, h, r, out):
        _check(lib().cr_smooth(self._h, h, _dev(r), _dev(out), _dtype_code(r)))
        return out

    def pixel_smoother(self, h, maps, out):
        """out = M_h maps (``cr_pixel_smoother``): the pixel-space smoother
        of level h on 1-16 maps [nrhs][12 nside_h^2] (RING order)."""
        nrhs = 1 if maps.dim() == 1 else maps.shape[0]
        _check(lib().cr_pixel_smoother(self._h, h, _dev(maps), _dev(out), nrhs, _dtype_code(maps)))
        return out

    def bottom_solve(self, b, out):
        _check(lib().cr_bottom_solve(self._h, _dev(b), _dev(out), _dtype_code(b)))
        return out

    def bottom_matrix(self):
        nd = ctypes.c_int()
        _check(lib().cr_bottom_matrix(self._h, None, ctypes.byref(nd)))
        out = np.zeros((nd.value, nd.value))
        _check(lib().cr_bottom_matrix(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(nd)))
        return out

    def wcycle(self, x, b):
        nrhs = self._nrhs(b, n_lm(self.lmax))
        _check(lib().cr_wcycle(self._h, _dev(x), _dev(b), nrhs, _dtype_code(b)))
        return x

    def solve(self, b, x, eps=1e-12, max_cycles=30, mode=CR_F64, check=True):
        """CR-Solve.  Returns (cycles, relres, history) per right-hand side;
        with check=False a CR_EDIVERGED / CR_EMAXITER status is returned as
        the 4th element instead of raising."""
        nrhs = self._nrhs(b, n_lm(self.lmax))
        cyc = (ctypes.c_int * nrhs)()
        rel = (ctypes.c_double * nrhs)()
        hist = np.zeros((nrhs, max_cycles))
        rc = lib().cr_solve(self._h, _dev(x), _dev(b), nrhs, float(eps), int(max_cycles), int(mode), cyc, rel,
                            hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if check:
            _check(rc)
        out = (list(cyc), list(rel), hist)
        return out if check else out + (rc,)

    def apply_A(self, x, out, level=0, tensor_cores=False):
        """out = A x; tensor_cores=True (level 0, complex64): both Legendre
        stages of every 16 right-hand sides on the tensor cores (CR_TC)."""
        nrhs = self._nrhs(x, n_lm(self.lmax)) if level == 0 else x.numel() // max(1, out.numel())
        if tensor_cores and level != 0:
            raise ValueError("apply_A: tensor cores at level 0 only")
        code = _tc_code(_dtype_code(x), tensor_cores, "apply_A")
        _check(lib().cr_apply_A(self._h, level, _dev(x), _dev(out), nrhs, code))
        return out


class Batch:
    """Fixed-count CR-Solves of many right-hand sides over one or more plans
    (mixed resolutions) captured into one CUDA graph (cr_batch_create);
    run() replays it with a single launch."""

    def __init__(self, plans, xs, bs, cycles, mode=CR_MIXED):
        n = len(plans)
        hp = (ctypes.c_void_p * n)(*[p._h.value for p in plans])
        xp = (ctypes.c_void_p * n)(*[_dev(x).value for x in xs])
        bp = (ctypes.c_void_p * n)(*[_dev(b).value for b in bs])
        nr = (ctypes.c_int * n)(*[p._nrhs(b, n_lm(p.lmax)) for p, b in zip(plans, bs)])
        h = ctypes.c_void_p()
        _check(lib().cr_batch_create(ctypes.byref(h), n, hp, xp, bp, nr, int(cycles), int(mode)))
        self._h = h
        self._keep = (plans, xs, bs)

    def run(self):
        _check(lib().cr_batch_run(self._h))

    def nodes(self):
        n = ctypes.c_int64()
        _check(lib().cr_batch_nodes(self._h, ctypes.byref(n), None))
        return n.value

    def kernel_nodes(self):
        k = ctypes.c_int64()
        _check(lib().cr_batch_nodes(self._h, None, ctypes.byref(k)))
        return k.value

    def close(self):
        if getattr(self, "_h", None):
            lib().cr_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
