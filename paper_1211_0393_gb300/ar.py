"""ctypes binding of ``libar.so``: the C ABI of ``include/ar.h`` under the same names.

Argument marshalling only: every function checks tensor placement, dtype and
shape, passes raw pointers and the current CUDA stream, and turns a non-zero
``ar_status`` into :class:`ARError`.  All arithmetic happens in the library's
CUDA kernels.  Importing this module on a machine without the built library
raises immediately; there is no fallback.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libar.so")

STATUS = {
    0: "AR_OK", 1: "AR_ERR_INVALID_ARG", 2: "AR_ERR_ALIAS", 3: "AR_ERR_PSF_NOT_NORMALIZED",
    4: "AR_ERR_ALLOC", 5: "AR_ERR_CUDA", 6: "AR_ERR_NONFINITE", 7: "AR_ERR_TIMEOUT",
    8: "AR_ERR_UNSUPPORTED",
}

EXPORTS = [
    "ar_blur_apply", "ar_reblur_apply", "ar_symprec_setup", "ar_symprec_solve",
    "ar_symprec_eigenvalues", "ar_symprec_shape", "ar_symprec_destroy", "ar_restore",
    "ar_status_string", "ar_last_error_detail", "ar_version", "ar_kernel_launches",
    "ar_profile_begin", "ar_profile_end", "ar_restore_plain_static", "ar_symprec_setup_ex",
    "ar_restore_ex", "ar_batch_create", "ar_batch_run", "ar_batch_results", "ar_batch_destroy",
    "ar_blur_apply_bc", "ar_reblur_apply_bc", "ar_symprec_setup_bc", "ar_restore_bc",
    "ar_corr_param_count", "ar_corr_create", "ar_corr_params", "ar_corr_destroy",
    "ar_corr_targets", "ar_corr_train", "ar_corr_predict", "ar_symprec_setup_corrected",
    "ar_restore_prec", "ar_restore_residuals", "ar_set_stencil_wait_polls",
    "ar_inject_alloc_failures", "ar_corr_train_tables", "ar_corr_restoration_targets",
    "ar_batch_tuning", "ar_symprec_precision", "ar_blur_apply_ex", "ar_reblur_apply_ex",
]

DEFAULT_WAIT_POLLS = 1 << 24

CORR_GRID = 33      # the correction model's delta table is CORR_GRID x CORR_GRID


class BatchItem(ctypes.Structure):
    """Mirror of ``ar_batch_item``."""
    _fields_ = [("g", ctypes.c_void_p), ("psf_host", ctypes.c_void_p), ("n1", ctypes.c_int),
                ("n2", ctypes.c_int), ("q1", ctypes.c_int), ("q2", ctypes.c_int),
                ("alpha", ctypes.c_double), ("f_true", ctypes.c_void_p), ("x_out", ctypes.c_void_p)]

PRECISION = {"fp32": 0, "bf16x2": 1, "fft": 2, "auto": 3}
PRECISION_NAME = {v: k for k, v in PRECISION.items()}

# stencil arithmetic (ar.h AR_STENCIL_*): float32 FMAs, tensor-core fp16 split, or
# the faster of the two for the shape (measured once)
STENCIL = {"fp32": 0, "f16x2": 16, "auto": 32}

# ar_bc: the method's anti-reflective BCs and the two comparison BCs
BC = {"ar": 0, "reflective": 1, "periodic": 2}

PROF_KINDS = ("stencil", "contraction", "setup", "other")


class ARError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        self.name = STATUS.get(status, f"AR_UNKNOWN({status})")
        super().__init__(f"{where}: {self.name}: {detail}")


_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double


def lib() -> ctypes.CDLL:
    """Load ``libar.so`` once; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        sig = {
            "ar_blur_apply": [_vp, _vp, _i, _i, _vp, _i, _i, _vp],
            "ar_reblur_apply": [_vp, _vp, _i, _i, _vp, _i, _i, _vp],
            "ar_blur_apply_bc": [_vp, _vp, _i, _i, _vp, _i, _i, _i, _vp],
            "ar_reblur_apply_bc": [_vp, _vp, _i, _i, _vp, _i, _i, _i, _vp],
            "ar_blur_apply_ex": [_vp, _vp, _i, _i, _vp, _i, _i, _i, _i, _vp],
            "ar_reblur_apply_ex": [_vp, _vp, _i, _i, _vp, _i, _i, _i, _i, _vp],
            "ar_symprec_setup_bc": [_vp, _i, _i, _i, _i, _d, _i, _i, _vp, ctypes.POINTER(_vp)],
            "ar_restore_bc": [_vp, _vp, _i, _i, _i, _i, _d, _d, _i, _i, _i, _i, _vp, _vp, _vp, _vp,
                              _vp, _vp],
            "ar_restore_residuals": [_vp, _vp, _i, _i, _i, _i, _d, _d, _i, _i, _i, _i, _vp, _vp, _vp,
                                     _vp, _vp, _vp, _vp],
            "ar_symprec_setup": [_vp, _i, _i, _i, _i, _d, _vp, ctypes.POINTER(_vp)],
            "ar_symprec_setup_ex": [_vp, _i, _i, _i, _i, _d, _i, _vp, ctypes.POINTER(_vp)],
            "ar_restore_ex": [_vp, _vp, _i, _i, _i, _i, _d, _d, _i, _i, _i, _vp, _vp, _vp, _vp, _vp,
                              _vp],
            "ar_symprec_solve": [_vp, _vp, _vp, _vp],
            "ar_symprec_eigenvalues": [_vp, _vp, _vp],
            "ar_symprec_shape": [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i)],
            "ar_restore": [_vp, _vp, _i, _i, _i, _i, _d, _d, _i, _i, _vp, _vp, _vp, _vp, _vp, _vp],
            "ar_restore_plain_static": [_vp, _vp, _i, _i, _i, _i, _d, _i, _vp, _vp, _vp, _vp, _vp,
                                        _vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = _i
        L.ar_symprec_destroy.argtypes = [_vp]
        L.ar_symprec_destroy.restype = None
        for name in ("ar_status_string",):
            getattr(L, name).argtypes = [_i]
            getattr(L, name).restype = ctypes.c_char_p
        for name in ("ar_last_error_detail", "ar_version"):
            getattr(L, name).argtypes = []
            getattr(L, name).restype = ctypes.c_char_p
        L.ar_batch_create.argtypes = [_vp, _i, _d, _i, _i, _i, _i, _vp, ctypes.POINTER(_vp)]
        L.ar_batch_create.restype = _i
        L.ar_batch_run.argtypes = [_vp, _vp]
        L.ar_batch_run.restype = _i
        L.ar_batch_results.argtypes = [_vp, _vp, _vp, _vp]
        L.ar_batch_results.restype = _i
        L.ar_symprec_precision.argtypes = [_vp, ctypes.POINTER(_i)]
        L.ar_symprec_precision.restype = _i
        L.ar_batch_tuning.argtypes = [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i),
                                      ctypes.POINTER(_i), ctypes.POINTER(_i), _vp, _vp, _vp, _i]
        L.ar_batch_tuning.restype = _i
        L.ar_batch_destroy.argtypes = [_vp]
        L.ar_batch_destroy.restype = None
        L.ar_set_stencil_wait_polls.argtypes = [ctypes.c_uint]
        L.ar_set_stencil_wait_polls.restype = _i
        L.ar_inject_alloc_failures.argtypes = [_i, _i]
        L.ar_inject_alloc_failures.restype = None
        L.ar_profile_begin.argtypes = []
        L.ar_profile_begin.restype = _i
        L.ar_profile_end.argtypes = [_vp, _vp, _i]
        L.ar_profile_end.restype = _i
        L.ar_kernel_launches.argtypes = []
        L.ar_kernel_launches.restype = ctypes.c_ulonglong
        L.ar_corr_param_count.argtypes = []
        L.ar_corr_param_count.restype = ctypes.c_size_t
        for name, args in {
            "ar_corr_create": [_vp, ctypes.POINTER(_vp)],
            "ar_corr_params": [_vp, _vp],
            "ar_corr_targets": [_vp, _i, _vp],
            "ar_corr_train": [_vp, _vp, _i, _i, _i, _d, _vp, _vp],
            "ar_corr_train_tables": [_vp, _vp, _vp, _i, _i, _i, _d, _vp, _vp],
            "ar_corr_restoration_targets": [_vp, _vp, _i, _i, _vp, _i, _d, _d, _d, _i, _vp, _vp],
            "ar_corr_predict": [_vp, _vp, _vp],
            "ar_symprec_setup_corrected": [_vp, _i, _i, _i, _i, _d, _vp, _i, _vp,
                                           ctypes.POINTER(_vp)],
            "ar_restore_prec": [_vp, _vp, _vp, _d, _i, _vp, _vp, _vp, _vp, _vp, _vp],
        }.items():
            getattr(L, name).argtypes = args
            getattr(L, name).restype = _i
        L.ar_corr_destroy.argtypes = [_vp]
        L.ar_corr_destroy.restype = None
        _lib = L
    return _lib


def _check(status: int, where: str) -> None:
    if status != 0:
        raise ARError(status, where, lib().ar_last_error_detail().decode())


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _image(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or t.dim() != 2:
        raise TypeError(f"{name} must be a 2D float32 CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _support(psf_shape) -> tuple[int, int]:
    k1, k2 = psf_shape
    if k1 % 2 == 0 or k2 % 2 == 0:
        raise ValueError("PSF sides must be odd")
    return (k1 - 1) // 2, (k2 - 1) // 2


def _host_psf(psf) -> np.ndarray:
    h = psf.detach().cpu().numpy() if isinstance(psf, torch.Tensor) else np.asarray(psf)
    return np.ascontiguousarray(h, dtype=np.float64)


def ar_blur_apply(x: torch.Tensor, psf: torch.Tensor, y: torch.Tensor | None = None,
                  stream=None, bc: str = "ar", stencil: str = "fp32") -> torch.Tensor:
    """``y = A_n x`` (blur under ``bc``: "ar", "reflective" or "periodic").

    ``psf`` is a float32 CUDA tensor of odd sides; ``stencil`` "fp32" (CUDA-core
    FMAs), "f16x2" (tensor cores, two-plane fp16 split, where it applies) or "auto"
    (the faster of the two for the shape, measured the first time)."""
    return _apply("ar_blur_apply", x, psf, y, stream, bc, stencil)


def ar_reblur_apply(x: torch.Tensor, psf: torch.Tensor, y: torch.Tensor | None = None,
                    stream=None, bc: str = "ar", stencil: str = "fp32") -> torch.Tensor:
    """``y = A' x`` (the blur under ``bc`` with the PSF rotated by 180 degrees)."""
    return _apply("ar_reblur_apply", x, psf, y, stream, bc, stencil)


def _apply(name, x, psf, y, stream, bc="ar", stencil="fp32"):
    _image(x, "x")
    if not isinstance(psf, torch.Tensor) or not psf.is_cuda or psf.dtype != torch.float32:
        raise TypeError("psf must be a float32 CUDA tensor")
    psf = psf.contiguous()
    q1, q2 = _support(psf.shape)
    if y is None:
        y = torch.empty_like(x)
    _image(y, "y")
    if y.shape != x.shape:
        raise ValueError("y must have the shape of x")
    n1, n2 = x.shape
    if stencil != "fp32":
        name += "_ex"
        _check(getattr(lib(), name)(x.data_ptr(), y.data_ptr(), n1, n2, psf.data_ptr(), q1, q2,
                                    BC[bc], STENCIL[stencil], _stream(stream)), name)
    elif bc == "ar":
        _check(getattr(lib(), name)(x.data_ptr(), y.data_ptr(), n1, n2, psf.data_ptr(), q1, q2,
                                    _stream(stream)), name)
    else:
        name += "_bc"
        _check(getattr(lib(), name)(x.data_ptr(), y.data_ptr(), n1, n2, psf.data_ptr(), q1, q2,
                                    BC[bc], _stream(stream)), name)
    return y


class Prec:
    """Owner of an ``ar_prec*`` (freed with ``ar_symprec_destroy``)."""

    def __init__(self, handle: int, n1: int, n2: int):
        self.handle = handle
        self.shape = (n1, n2)

    def close(self) -> None:
        if self.handle:
            lib().ar_symprec_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ar_symprec_setup(psf, n1: int, n2: int, alpha: float, stream=None,
                     precision: str = "fp32", bc: str = "ar") -> Prec:
    """Build the optimal preconditioner of ``bc`` (float64 setup on the GPU).

    ``precision``: "fp32" (three bf16 planes, six products), "bf16x2" (two
    planes, three products) for the transform contractions, "fft" (the
    FFT-style float32 transform, AR only) or "auto" (the faster of "fft" and
    "fp32" for the size, measured once).  ``bc``: "ar"
    (symmetrized PSF, AR transform), "reflective" (symmetrized PSF, DCT-III)
    or "periodic" (circulant of the PSF)."""
    h = _host_psf(psf)
    q1, q2 = _support(h.shape)
    out = _vp()
    _check(lib().ar_symprec_setup_bc(h.ctypes.data, q1, q2, n1, n2, float(alpha), BC[bc],
                                     PRECISION[precision], _stream(stream), ctypes.byref(out)),
           "ar_symprec_setup_bc")
    return Prec(out.value, n1, n2)


def ar_symprec_solve(P: Prec, y: torch.Tensor, z: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
    """``z = D y = T diag(d) T~ y``."""
    _image(y, "y")
    if tuple(y.shape) != P.shape:
        raise ValueError(f"y has shape {tuple(y.shape)}, preconditioner expects {P.shape}")
    if z is None:
        z = torch.empty_like(y)
    _image(z, "z")
    _check(lib().ar_symprec_solve(P.handle, y.data_ptr(), z.data_ptr(), _stream(stream)),
           "ar_symprec_solve")
    return z


def ar_symprec_eigenvalues(P: Prec) -> tuple[np.ndarray, np.ndarray]:
    """Float64 ``(lambda, d)`` of the preconditioner, copied to the host."""
    lam = np.empty(P.shape, dtype=np.float64)
    d = np.empty(P.shape, dtype=np.float64)
    _check(lib().ar_symprec_eigenvalues(P.handle, lam.ctypes.data, d.ctypes.data),
           "ar_symprec_eigenvalues")
    return lam, d


def ar_symprec_precision(P: Prec) -> str:
    """The transform arithmetic P runs with ("fp32", "bf16x2" or "fft"; the choice
    of "auto")."""
    v = _i()
    _check(lib().ar_symprec_precision(P.handle, ctypes.byref(v)), "ar_symprec_precision")
    return PRECISION_NAME[v.value]


def ar_symprec_shape(P: Prec) -> tuple[int, int]:
    a, b = _i(), _i()
    _check(lib().ar_symprec_shape(P.handle, ctypes.byref(a), ctypes.byref(b)), "ar_symprec_shape")
    return a.value, b.value


def ar_restore(g: torch.Tensor, psf, alpha: float, tau: float = 1.0, iters: int = 20,
               precondition: bool = True, x0: torch.Tensor | None = None,
               f_true: torch.Tensor | None = None, x_out: torch.Tensor | None = None,
               trace: bool = True, stream=None, precision: str = "fp32", bc: str = "ar",
               stencil: str = "fp32"):
    """(D-)Landweber restoration under ``bc``; ``stencil`` as ``ar_blur_apply``.

    Returns ``(x, rre_trace or None, best_iter or None)``."""
    _image(g, "g")
    h = _host_psf(psf)
    q1, q2 = _support(h.shape)
    n1, n2 = g.shape
    if x_out is None:
        x_out = torch.empty_like(g)
    _image(x_out, "x_out")
    want = f_true is not None and trace
    tr = np.zeros(max(iters, 1), dtype=np.float64) if want else None
    best = _i(0)
    _check(lib().ar_restore_bc(
        g.data_ptr(), h.ctypes.data, n1, n2, q1, q2, float(alpha), float(tau), int(iters),
        BC[bc], 1 if precondition else 0, PRECISION[precision] | STENCIL[stencil],
        _image(x0, "x0").data_ptr() if x0 is not None else None,
        _image(f_true, "f_true").data_ptr() if f_true is not None else None,
        x_out.data_ptr(),
        tr.ctypes.data if want else None,
        ctypes.addressof(best) if want else None,
        _stream(stream)), "ar_restore")
    return x_out, (tr[:iters] if want else None), (best.value if want else None)


def ar_restore_residuals(g: torch.Tensor, psf, alpha: float, tau: float = 1.0, iters: int = 20,
                         precondition: bool = True, x0: torch.Tensor | None = None,
                         f_true: torch.Tensor | None = None, x_out: torch.Tensor | None = None,
                         stream=None, precision: str = "fp32", bc: str = "ar",
                         stencil: str = "fp32"):
    """``ar_restore`` that also returns the residual norms ``||g - A x_k||_F`` of the
    iterates, k = 0 .. iters.

    Returns ``(x, rre_trace or None, best_iter or None, residual_norms)``."""
    _image(g, "g")
    h = _host_psf(psf)
    q1, q2 = _support(h.shape)
    n1, n2 = g.shape
    if x_out is None:
        x_out = torch.empty_like(g)
    _image(x_out, "x_out")
    want = f_true is not None
    tr = np.zeros(max(iters, 1), dtype=np.float64) if want else None
    res = np.zeros(iters + 1, dtype=np.float64)
    best = _i(0)
    _check(lib().ar_restore_residuals(
        g.data_ptr(), h.ctypes.data, n1, n2, q1, q2, float(alpha), float(tau), int(iters),
        BC[bc], 1 if precondition else 0, PRECISION[precision] | STENCIL[stencil],
        _image(x0, "x0").data_ptr() if x0 is not None else None,
        _image(f_true, "f_true").data_ptr() if f_true is not None else None,
        x_out.data_ptr(),
        tr.ctypes.data if want else None,
        ctypes.addressof(best) if want else None,
        res.ctypes.data,
        _stream(stream)), "ar_restore_residuals")
    return x_out, (tr[:iters] if want else None), (best.value if want else None), res


def ar_profile_begin() -> None:
    """Start per-kernel-class event timing (see ``ar_profile_end``)."""
    _check(lib().ar_profile_begin(), "ar_profile_begin")


def ar_profile_end() -> dict:
    """Stop timing; returns ``{class: (milliseconds, launches)}``."""
    n = len(PROF_KINDS)
    ms = np.zeros(n, dtype=np.float64)
    cnt = np.zeros(n, dtype=np.uint64)
    _check(lib().ar_profile_end(ms.ctypes.data, cnt.ctypes.data, n), "ar_profile_end")
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(PROF_KINDS)}


def ar_restore_plain_static(g: torch.Tensor, psf, tau: float = 1.0, iters: int = 20,
                            x0: torch.Tensor | None = None, f_true: torch.Tensor | None = None,
                            x_out: torch.Tensor | None = None, trace: bool = True, stream=None):
    """Plain Landweber restoration with no memory allocated by the library.

    Same result as ``ar_restore(..., precondition=False)``; the library's scratch
    is a static device array (see ``include/ar.h`` for the size limits).  The
    caller provides ``x_out`` (allocated here only when omitted).
    """
    _image(g, "g")
    h = _host_psf(psf)
    q1, q2 = _support(h.shape)
    n1, n2 = g.shape
    if x_out is None:
        x_out = torch.empty_like(g)
    _image(x_out, "x_out")
    want = f_true is not None and trace
    tr = np.zeros(max(iters, 1), dtype=np.float64) if want else None
    best = _i(0)
    _check(lib().ar_restore_plain_static(
        g.data_ptr(), h.ctypes.data, n1, n2, q1, q2, float(tau), int(iters),
        _image(x0, "x0").data_ptr() if x0 is not None else None,
        _image(f_true, "f_true").data_ptr() if f_true is not None else None,
        x_out.data_ptr(),
        tr.ctypes.data if want else None,
        ctypes.addressof(best) if want else None,
        _stream(stream)), "ar_restore_plain_static")
    return x_out, (tr[:iters] if want else None), (best.value if want else None)


class Batch:
    """Owner of an ``ar_batch*``: many images restored by one CUDA-graph launch.

    ``images`` is a list of dicts with keys g, psf, alpha, x_out and optional
    f_true (device float32 tensors; psf a host array).  The tensors must stay
    alive while the batch exists."""

    def __init__(self, images, tau=1.0, iters=50, precondition=True, precision="fp32",
                 tuning=0, stream=None):
        self.count = len(images)
        self.iters = int(iters)
        self._keep = []
        arr = (BatchItem * self.count)()
        for j, im in enumerate(images):
            g = _image(im["g"], "g")
            x = _image(im["x_out"], "x_out")
            h = _host_psf(im["psf"])
            q1, q2 = _support(h.shape)
            f = im.get("f_true")
            self._keep += [g, x, h, f]
            arr[j] = BatchItem(g.data_ptr(), h.ctypes.data, g.shape[0], g.shape[1], q1, q2,
                               float(im.get("alpha", 0.0)),
                               _image(f, "f_true").data_ptr() if f is not None else None,
                               x.data_ptr())
        self._items = arr
        out = _vp()
        _check(lib().ar_batch_create(arr, self.count, float(tau), self.iters,
                                     1 if precondition else 0, PRECISION[precision],
                                     int(tuning), _stream(stream), ctypes.byref(out)),
               "ar_batch_create")
        self.handle = out.value

    def run(self, stream=None) -> None:
        _check(lib().ar_batch_run(self.handle, _stream(stream)), "ar_batch_run")

    def results(self):
        """(rre traces [count, iters], best iterations [count], kernels per run)."""
        tr = np.zeros((self.count, max(self.iters, 1)), dtype=np.float64)
        best = np.zeros(self.count, dtype=np.int32)
        kpr = ctypes.c_ulonglong(0)
        _check(lib().ar_batch_results(self.handle, tr.ctypes.data, best.ctypes.data,
                                      ctypes.byref(kpr)), "ar_batch_results")
        return tr[:, :self.iters], best, int(kpr.value)

    def tuning(self) -> dict:
        """The stencil configuration in use and the autotuner's timed candidates."""
        geo, ctas, tf, n = _i(), _i(), _i(), _i()
        cg = np.zeros(16, dtype=np.int32)
        cc = np.zeros(16, dtype=np.int32)
        cm = np.zeros(16, dtype=np.float64)
        _check(lib().ar_batch_tuning(self.handle, ctypes.byref(geo), ctypes.byref(ctas),
                                     ctypes.byref(tf), ctypes.byref(n), cg.ctypes.data,
                                     cc.ctypes.data, cm.ctypes.data, 16), "ar_batch_tuning")
        k = min(n.value, 16)
        return {"geometry": ("64-row", "54-row")[geo.value], "ctas_per_sm": ctas.value,
                "folded_input": bool(tf.value & 1), "paired_last_product": bool(tf.value & 2),
                "candidates": [{"geometry": ("64-row", "54-row")[int(cg[i])],
                                "ctas_per_sm": int(cc[i]), "ms_3_iters": float(cm[i])}
                               for i in range(k)]}

    def close(self) -> None:
        if self.handle:
            lib().ar_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Corr:
    """Owner of an ``ar_corr*``: the MLP that predicts the spectral correction
    delta (33 x 33 table) from the antisymmetric part of a 15 x 15 PSF."""

    def __init__(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != param_count():
            raise ValueError(f"expected {param_count()} parameters, got {p.size}")
        out = _vp()
        _check(lib().ar_corr_create(p.ctypes.data, ctypes.byref(out)), "ar_corr_create")
        self.handle = out.value

    def params(self) -> np.ndarray:
        p = np.empty(param_count(), dtype=np.float32)
        _check(lib().ar_corr_params(self.handle, p.ctypes.data), "ar_corr_params")
        return p

    def train(self, psfs, epochs: int, batch: int, lr: float, stream=None,
              tables=None) -> np.ndarray:
        """Adam on the mean squared error of the delta tables; returns the loss per epoch.

        ``tables`` (count x 33 x 33) replaces the closed-form targets, e.g. with
        those of :func:`corr_restoration_targets`."""
        h = np.ascontiguousarray(psfs, dtype=np.float64).reshape(-1, 225)
        tr = np.zeros(max(int(epochs), 1), dtype=np.float32)
        if tables is None:
            _check(lib().ar_corr_train(self.handle, h.ctypes.data, h.shape[0], int(epochs),
                                       int(batch), float(lr), tr.ctypes.data, _stream(stream)),
                   "ar_corr_train")
        else:
            t = np.ascontiguousarray(tables, dtype=np.float64).reshape(h.shape[0], -1)
            if t.shape[1] != CORR_GRID * CORR_GRID:
                raise ValueError("tables must be count x 33 x 33")
            _check(lib().ar_corr_train_tables(self.handle, h.ctypes.data, t.ctypes.data,
                                              h.shape[0], int(epochs), int(batch), float(lr),
                                              tr.ctypes.data, _stream(stream)),
                   "ar_corr_train_tables")
        return tr[:int(epochs)]

    def predict(self, psf) -> np.ndarray:
        h = np.ascontiguousarray(psf, dtype=np.float64).reshape(225)
        t = np.empty(CORR_GRID * CORR_GRID, dtype=np.float32)
        _check(lib().ar_corr_predict(self.handle, h.ctypes.data, t.ctypes.data), "ar_corr_predict")
        return t.reshape(CORR_GRID, CORR_GRID)

    def close(self) -> None:
        if self.handle:
            lib().ar_corr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def param_count() -> int:
    return int(lib().ar_corr_param_count())


def corr_targets(psfs) -> np.ndarray:
    """Exact delta tables (float64, computed on the GPU) of 15 x 15 PSFs."""
    h = np.ascontiguousarray(psfs, dtype=np.float64).reshape(-1, 225)
    out = np.empty((h.shape[0], CORR_GRID * CORR_GRID), dtype=np.float64)
    _check(lib().ar_corr_targets(h.ctypes.data, h.shape[0], out.ctypes.data), "ar_corr_targets")
    return out.reshape(-1, CORR_GRID, CORR_GRID)


def corr_restoration_targets(f: torch.Tensor, e: torch.Tensor, psfs, nu: float, alpha: float,
                             tau: float = 1.0, iters: int = 8, stream=None) -> np.ndarray:
    """Training tables (count x 33 x 33, float64) read off restorations of the scene
    ``f`` (noise field ``e``, relative level ``nu``) by the symmetrized D-Landweber,
    one per 15 x 15 PSF (see ``include/ar.h``)."""
    _image(f, "f")
    _image(e, "e")
    if f.shape != e.shape:
        raise ValueError("f and e must have the same shape")
    h = np.ascontiguousarray(psfs, dtype=np.float64).reshape(-1, 225)
    out = np.empty((h.shape[0], CORR_GRID * CORR_GRID), dtype=np.float64)
    n1, n2 = f.shape
    _check(lib().ar_corr_restoration_targets(
        f.data_ptr(), e.data_ptr(), n1, n2, h.ctypes.data, h.shape[0], float(nu), float(alpha),
        float(tau), int(iters), out.ctypes.data, _stream(stream)), "ar_corr_restoration_targets")
    return out.reshape(-1, CORR_GRID, CORR_GRID)


def ar_symprec_setup_corrected(psf, n1: int, n2: int, alpha: float, model: "Corr | None" = None,
                               stream=None, precision: str = "fp32") -> Prec:
    """AR preconditioner with d = 1/(lambda_s^2 + delta + alpha); delta exact
    (model None) or predicted by ``model``."""
    h = _host_psf(psf)
    q1, q2 = _support(h.shape)
    out = _vp()
    _check(lib().ar_symprec_setup_corrected(h.ctypes.data, q1, q2, n1, n2, float(alpha),
                                            model.handle if model is not None else None,
                                            PRECISION[precision], _stream(stream),
                                            ctypes.byref(out)), "ar_symprec_setup_corrected")
    return Prec(out.value, n1, n2)


def ar_restore_prec(P: Prec, g: torch.Tensor, psf, tau: float = 1.0, iters: int = 20,
                    x0: torch.Tensor | None = None, f_true: torch.Tensor | None = None,
                    x_out: torch.Tensor | None = None, trace: bool = True, stream=None):
    """D-Landweber with a preconditioner built beforehand.  Returns ``(x, trace, best)``."""
    _image(g, "g")
    if tuple(g.shape) != P.shape:
        raise ValueError(f"g has shape {tuple(g.shape)}, preconditioner expects {P.shape}")
    h = _host_psf(psf)
    if x_out is None:
        x_out = torch.empty_like(g)
    _image(x_out, "x_out")
    want = f_true is not None and trace
    tr = np.zeros(max(iters, 1), dtype=np.float64) if want else None
    best = _i(0)
    _check(lib().ar_restore_prec(
        P.handle, g.data_ptr(), h.ctypes.data, float(tau), int(iters),
        _image(x0, "x0").data_ptr() if x0 is not None else None,
        _image(f_true, "f_true").data_ptr() if f_true is not None else None,
        x_out.data_ptr(), tr.ctypes.data if want else None,
        ctypes.addressof(best) if want else None, _stream(stream)), "ar_restore_prec")
    return x_out, (tr[:iters] if want else None), (best.value if want else None)


def set_stencil_wait_polls(polls: int = DEFAULT_WAIT_POLLS) -> None:
    """Polls of the stencils' halo-tile waits before they give up (failure-detection
    tests; ``0`` makes every wait give up, the default restores the normal bound)."""
    _check(lib().ar_set_stencil_wait_polls(int(polls)), "ar_set_stencil_wait_polls")


def inject_alloc_failures(count: int, skip: int = 0) -> None:
    """Let the library's next ``skip`` scratch / preconditioner allocations succeed and
    make the ``count`` after them fail (``count=0`` clears the injection)."""
    lib().ar_inject_alloc_failures(int(skip), int(count))


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().ar_kernel_launches())


def version() -> str:
    return lib().ar_version().decode()
