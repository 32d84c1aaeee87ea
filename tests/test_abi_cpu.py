"""CPU checks of the C ABI: the library loads, exports every symbol the header
declares, and its host-side validation rejects bad arguments before touching
the GPU (only calls that fail validation are made here)."""

import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1211_0393_gb300 import _build
    from paper_1211_0393_gb300 import ar

    if not os.path.exists(ar.LIB_PATH):
        _build.build()
    return ar.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ar.h")).read()
    return sorted(set(re.findall(r"AR_API\s+[\w\s\*]*?\b(ar_\w+)\s*\(", src)))


def test_header_declares_the_five_calls_of_the_path():
    syms = declared_symbols()
    for s in ["ar_blur_apply", "ar_reblur_apply", "ar_symprec_setup", "ar_symprec_solve",
              "ar_restore", "ar_symprec_destroy", "ar_status_string"]:
        assert s in syms


def test_library_exports_every_declared_symbol(L):
    from paper_1211_0393_gb300 import ar

    for s in declared_symbols():
        assert hasattr(L, s), s
    assert sorted(ar.EXPORTS) == declared_symbols()


def test_status_strings(L):
    from paper_1211_0393_gb300.ar import STATUS

    for code, name in STATUS.items():
        assert L.ar_status_string(code).decode() == name
    assert L.ar_status_string(99).decode() == "AR_UNKNOWN"
    assert "sm_103a" in L.ar_version().decode()


FAKE = 0x10000  # never dereferenced: every call below fails validation first


@pytest.mark.parametrize("args,code", [
    ((None, FAKE, 8, 8, FAKE, 1, 1), 1),          # null x
    ((FAKE, FAKE + 4, 8, 8, FAKE * 16, 1, 1), 2),  # y overlaps x
    ((FAKE, FAKE * 4, 8, 8, FAKE * 16, 8, 1), 1),  # q1 > n1 - 1
    ((FAKE, FAKE * 4, 0, 8, FAKE * 16, 0, 0), 1),  # n1 < 1
    ((FAKE, FAKE * 4, 8, 8, FAKE * 16, -1, 0), 1),  # q < 0
])
def test_apply_validation(L, args, code):
    assert L.ar_blur_apply(*args, None) == code
    assert L.ar_reblur_apply(*args, None) == code
    assert L.ar_last_error_detail().decode() != ""


def _psf(q1, q2, scale=1.0):
    h = np.ones((2 * q1 + 1, 2 * q2 + 1))
    return np.ascontiguousarray(h / h.sum() * scale)


def test_setup_validation(L):
    out = ctypes.c_void_p()
    h = _psf(1, 1)
    assert L.ar_symprec_setup(None, 1, 1, 8, 8, 0.1, None, ctypes.byref(out)) == 1
    assert L.ar_symprec_setup(h.ctypes.data, 1, 1, 8, 8, 0.1, None, None) == 1
    assert L.ar_symprec_setup(h.ctypes.data, 1, 1, 2, 8, 0.1, None, ctypes.byref(out)) == 1
    assert L.ar_symprec_setup(h.ctypes.data, 1, 1, 8, 8, 0.0, None, ctypes.byref(out)) == 1
    assert L.ar_symprec_setup(h.ctypes.data, 1, 1, 8, 8, float("nan"), None, ctypes.byref(out)) == 1
    h6 = _psf(3, 3)
    assert L.ar_symprec_setup(h6.ctypes.data, 3, 3, 5, 8, 0.1, None, ctypes.byref(out)) == 1  # q > n-3
    hb = _psf(1, 1, scale=1.01)
    assert L.ar_symprec_setup(hb.ctypes.data, 1, 1, 8, 8, 0.1, None, ctypes.byref(out)) == 3
    hn = _psf(1, 1)
    hn[0, 0] = np.nan
    assert L.ar_symprec_setup(hn.ctypes.data, 1, 1, 8, 8, 0.1, None, ctypes.byref(out)) == 1
    assert out.value is None


def test_restore_validation(L):
    h = _psf(2, 2)
    hp = h.ctypes.data
    base = dict(g=FAKE, h=hp, n1=16, n2=16, q1=2, q2=2, alpha=0.1, tau=1.0, iters=3, pc=1,
                x0=None, f=None, x=FAKE * 64, tr=None, best=None)

    def call(**kw):
        a = dict(base, **kw)
        return L.ar_restore(a["g"], a["h"], a["n1"], a["n2"], a["q1"], a["q2"], a["alpha"],
                            a["tau"], a["iters"], a["pc"], a["x0"], a["f"], a["x"], a["tr"],
                            a["best"], None)

    assert call(g=None) == 1
    assert call(x=None) == 1
    assert call(iters=-1) == 1
    assert call(tau=0.0) == 1
    assert call(alpha=-1.0) == 1
    assert call(tr=FAKE) == 1                     # trace without f_true
    assert call(x=FAKE + 64) == 2                 # x_out overlaps g
    assert call(f=FAKE * 64 + 32) == 2            # x_out overlaps f_true
    assert call(x0=FAKE * 64 + 8) == 2            # x0 partially overlaps x_out
    assert call(q1=14) == 1                       # q > n-3 with the preconditioner
    hb = _psf(2, 2, scale=0.5)
    assert call(h=hb.ctypes.data) == 3


def test_binding_refuses_cpu_tensors():
    import torch

    from paper_1211_0393_gb300 import ar

    x = torch.zeros(8, 8)
    with pytest.raises(TypeError):
        ar.ar_blur_apply(x, torch.ones(3, 3))


def test_bc_validation(L):
    args = (FAKE, FAKE * 4, 8, 8, FAKE * 16, 1, 1)
    for bc in (-1, 3):
        assert L.ar_blur_apply_bc(*args, bc, None) == 1
        assert L.ar_reblur_apply_bc(*args, bc, None) == 1
    for bc in (1, 2):
        assert L.ar_blur_apply_bc(FAKE, FAKE + 4, 8, 8, FAKE * 16, 1, 1, bc, None) == 2
        assert L.ar_blur_apply_bc(FAKE, FAKE * 4, 8, 8, FAKE * 16, 8, 1, bc, None) == 1
    out = ctypes.c_void_p()
    h = _psf(1, 1)
    assert L.ar_symprec_setup_bc(h.ctypes.data, 1, 1, 8, 8, 0.1, 3, 0, None,
                                 ctypes.byref(out)) == 1
    assert L.ar_symprec_setup_bc(h.ctypes.data, 1, 1, 8, 8, 0.1, 1, 7, None,
                                 ctypes.byref(out)) == 1          # unknown precision
    h6 = _psf(6, 6)
    assert L.ar_symprec_setup_bc(h6.ctypes.data, 6, 6, 6, 6, 0.1, 1, 0, None,
                                 ctypes.byref(out)) == 1          # q > n - 1
    assert out.value is None
    hp = _psf(2, 2).ctypes.data
    assert L.ar_restore_bc(FAKE, hp, 16, 16, 2, 2, 0.1, 1.0, 3, 5, 1, 0, None, None,
                           FAKE * 64, None, None, None) == 1      # unknown bc
    assert L.ar_restore_bc(FAKE, hp, 16, 16, 2, 2, 0.1, 1.0, 3, 1, 1, 0, None, None,
                           FAKE + 64, None, None, None) == 2      # x_out overlaps g


def test_correction_validation(L):
    out = ctypes.c_void_p()
    assert L.ar_corr_param_count() == 225 * 256 + 256 + 256 * 256 + 256 + 256 * 1089 + 1089
    assert L.ar_corr_create(None, ctypes.byref(out)) == 1
    bad = np.zeros(L.ar_corr_param_count(), dtype=np.float32)
    bad[7] = np.nan
    assert L.ar_corr_create(bad.ctypes.data, ctypes.byref(out)) == 1
    assert out.value is None
    h = np.ones(225) / 225.0
    assert L.ar_corr_targets(h.ctypes.data, 0, FAKE) == 1
    assert L.ar_corr_train(None, h.ctypes.data, 1, 1, 1, 1e-3, None, None) == 1
    assert L.ar_corr_predict(None, h.ctypes.data, FAKE) == 1
    h3 = _psf(1, 1)
    # a model takes 15 x 15 PSFs only (the model pointer is not dereferenced)
    assert L.ar_symprec_setup_corrected(h3.ctypes.data, 1, 1, 16, 16, 0.1, FAKE, 0, None,
                                        ctypes.byref(out)) == 1
    assert L.ar_symprec_setup_corrected(h3.ctypes.data, 1, 1, 16, 16, 0.0, None, 0, None,
                                        ctypes.byref(out)) == 1
    assert L.ar_restore_prec(None, FAKE, h3.ctypes.data, 1.0, 3, None, None, FAKE * 64, None,
                             None, None) == 1


def test_residual_restore_validation(L):
    hp = _psf(2, 2).ctypes.data
    res = np.zeros(4)

    def call(x=FAKE * 64, r=res.ctypes.data, bc=0, pc=1, q1=2, tr=None):
        return L.ar_restore_residuals(FAKE, hp, 16, 16, q1, 2, 0.1, 1.0, 3, bc, pc, 0, None,
                                      None, x, tr, None, r, None)

    assert call(r=None) == 1                      # the residual trace is the point of the call
    assert call(x=None) == 1
    assert call(bc=5) == 1
    assert call(tr=FAKE) == 1                     # RRE trace without f_true
    assert call(x=FAKE + 64) == 2                 # x_out overlaps g
    assert call(q1=14) == 1                       # q > n-3 with the preconditioner


def test_injected_allocation_failure_is_reported(L):
    """A host-side fake of a failing device allocation (no GPU involved): the
    restoration and the preconditioner setup return AR_ERR_ALLOC before any GPU
    work, name the failed allocation, and the injection is used up."""
    hp = _psf(2, 2).ctypes.data
    out = ctypes.c_void_p()
    try:
        L.ar_inject_alloc_failures(0, 1)
        st = L.ar_restore(FAKE, hp, 16, 16, 2, 2, 0.1, 1.0, 3, 1, None, None, FAKE * 64, None,
                          None, None)
        assert st == 4, st
        assert "cudaMallocAsync" in L.ar_last_error_detail().decode()
        L.ar_inject_alloc_failures(0, 1)
        assert L.ar_symprec_setup(hp, 2, 2, 16, 16, 0.1, None, ctypes.byref(out)) == 4
        assert out.value is None
        L.ar_inject_alloc_failures(0, 2)
        assert L.ar_restore(FAKE, hp, 16, 16, 2, 2, 0.1, 1.0, 3, 0, None, None, FAKE * 64,
                            None, None, None) == 4
        assert L.ar_restore(FAKE, hp, 16, 16, 2, 2, 0.1, 1.0, 3, 0, None, None, FAKE * 64,
                            None, None, None) == 4
    finally:
        L.ar_inject_alloc_failures(0, 0)


def test_stencil_arithmetic_validation(L):
    """AR_STENCIL_F16X2 (16) and AR_STENCIL_AUTO (32) are accepted by the apply calls
    and OR-ed into the restoration's precision (not both); anything else is
    rejected before any GPU work."""
    args = (FAKE, FAKE * 4, 8, 8, FAKE * 16, 1, 1, 0)
    for stencil in (3, 17, -1):
        assert L.ar_blur_apply_ex(*args, stencil, None) == 1
        assert L.ar_reblur_apply_ex(*args, stencil, None) == 1
    for stencil in (0, 16, 32):                # accepted: the alias check runs next
        assert L.ar_blur_apply_ex(FAKE, FAKE + 4, 8, 8, FAKE * 16, 1, 1, 0, stencil, None) == 2
    hp = _psf(2, 2).ctypes.data
    for precision in (16 | 7, 64, 16 | 32):     # unknown, or both stencil flags
        assert L.ar_restore_bc(FAKE, hp, 16, 16, 2, 2, 0.1, 1.0, 3, 0, 1, precision, None,
                               None, FAKE * 64, None, None, None) == 1
    assert L.ar_restore_bc(FAKE, hp, 16, 16, 2, 2, 0.1, 1.0, 3, 0, 1, 16 | 1, None, None,
                           FAKE + 64, None, None, None) == 2      # flag accepted; x_out overlaps g
