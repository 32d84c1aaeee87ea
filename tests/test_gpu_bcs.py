"""GPU parity of the comparison boundary conditions (Reflective, Periodic)
against the FP64 oracle: blur / reblur, preconditioner setup and solve, and
(D-)Landweber restoration, through the C ABI's *_bc entry points.

Tolerances are those of the AR path (see test_gpu_parity), except the
Periodic solve: it is the sum of two synthesised terms (the parts of d even
in each frequency and odd in both), each with the AR bound relative to the
whole, so its bound is twice tol(alpha)."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1211_0393_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BCS = {"reflective": O.BC_REFLECTIVE, "periodic": O.BC_PERIODIC}
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def ar():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0393_gb300 import ar as mod

    mod.lib()
    return mod


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def tol_alpha(alpha, bc):
    t = max(1e-5, 3 * U32 / alpha)
    return 2 * t if bc == "periodic" else t


def tol_fast(alpha, bc):
    t = max(1e-4, 3 * 2.0 ** -16 / alpha)
    return 2 * t if bc == "periodic" else t


def assert_trace_close(tr, to, tol):
    """RRE_k = ||x_k - f|| / ||f||: by the triangle inequality the RRE differs
    by at most ||x_k - x_k^oracle|| / ||f|| <= tol ||x_k|| / ||f|| <= tol (1 + RRE_k)."""
    tr, to = np.asarray(tr), np.asarray(to)
    assert np.all(np.abs(tr - to) <= tol * (1.0 + to)), np.max(np.abs(tr - to) / (1.0 + to))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rand_psf(rng, q1, q2):
    h = rng.uniform(0.0, 1.0, size=(2 * q1 + 1, 2 * q2 + 1))
    return h / h.sum()


BLUR_CASES = [
    (64, 64, 4, 4),
    (3, 3, 1, 1),
    (5, 4, 0, 3),         # q2 = n2 - 1
    (8, 9, 7, 8),         # q_j = n_j - 1 on both axes
    (130, 200, 7, 7),     # several tiles, ragged tails
    (77, 301, 2, 6),      # non-square support, padded fast path
    (70, 90, 16, 20),     # generic kernel (q > 15)
    (257, 129, 15, 15),
]


@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("n1,n2,q1,q2", BLUR_CASES)
def test_blur_and_reblur_match_oracle(ar, bc, n1, n2, q1, q2):
    rng = np.random.default_rng(n1 * 5 + n2 * 11 + q1 + q2)
    h = rand_psf(rng, q1, q2).astype(np.float32)
    x = rng.uniform(0, 1, (n1, n2)).astype(np.float32)
    xd, hd = dev(x), dev(h)
    y = ar.ar_blur_apply(xd, hd, bc=bc).cpu().numpy()
    yr = ar.ar_reblur_apply(xd, hd, bc=bc).cpu().numpy()
    ref = O.blur_bc(x.astype(np.float64), h.astype(np.float64), BCS[bc])
    refr = O.reblur_bc(x.astype(np.float64), h.astype(np.float64), BCS[bc])
    for got, want in ((y, ref), (yr, refr)):
        assert rel_l2(got, want) <= 2e-6
        assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want))


def test_bc_changes_only_the_border(ar):
    """Away from the border (distance > q) all three BCs give the same blur."""
    rng = np.random.default_rng(3)
    h = dev(rand_psf(rng, 3, 2))
    x = dev(rng.uniform(0, 1, (96, 80)))
    ys = [ar.ar_blur_apply(x, h, bc=b).cpu().numpy() for b in ("ar", "reflective", "periodic")]
    for y in ys[1:]:
        assert np.array_equal(y[3:-3, 2:-2], ys[0][3:-3, 2:-2])
        assert not np.array_equal(y, ys[0])


SETUP_CASES = [(8, 8, 2, 2, 0.1), (64, 64, 4, 4, 0.03), (37, 53, 5, 3, 0.01), (3, 3, 0, 0, 1.0),
               (5, 6, 4, 5, 0.5), (200, 120, 10, 1, 0.05), (1024, 1024, 7, 7, 0.3)]


@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("n1,n2,q1,q2,alpha", SETUP_CASES)
def test_setup_eigenvalues_match_oracle(ar, bc, n1, n2, q1, q2, alpha):
    rng = np.random.default_rng(n1 + 2 * n2 + q1)
    h = rand_psf(rng, q1, q2)
    P = ar.ar_symprec_setup(h, n1, n2, alpha, bc=bc)
    lam, d = ar.ar_symprec_eigenvalues(P)
    prec = O.symprec_setup_bc(h, n1, n2, alpha, BCS[bc])
    assert np.max(np.abs(lam - prec["lam"])) <= 1e-13
    assert np.max(np.abs(d - prec["d"]) / prec["d"]) <= 1e-12
    assert lam[0, 0] == pytest.approx(1.0, abs=1e-14)      # zero frequency: sum(h) = 1
    P.close()


SOLVE_CASES = [(8, 8, 2, 2, 0.1), (64, 64, 4, 4, 0.03), (37, 53, 5, 3, 0.01), (130, 257, 7, 7, 0.3),
               (3, 3, 0, 0, 1.0), (5, 6, 4, 5, 0.5), (1024, 1024, 7, 7, 0.3)]


@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("n1,n2,q1,q2,alpha", SOLVE_CASES)
def test_solve_matches_oracle(ar, bc, n1, n2, q1, q2, alpha):
    rng = np.random.default_rng(n1 * n2 + q2 + 1)
    h = rand_psf(rng, q1, q2)
    y = rng.standard_normal((n1, n2)).astype(np.float32)
    P = ar.ar_symprec_setup(h, n1, n2, alpha, bc=bc)
    z = ar.ar_symprec_solve(P, dev(y)).cpu().numpy()
    want = O.symprec_solve_bc(O.symprec_setup_bc(h, n1, n2, alpha, BCS[bc]), y.astype(np.float64))
    assert rel_l2(z, want) <= tol_alpha(alpha, bc)
    yd = dev(y)
    ar.ar_symprec_solve(P, yd, yd)                           # in place
    assert rel_l2(yd.cpu().numpy(), want) <= tol_alpha(alpha, bc)
    P.close()


@pytest.mark.parametrize("bc", list(BCS))
def test_solve_bf16x2_mode_matches_oracle(ar, bc):
    rng = np.random.default_rng(11)
    h = rand_psf(rng, 7, 7)
    y = rng.standard_normal((130, 257)).astype(np.float32)
    P = ar.ar_symprec_setup(h, 130, 257, 0.3, precision="bf16x2", bc=bc)
    z = ar.ar_symprec_solve(P, dev(y)).cpu().numpy()
    want = O.symprec_solve_bc(O.symprec_setup_bc(h, 130, 257, 0.3, BCS[bc]), y.astype(np.float64))
    assert rel_l2(z, want) <= tol_fast(0.3, bc)
    P.close()


def _workload(n, psf, scene, cidx, nu):
    q1, q2 = O.psf_support(psf)
    ext, f, e = W.make_inputs(n, n, psf, scene, cidx)
    g = W.add_noise(W.crop(O.ar_blur(ext, psf), q1, q2), e, nu)
    return g.astype(np.float32), f.astype(np.float32)


RESTORE_CASES = [
    # n, psf, scene, cfg, nu, alpha, iters, precondition
    (64, "config1", "blocks", 0, 0.01, 0.03, 20, True),
    (64, "config1", "blocks", 0, 0.01, 0.0, 30, False),
    (200, "config2", "ellipses", 1, 0.005, 0.3, 10, True),
    (200, "config2", "ellipses", 1, 0.005, 0.0, 10, False),
]


@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("n,psf,scene,cidx,nu,alpha,iters,pc", RESTORE_CASES)
def test_restore_matches_oracle(ar, bc, n, psf, scene, cidx, nu, alpha, iters, pc):
    h = W.psf_named(psf)
    g, f = _workload(n, h, scene, cidx, nu)
    x, tr, best = ar.ar_restore(dev(g), h, alpha, 1.0, iters, pc, f_true=dev(f), bc=bc)
    xo, to, bo = O.restore_bc(g.astype(np.float64), h, alpha, BCS[bc], 1.0, iters, pc,
                              f_true=f.astype(np.float64))
    tol = tol_alpha(alpha, bc) if pc else 1e-5
    assert rel_l2(x.cpu().numpy(), xo) <= tol
    assert_trace_close(tr, to, tol)
    srt = np.sort(to)
    if iters > 1 and srt[1] - srt[0] > 1e-4 * srt[0]:
        assert best == bo
    else:
        assert to[best - 1] <= to.min() * (1 + 1e-4)


@pytest.mark.parametrize("bc", list(BCS))
def test_restore_full_size_first_iterations(ar, bc):
    """ellipses 1024^2 with the 15x15 motion PSF under the comparison BC:
    first 3 preconditioned iterations against the oracle."""
    h = W.psf_config2()
    g, f = _workload(1024, h, "ellipses", 1, 0.005)
    x, tr, _ = ar.ar_restore(dev(g), h, 0.3, 1.0, 3, True, f_true=dev(f), bc=bc)
    xo, to, _ = O.restore_bc(g.astype(np.float64), h, 0.3, BCS[bc], 1.0, 3, True,
                             f_true=f.astype(np.float64))
    assert rel_l2(x.cpu().numpy(), xo) <= tol_alpha(0.3, bc)
    assert_trace_close(tr, to, tol_alpha(0.3, bc))


def test_unknown_bc_is_rejected(ar):
    import ctypes
    h = np.ascontiguousarray(W.psf_config1())
    out = ctypes.c_void_p()
    st = ar.lib().ar_symprec_setup_bc(h.ctypes.data, 4, 4, 16, 16, 0.1, 9, 0, None,
                                      ctypes.byref(out))
    assert st == 1 and out.value is None
