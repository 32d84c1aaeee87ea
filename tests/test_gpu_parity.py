"""GPU parity: every C-ABI call against the FP64 oracle on identical seeded inputs.

Tolerances (derived from the arithmetic; see the design notes):
* blur / reblur: float32 sums of K = (2q1+1)(2q2+1) products of O(1) data:
  rel-L2 <= 2e-6 and max |err| <= 1e-5 max|y|.
* setup (float64 on both sides): |d_gpu - d| <= 1e-12 d.
* preconditioner and restoration (float32 data, transforms with float32-
  grade accuracy): rel-L2 <= 1e-5 per iterate for alpha >= 0.018.  Below that
  the float32 arithmetic itself does not reach 1e-5: the errors of the two
  contractions before the filter (float32 sums with cancellation, since a
  smooth image has small high-frequency coefficients) and the float32 stores of
  their inputs are absolute relative to the image's norm, and the filter d of
  eq. TikFilter multiplies them by up to max(d) = 1/alpha.  Attribution on the
  config-1 input at alpha = 0.01 (first iterate, numpy float64 vs float32
  emulations of the chain): round-to-nearest float32 products and sums 8.8e-6,
  the stores of the reblurred image and of the first contraction's output
  2.9e-6 together, the stores after the filter 3e-8; the tensor-core path
  measures 1.5e-5 at the first iterate and 1.3e-5 at the twentieth.  So the
  bound is tol(alpha) = max(1e-5, 3 u / alpha), u = 2^-24: 1.8e-5 at
  alpha = 0.01.
* the bf16x2 precision mode (two planes, three products) keeps 16 significant
  bits per operand: the same argument with u = 2^-16 gives
  tol_fast(alpha) = max(1e-4, 3 * 2^-16 / alpha).
"""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1211_0393_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ar():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0393_gb300 import ar as mod

    mod.lib()
    return mod


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


U32 = 2.0 ** -24
U_BF16X2 = 2.0 ** -16     # two bf16 planes keep 16 significant bits; the a1*b1 product is dropped


def tol_alpha(alpha):
    return max(1e-5, 3 * U32 / alpha)


def tol_fast(alpha):
    """Same derivation as tol_alpha with the two-plane split's unit 2^-16."""
    return max(1e-4, 3 * U_BF16X2 / alpha)


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
    (64, 64, 4, 4),       # config-1 geometry, one tile
    (3, 3, 1, 1),         # smallest image with a 3x3 PSF
    (5, 4, 0, 3),         # q1 = 0, q2 = n2 - 1 (maximum support)
    (8, 9, 7, 8),         # q_j = n_j - 1 on both axes
    (130, 200, 7, 7),     # several tiles, ragged tails
    (77, 301, 2, 6),      # non-square support, padded fast path
    (70, 90, 16, 20),     # generic kernel (q > 15)
    (257, 129, 15, 15),   # largest fast-path support
    (1024, 1024, 7, 7),   # config-2 geometry
]


@pytest.mark.parametrize("n1,n2,q1,q2", BLUR_CASES)
def test_blur_and_reblur_match_oracle(ar, n1, n2, q1, q2):
    rng = np.random.default_rng(n1 * 7 + n2 * 3 + q1 + q2)
    h = rand_psf(rng, q1, q2).astype(np.float32)
    x = rng.uniform(0, 1, (n1, n2)).astype(np.float32)
    xd, hd = dev(x), dev(h)
    y = ar.ar_blur_apply(xd, hd).cpu().numpy()
    yr = ar.ar_reblur_apply(xd, hd).cpu().numpy()
    ref = O.ar_blur(x.astype(np.float64), h.astype(np.float64))
    refr = O.ar_reblur(x.astype(np.float64), h.astype(np.float64))
    for got, want in ((y, ref), (yr, refr)):
        assert rel_l2(got, want) <= 2e-6
        assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want))


# Shapes for the persistent TMA stencil (row pitch a multiple of 16 bytes):
# more tiles than resident CTAs, the largest support, ragged tails, thin images.
TMA_CASES = [
    (4096, 4096, 1, 1),
    (1000, 1028, 15, 15),
    (97, 260, 3, 9),
    (2048, 64, 2, 2),
    (3, 4, 1, 1),
    (65, 68, 0, 0),
]


@pytest.mark.parametrize("n1,n2,q1,q2", TMA_CASES)
def test_tma_stencil_matches_oracle(ar, n1, n2, q1, q2):
    rng = np.random.default_rng(n1 + 5 * n2 + q1)
    h = rand_psf(rng, q1, q2).astype(np.float32)
    x = rng.uniform(0, 1, (n1, n2)).astype(np.float32)
    xd, hd = dev(x), dev(h)
    for fn, ofn in ((ar.ar_blur_apply, O.ar_blur), (ar.ar_reblur_apply, O.ar_reblur)):
        got = fn(xd, hd).cpu().numpy()
        want = ofn(x.astype(np.float64), h.astype(np.float64))
        assert rel_l2(got, want) <= 2e-6
        assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want))


@pytest.mark.parametrize("bc", ["ar", "reflective"])
def test_tma_and_thread_loaded_stencils_agree_bitwise(ar, bc):
    """An image whose base is not 16-byte aligned takes the thread-loaded
    kernel; both kernels share the arithmetic, so the results are identical."""
    n = 256
    rng = np.random.default_rng(5)
    x = torch.from_numpy(rng.uniform(0, 1, (n, n)).astype(np.float32)).cuda()
    h = dev(rand_psf(rng, 7, 7))
    flat = torch.empty(n * n + 1, device="cuda")
    xu = flat[1:].view(n, n)
    xu.copy_(x)
    assert xu.data_ptr() % 16 != 0
    for fn in (ar.ar_blur_apply, ar.ar_reblur_apply):
        assert torch.equal(fn(x, h, bc=bc), fn(xu, h, bc=bc))


def test_blur_config2_psf_and_streams(ar):
    """The bench PSF at 1024^2 on a side stream, sampled against the oracle's
    per-pixel definition (eq. modello_discreto over the AR extension)."""
    n = 1024
    h = W.psf_config2().astype(np.float32)
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (n, n)).astype(np.float32)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        xd, hd = dev(x), dev(h)
        y = ar.ar_blur_apply(xd, hd, stream=s)
    s.synchronize()
    y = y.cpu().numpy()
    xp = O.ar_pad(x.astype(np.float64), 7, 7)
    hh = h.astype(np.float64)
    pts = [(0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1), (3, 500), (512, 6), (1000, 1017)]
    pts += [tuple(p) for p in rng.integers(0, n, size=(40, 2))]
    for i1, i2 in pts:
        # y_i = sum_s h_s xt_{i-s}; xt_{j} = xp[j + q]
        win = xp[i1:i1 + 15, i2:i2 + 15][::-1, ::-1]
        want = float(np.sum(hh * win))
        assert abs(y[i1, i2] - want) <= 1e-5 * max(1.0, abs(want)), (i1, i2)


def test_blur_rejects_alias_on_device(ar):
    x = torch.zeros(16, 16, device="cuda")
    h = torch.ones(3, 3, device="cuda") / 9
    with pytest.raises(ar.ARError) as ei:
        ar.ar_blur_apply(x, h, y=x)
    assert ei.value.name == "AR_ERR_ALIAS"


SETUP_CASES = [(8, 8, 2, 2, 0.1), (64, 64, 4, 4, 0.03), (37, 53, 5, 3, 0.01), (1024, 1024, 7, 7, 0.3),
               (3, 3, 0, 0, 1.0), (200, 120, 10, 1, 0.05)]


@pytest.mark.parametrize("n1,n2,q1,q2,alpha", SETUP_CASES)
def test_setup_eigenvalues_match_oracle(ar, n1, n2, q1, q2, alpha):
    rng = np.random.default_rng(n1 + n2 + q1)
    h = rand_psf(rng, q1, q2)
    P = ar.ar_symprec_setup(h, n1, n2, alpha)
    lam, d = ar.ar_symprec_eigenvalues(P)
    prec = O.symprec_setup(h, n1, n2, alpha)
    assert np.max(np.abs(lam - prec["lam"])) <= 1e-13
    assert np.max(np.abs(d - prec["d"]) / prec["d"]) <= 1e-12
    assert ar.ar_symprec_shape(P) == (n1, n2)
    # corners of Theorem 2: eigenvalue sum(h) = 1
    for c in [(0, 0), (0, n2 - 1), (n1 - 1, 0), (n1 - 1, n2 - 1)]:
        assert lam[c] == pytest.approx(1.0, abs=1e-14)
    P.close()


SOLVE_CASES = [(8, 8, 2, 2, 0.1), (64, 64, 4, 4, 0.03), (37, 53, 5, 3, 0.01), (130, 257, 7, 7, 0.3),
               (3, 3, 0, 0, 1.0), (256, 256, 7, 7, 0.3), (1024, 1024, 7, 7, 0.3),
               # odd n1 (G4's middle column s1 = (n1-1)/2 belongs to one parity) with a
               # folded input (n2 % 4 == 0)
               (37, 64, 5, 5, 0.1), (129, 200, 7, 3, 0.3)]


@pytest.mark.parametrize("n1,n2,q1,q2,alpha", SOLVE_CASES)
def test_solve_matches_oracle(ar, n1, n2, q1, q2, alpha):
    rng = np.random.default_rng(n1 * n2 + q2)
    h = rand_psf(rng, q1, q2)
    y = rng.standard_normal((n1, n2)).astype(np.float32)
    P = ar.ar_symprec_setup(h, n1, n2, alpha)
    z = ar.ar_symprec_solve(P, dev(y)).cpu().numpy()
    want = O.symprec_solve(O.symprec_setup(h, n1, n2, alpha), y.astype(np.float64))
    assert rel_l2(z, want) <= tol_alpha(alpha)
    # in place
    yd = dev(y)
    ar.ar_symprec_solve(P, yd, yd)
    assert rel_l2(yd.cpu().numpy(), want) <= tol_alpha(alpha)
    P.close()


def _workload(n, psf, scene, cidx, nu):
    q1, q2 = O.psf_support(psf)
    ext, f, e = W.make_inputs(n, n, psf, scene, cidx)
    g = W.add_noise(W.crop(O.ar_blur(ext, psf), q1, q2), e, nu)
    return g.astype(np.float32), f.astype(np.float32)


RESTORE_CASES = [
    # n, psf, scene, cfg, nu, alpha, iters, precondition
    (64, "config1", "blocks", 0, 0.01, 0.03, 20, True),
    (64, "config1", "blocks", 0, 0.01, 0.01, 20, True),
    (64, "config1", "blocks", 0, 0.01, 0.0, 30, False),
    (200, "config2", "ellipses", 1, 0.005, 0.3, 10, True),
    (200, "config2", "ellipses", 1, 0.005, 0.0, 10, False),
]


@pytest.mark.parametrize("n,psf,scene,cidx,nu,alpha,iters,pc", RESTORE_CASES)
def test_restore_matches_oracle(ar, n, psf, scene, cidx, nu, alpha, iters, pc):
    h = W.psf_named(psf)
    g, f = _workload(n, h, scene, cidx, nu)
    x, tr, best = ar.ar_restore(dev(g), h, alpha, 1.0, iters, pc, f_true=dev(f))
    xo, to, bo = O.restore(g.astype(np.float64), h, alpha, 1.0, iters, pc,
                           f_true=f.astype(np.float64))
    tol = tol_alpha(alpha) if pc else 1e-5
    assert rel_l2(x.cpu().numpy(), xo) <= tol
    assert_trace_close(tr, to, tol)
    # IT: equal when the oracle's minimum is clear, else the GPU's pick is a near-tie
    srt = np.sort(to)
    if iters > 1 and srt[1] - srt[0] > 1e-4 * srt[0]:
        assert best == bo
    else:
        assert to[best - 1] <= to.min() * (1 + 1e-4)


FOLD_CASES = [
    # n1, n2, q1, q2: the reblur writes the transform input folded along the
    # columns when n2 % 4 == 0 and q <= 15 (AR); the rest keep the plain input
    (40, 40, 3, 3),        # one column pair whose mirror tile starts left of the image
    (72, 120, 7, 5),       # rectangular, ragged column pairs
    (36, 52, 15, 15),      # widest folded halo
    (44, 48, 16, 2),       # q > 15: plain input, generic stencil
    (45, 51, 4, 4),        # odd sides: plain input
    (50, 50, 2, 2),        # n2 % 4 == 2: plain input
]


@pytest.mark.parametrize("n1,n2,q1,q2", FOLD_CASES)
def test_restore_folded_input_shapes(ar, n1, n2, q1, q2):
    rng = np.random.default_rng(n1 * 31 + n2 + q1)
    h = rand_psf(rng, q1, q2)
    f = rng.uniform(0, 1, (n1, n2))
    g = (O.ar_blur(f, h) + 0.01 * rng.standard_normal((n1, n2))).astype(np.float32)
    alpha = 0.05
    x, tr, _ = ar.ar_restore(dev(g), h, alpha, 1.0, 6, True, f_true=dev(f.astype(np.float32)))
    xo, to, _ = O.restore(g.astype(np.float64), h, alpha, 1.0, 6, True,
                          f_true=f.astype(np.float32).astype(np.float64))
    assert rel_l2(x.cpu().numpy(), xo) <= tol_alpha(alpha)
    assert_trace_close(tr, to, tol_alpha(alpha))


def test_restore_past_one_wave_matches_oracle(ar):
    """1104 x 1536: too many tiles for one wave, so the stencils (the residual blur
    and the folding reblur) take their 64-row geometry; two iterations against the
    oracle, then the plain-mode stencil with the x update."""
    rng = np.random.default_rng(1104)
    n1, n2 = 1104, 1536
    h = rand_psf(rng, 7, 6)
    f = rng.uniform(0, 1, (n1, n2))
    g = (O.ar_blur(f, h) + 0.005 * rng.standard_normal((n1, n2))).astype(np.float32)
    f32 = f.astype(np.float32)
    for pc, alpha in ((True, 0.3), (False, 0.0)):
        x, tr, _ = ar.ar_restore(dev(g), h, alpha, 1.0, 2, pc, f_true=dev(f32))
        xo, to, _ = O.restore(g.astype(np.float64), h, alpha, 1.0, 2, pc,
                              f_true=f32.astype(np.float64))
        tol = tol_alpha(alpha) if pc else 1e-5
        assert rel_l2(x.cpu().numpy(), xo) <= tol
        assert_trace_close(tr, to, tol)


_BC_CODE = {"ar": O.BC_AR, "reflective": O.BC_REFLECTIVE, "periodic": O.BC_PERIODIC}


@pytest.mark.parametrize("pc,alpha,bc,n1,n2,psf,precision", [
    (True, 0.03, "ar", 64, 64, "config1", "fp32"),        # TMA stencils
    (False, 0.0, "ar", 64, 64, "config1", "fp32"),
    (True, 0.05, "reflective", 64, 64, "config1", "fp32"),
    (True, 0.05, "periodic", 64, 64, "config1", "fp32"),  # thread-loaded stencil (conv_fast_kernel)
    (False, 0.0, "periodic", 64, 64, "config1", "fp32"),
    (True, 0.05, "ar", 60, 66, "config1", "fp32"),        # n2 % 4 != 0: conv_fast_kernel
    (True, 0.1, "ar", 70, 72, "wide", "fp32"),            # q > 15: conv_generic_kernel
    (False, 0.0, "ar", 70, 72, "wide", "fp32"),
    (True, 0.03, "ar", 64, 64, "config1", "bf16x2"),      # two-plane contractions
])
def test_residual_norms_match_oracle(ar, pc, alpha, bc, n1, n2, psf, precision):
    """||g - A x_k||_F of every iterate k = 0 .. iters (the residual step of eq.
    DLandweberMeth), against the oracle's iterates, through each stencil kernel
    that carries the residual sum (TMA tiles, thread-loaded tiles, the generic
    kernel for q > 15) and both precisions.  x_k differs from the oracle's by at
    most tol ||x_k|| (rel-L2 per iterate), so the norms differ by at most
    ||A|| tol ||x_k|| plus the float32 rounding of r."""
    rng = np.random.default_rng(n1 * 13 + n2)
    if psf == "wide":
        h = rand_psf(rng, 17, 16)
    else:
        h = W.psf_config1()
    f = rng.uniform(0, 1, (n1, n2))
    code = _BC_CODE[bc]
    g = (O.blur_bc(f, h, code) + 0.01 * rng.standard_normal((n1, n2))).astype(np.float32)
    f = f.astype(np.float32)
    iters = 6
    x, tr, best, res = ar.ar_restore_residuals(dev(g), h, alpha, 1.0, iters, pc, f_true=dev(f),
                                               bc=bc, precision=precision)
    assert res.shape == (iters + 1,)
    g64 = g.astype(np.float64)
    tol = (tol_fast(alpha) if precision == "bf16x2" else tol_alpha(alpha)) if pc else 1e-5
    if bc == "periodic" and pc:
        tol *= 2            # the periodic solve sums two synthesised terms
    for k in range(iters + 1):
        xk = (np.zeros_like(g64) if k == 0 else O.restore_bc(g64, h, alpha, code, 1.0, k, pc)[0])
        want = np.linalg.norm(g64 - O.blur_bc(xk, h, code))
        assert abs(res[k] - want) <= 2 * tol * np.linalg.norm(xk) + 1e-5 * want, (k, res[k], want)
    xo, _, _ = O.restore_bc(g64, h, alpha, code, 1.0, iters, pc)
    assert rel_l2(x.cpu().numpy(), xo) <= tol


def test_restore_warm_start_and_in_place(ar):
    h = W.psf_config1()
    g, f = _workload(64, h, "blocks", 0, 0.01)
    gd = dev(g)
    x3, _, _ = ar.ar_restore(gd, h, 0.03, 1.0, 3, True)
    x = x3.clone()
    ar.ar_restore(gd, h, 0.03, 1.0, 3, True, x0=x, x_out=x)      # x0 == x_out
    x6, _, _ = ar.ar_restore(gd, h, 0.03, 1.0, 6, True)
    assert rel_l2(x.cpu().numpy(), x6.cpu().numpy().astype(np.float64)) <= 1e-6


def test_restore_zero_iterations(ar):
    h = W.psf_config1()
    g, f = _workload(64, h, "blocks", 0, 0.01)
    x, tr, best = ar.ar_restore(dev(g), h, 0.03, 1.0, 0, True, f_true=dev(f))
    assert torch.count_nonzero(x).item() == 0 and best == 0 and len(tr) == 0


def test_restore_bench_workload_full_length(ar):
    """The benchmarked call itself: ellipses 1024^2, 15x15 motion-blur PSF, 0.5%
    noise, alpha 0.3, tau 1, 50 D-Landweber iterations with the RRE trace.  Every
    iterate x_k (k = 1 .. 50, from k-iteration calls; the iteration is
    deterministic) against the oracle's, the RRE trace at every iterate and IT."""
    h = W.psf_config2()
    g, f = _workload(1024, h, "ellipses", 1, 0.005)
    iters = 50
    gd, fd = dev(g), dev(f)
    x, tr, best = ar.ar_restore(gd, h, 0.3, 1.0, iters, True, f_true=fd)
    xs = {iters: x.cpu().numpy()}
    for k in range(1, iters):
        xs[k] = ar.ar_restore(gd, h, 0.3, 1.0, k, True)[0].cpu().numpy()
    errs = {}

    def each(k, xk):
        errs[k] = rel_l2(xs[k], xk)

    xo, to, bo = O.restore(g.astype(np.float64), h, 0.3, 1.0, iters, True,
                           f_true=f.astype(np.float64), each=each)
    print({"bench_workload_max_rel_l2": max(errs.values()), "at": max(errs, key=errs.get)})
    assert len(errs) == iters
    assert max(errs.values()) <= 1e-5, errs
    assert_trace_close(tr, to, 1e-5)
    assert best == bo


def test_restore_flags_nonfinite_input(ar):
    h = W.psf_config1()
    g, f = _workload(64, h, "blocks", 0, 0.01)
    g[10, 10] = np.nan
    with pytest.raises(ar.ARError) as ei:
        ar.ar_restore(dev(g), h, 0.03, 1.0, 2, True)
    assert ei.value.name == "AR_ERR_NONFINITE"


def test_restore_rejects_unnormalized_psf(ar):
    h = W.psf_config1() * 1.1
    g = torch.zeros(64, 64, device="cuda")
    with pytest.raises(ar.ARError) as ei:
        ar.ar_restore(g, h, 0.03, 1.0, 2, True)
    assert ei.value.name == "AR_ERR_PSF_NOT_NORMALIZED"


FAST_SOLVE_CASES = [(64, 64, 4, 4, 0.03), (130, 257, 7, 7, 0.3), (1024, 1024, 7, 7, 0.3), (9, 8, 2, 1, 0.1)]


@pytest.mark.parametrize("n1,n2,q1,q2,alpha", FAST_SOLVE_CASES)
def test_solve_bf16x2_mode_matches_oracle(ar, n1, n2, q1, q2, alpha):
    rng = np.random.default_rng(n1 + 3 * n2 + q1)
    h = rand_psf(rng, q1, q2)
    y = rng.standard_normal((n1, n2)).astype(np.float32)
    P = ar.ar_symprec_setup(h, n1, n2, alpha, precision="bf16x2")
    z = ar.ar_symprec_solve(P, dev(y)).cpu().numpy()
    want = O.symprec_solve(O.symprec_setup(h, n1, n2, alpha), y.astype(np.float64))
    err = rel_l2(z, want)
    assert err <= tol_fast(alpha)
    # the fast mode is really a different (coarser) arithmetic than the default
    P3 = ar.ar_symprec_setup(h, n1, n2, alpha)
    z3 = ar.ar_symprec_solve(P3, dev(y)).cpu().numpy()
    assert rel_l2(z3, want) <= tol_alpha(alpha)
    P.close()
    P3.close()


@pytest.mark.parametrize("n,psf,scene,cidx,nu,alpha,iters", [
    (64, "config1", "blocks", 0, 0.01, 0.03, 20),
    (200, "config2", "ellipses", 1, 0.005, 0.3, 10),
])
def test_restore_bf16x2_mode_matches_oracle(ar, n, psf, scene, cidx, nu, alpha, iters):
    h = W.psf_named(psf)
    g, f = _workload(n, h, scene, cidx, nu)
    x, tr, best = ar.ar_restore(dev(g), h, alpha, 1.0, iters, True, f_true=dev(f),
                                precision="bf16x2")
    xo, to, bo = O.restore(g.astype(np.float64), h, alpha, 1.0, iters, True,
                           f_true=f.astype(np.float64))
    tol = tol_fast(alpha)
    assert rel_l2(x.cpu().numpy(), xo) <= tol
    assert_trace_close(tr, to, tol)


def test_unknown_precision_is_rejected(ar):
    import ctypes
    h = np.ascontiguousarray(W.psf_config1())
    out = ctypes.c_void_p()
    st = ar.lib().ar_symprec_setup_ex(h.ctypes.data, 4, 4, 16, 16, 0.1, 7, None, ctypes.byref(out))
    assert st == 1 and out.value is None
