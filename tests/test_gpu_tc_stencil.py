"""GPU parity of the tensor-core stencil (AR_STENCIL_F16X2) against the FP64 oracle.

Error bound of one output y_i = sum_s h_s xt_{i-s} (eq. modello_discreto over
the extension of Section 2.2 / 2.1), derived from the arithmetic: the tile's
input and the PSF are scaled by powers of two (exact) and split into fp16
parts carrying 11 + 11 significant bits, so each factor is represented to
2^-22 of itself and the dropped product x_lo h_lo is below 2^-22 of the term:
about 3 * 2^-22 per term.  The products are exact in the float32 accumulator;
each output takes at most 2 (q1 + 1) MMA accumulations per plane pair plus the
final P + R sum, under 61 float32 roundings (2^-24 each) of partial sums
bounded by M_i = sum_s |h_s| |xt_{i-s}|.  Together below 2^-17 M_i, the bound
checked element by element (the float32 stencil's worst case, 225 sequential
roundings at 15 x 15, is 1.3e-5 M_i).  The scaling is per tile: a factor whose
magnitude is far below its tile's (or PSF's) largest falls into fp16's
subnormal range, where its absolute error is at most 2^-39 of that largest
(2^-25 in units where the largest is at least 2^14).  So the full bound adds
2^-36 K max|h| B_i, K = (2q1+1)(2q2+1) taps and B_i the largest |xt| in the
halo box of the 128 x 64 tile holding output i (rows r0 - 8 .. r0 + 135,
columns c0 - 8 .. c0 + 71 of the extension): negligible for images of
moderate dynamic range, and the limit for a tile whose halo holds values
2^28 times its own.
"""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1211_0393_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TC_BOUND = 2.0 ** -17
BCS = {"ar": O.BC_AR, "reflective": O.BC_REFLECTIVE, "periodic": O.BC_PERIODIC}


@pytest.fixture(scope="module")
def ar():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0393_gb300 import ar as mod

    mod.lib()
    return mod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def rand_psf(rng, q1, q2):
    h = rng.uniform(0.0, 1.0, size=(2 * q1 + 1, 2 * q2 + 1))
    return h / h.sum()


def magnitude(x, h, bc):
    """M_i = sum_s |h_s| |xt_{i-s}| over the oracle's extension of x."""
    h = np.abs(np.asarray(h, np.float64))
    q1, q2 = O.psf_support(h)
    n1, n2 = x.shape
    xp = np.abs(O.pad_bc(np.asarray(x, np.float64), q1, q2, BCS[bc]))
    m = np.zeros((n1, n2))
    for s1 in range(-q1, q1 + 1):
        for s2 in range(-q2, q2 + 1):
            m += h[s1 + q1, s2 + q2] * xp[q1 - s1:q1 - s1 + n1, q2 - s2:q2 - s2 + n2]
    return m


def tile_box_max(x, h, bc):
    """B_i: the largest |xt| over the halo box of the output tile holding i."""
    q1, q2 = O.psf_support(h)
    n1, n2 = x.shape
    xp = np.abs(O.pad_bc(np.asarray(x, np.float64), q1, q2, BCS[bc]))
    b = np.zeros((n1, n2))
    for r0 in range(0, n1, 128):
        for c0 in range(0, n2, 64):
            # box rows r0 - 8 .. r0 + 135 -> xp rows shifted by q1, clipped to the extension
            ra, rb = max(0, r0 - 8 + q1), min(n1 + 2 * q1, r0 + 136 + q1)
            ca, cb = max(0, c0 - 8 + q2), min(n2 + 2 * q2, c0 + 72 + q2)
            b[r0:r0 + 128, c0:c0 + 64] = xp[ra:rb, ca:cb].max()
    return b


def check_stencil(ar, x, h, bc, norm_check=True):
    xd, hd = dev(x), dev(h)
    for fn, flip in ((ar.ar_blur_apply, False), (ar.ar_reblur_apply, True)):
        got = fn(xd, hd, bc=bc, stencil="f16x2").cpu().numpy().astype(np.float64)
        hh = h.astype(np.float64)
        hh = hh[::-1, ::-1] if flip else hh
        want = O.blur_bc(x.astype(np.float64), hh, BCS[bc])
        bound = TC_BOUND * magnitude(x, hh, bc)
        bound += 2.0 ** -36 * hh.size * np.max(np.abs(hh)) * tile_box_max(x, hh, bc)
        err = np.abs(got - want)
        assert np.all(err <= bound), float(np.max(err / np.maximum(bound, 1e-300)))
        if norm_check:
            assert rel_l2(got, want) <= 2e-6


TC_CASES = [
    # n1, n2, q1, q2, bc: one tile with every border, ragged row and column tiles,
    # the largest support (q = 8) and q = n - 1, the bench geometry, Reflective BCs
    (64, 64, 4, 4, "ar"),
    (3, 4, 1, 1, "ar"),
    (9, 12, 8, 8, "ar"),
    (130, 200, 7, 7, "ar"),
    (257, 132, 8, 8, "ar"),
    (128, 64, 0, 0, "ar"),
    (300, 512, 3, 8, "ar"),
    (1000, 1028, 7, 7, "ar"),
    (1024, 1024, 7, 7, "ar"),
    (77, 300, 2, 6, "reflective"),
    (65, 68, 5, 3, "reflective"),
    # more tiles than SMs: every CTA walks several tiles through both plane and
    # accumulator sets (512 and 216 tiles), with ragged last rows and columns
    (2048, 2048, 7, 7, "ar"),
    (1500, 1100, 4, 6, "reflective"),
]


@pytest.mark.parametrize("n1,n2,q1,q2,bc", TC_CASES)
def test_tc_stencil_matches_oracle(ar, n1, n2, q1, q2, bc):
    rng = np.random.default_rng(n1 * 11 + n2 * 5 + q1 * 3 + q2)
    h = rand_psf(rng, q1, q2).astype(np.float32)
    x = rng.uniform(0, 1, (n1, n2)).astype(np.float32)
    check_stencil(ar, x, h, bc)


def test_tc_stencil_signed_psf_and_dynamic_range(ar):
    """A PSF with negative taps (not normalised) and an image whose tiles span
    magnitudes from 1e-30 to 1e30, negative values and an all-zero tile: the
    per-tile power-of-two scaling keeps each tile's error relative to its own
    largest magnitude."""
    rng = np.random.default_rng(77)
    n1, n2 = 384, 256
    h = rng.standard_normal((15, 13)).astype(np.float32)
    x = rng.standard_normal((n1, n2))
    x[:128, :64] *= 1e30
    x[128:256, 64:128] *= 1e-30
    x[256:, 128:192] = 0.0
    x[:128, 192:] = np.abs(x[:128, 192:]) * 3e-5
    check_stencil(ar, x.astype(np.float32), h, "ar", norm_check=False)


def test_tc_stencil_bench_psf_against_fp32_stencil(ar):
    """The bench PSF at 1024^2: the two stencil arithmetics agree within the
    sum of their bounds, element by element."""
    n = 1024
    h = W.psf_config2().astype(np.float32)
    x = np.random.default_rng(3).uniform(0, 1, (n, n)).astype(np.float32)
    xd, hd = dev(x), dev(h)
    m = magnitude(x, h, "ar")
    a = ar.ar_blur_apply(xd, hd, stencil="f16x2").cpu().numpy().astype(np.float64)
    b = ar.ar_blur_apply(xd, hd).cpu().numpy().astype(np.float64)
    assert np.all(np.abs(a - b) <= (TC_BOUND + 225 * 2.0 ** -24) * m)


@pytest.mark.parametrize("n1,n2,q1,q2,bc,why", [
    (64, 64, 2, 2, "periodic", "periodic BCs"),
    (64, 64, 9, 9, "ar", "q > 8"),
    (64, 66, 2, 2, "ar", "n2 % 4 != 0"),
])
def test_tc_stencil_falls_back_to_fp32(ar, n1, n2, q1, q2, bc, why):
    """Where the tensor-core path does not apply the float32 stencil runs:
    identical results."""
    rng = np.random.default_rng(n2 + q1)
    h = dev(rand_psf(rng, q1, q2))
    x = dev(rng.uniform(0, 1, (n1, n2)))
    for fn in (ar.ar_blur_apply, ar.ar_reblur_apply):
        assert torch.equal(fn(x, h, bc=bc, stencil="f16x2"), fn(x, h, bc=bc)), why


def test_tc_stencil_rejects_unknown_arithmetic(ar):
    x = torch.zeros(16, 16, device="cuda")
    h = torch.ones(3, 3, device="cuda") / 9
    y = torch.empty_like(x)
    st = ar.lib().ar_blur_apply_ex(x.data_ptr(), y.data_ptr(), 16, 16, h.data_ptr(), 1, 1, 0, 3,
                                   None)
    assert ar.STATUS[st] == "AR_ERR_INVALID_ARG"


def _workload(n, psf, scene, cidx, nu):
    q1, q2 = O.psf_support(psf)
    ext, f, e = W.make_inputs(n, n, psf, scene, cidx)
    g = W.add_noise(W.crop(O.ar_blur(ext, psf), q1, q2), e, nu)
    return g.astype(np.float32), f.astype(np.float32)


def tol_alpha(alpha):
    return max(1e-5, 3 * 2.0 ** -24 / alpha)


@pytest.mark.parametrize("n,psf,scene,cidx,nu,alpha,iters,pc", [
    (64, "config1", "blocks", 0, 0.01, 0.03, 20, True),
    (64, "config1", "blocks", 0, 0.01, 0.0, 30, False),
    (200, "config2", "ellipses", 1, 0.005, 0.3, 10, True),
    (200, "config2", "ellipses", 1, 0.005, 0.0, 10, False),
])
def test_restore_tc_stencil_matches_oracle(ar, n, psf, scene, cidx, nu, alpha, iters, pc):
    """Restorations with both stencils on the tensor cores (the residual blur,
    the folding reblur or the x update of plain mode) against the oracle, at the
    float32 path's tolerances."""
    h = W.psf_named(psf)
    g, f = _workload(n, h, scene, cidx, nu)
    x, tr, best = ar.ar_restore(dev(g), h, alpha, 1.0, iters, pc, f_true=dev(f), stencil="f16x2")
    xo, to, bo = O.restore(g.astype(np.float64), h, alpha, 1.0, iters, pc,
                           f_true=f.astype(np.float64))
    tol = tol_alpha(alpha) if pc else 1e-5
    assert rel_l2(x.cpu().numpy(), xo) <= tol
    assert np.all(np.abs(np.asarray(tr) - to) <= tol * (1.0 + to))


@pytest.mark.parametrize("n1,n2,q1,q2", [(40, 40, 3, 3), (72, 120, 7, 5), (36, 52, 8, 8),
                                         (136, 264, 6, 2)])
def test_restore_tc_folded_input_shapes(ar, n1, n2, q1, q2):
    """The folding reblur's cluster pairs: mirror tiles left of the image,
    ragged column pairs, the widest tensor-core halo, several row tiles."""
    rng = np.random.default_rng(n1 * 31 + n2 + q1)
    h = rand_psf(rng, q1, q2)
    f = rng.uniform(0, 1, (n1, n2))
    g = (O.ar_blur(f, h) + 0.01 * rng.standard_normal((n1, n2))).astype(np.float32)
    alpha = 0.05
    x, tr, _ = ar.ar_restore(dev(g), h, alpha, 1.0, 6, True, f_true=dev(f.astype(np.float32)),
                             stencil="f16x2")
    xo, to, _ = O.restore(g.astype(np.float64), h, alpha, 1.0, 6, True,
                          f_true=f.astype(np.float32).astype(np.float64))
    assert rel_l2(x.cpu().numpy(), xo) <= tol_alpha(alpha)


@pytest.mark.parametrize("pc,alpha,bc", [(True, 0.03, "ar"), (False, 0.0, "ar"),
                                         (True, 0.05, "reflective")])
def test_residual_norms_tc_stencil(ar, pc, alpha, bc):
    """||g - A x_k|| summed in the tensor-core blur's residual epilogue."""
    n1 = n2 = 64
    rng = np.random.default_rng(13)
    h = W.psf_config1()
    f = rng.uniform(0, 1, (n1, n2))
    code = BCS[bc]
    g = (O.blur_bc(f, h, code) + 0.01 * rng.standard_normal((n1, n2))).astype(np.float32)
    iters = 5
    x, tr, best, res = ar.ar_restore_residuals(dev(g), h, alpha, 1.0, iters, pc,
                                               f_true=dev(f.astype(np.float32)), bc=bc,
                                               stencil="f16x2")
    g64 = g.astype(np.float64)
    tol = tol_alpha(alpha) if pc else 1e-5
    for k in range(iters + 1):
        xk = (np.zeros_like(g64) if k == 0 else O.restore_bc(g64, h, alpha, code, 1.0, k, pc)[0])
        want = np.linalg.norm(g64 - O.blur_bc(xk, h, code))
        assert abs(res[k] - want) <= 2 * tol * np.linalg.norm(xk) + 1e-5 * want, (k, res[k], want)


def test_restore_tc_stencil_bench_workload(ar):
    """The bench workload (1024^2, 15 x 15 motion PSF, alpha 0.3, 50 iterations)
    with the tensor-core stencils: sampled iterates against the oracle's at the
    float32 path's 1e-5, the RRE trace, and IT."""
    h = W.psf_config2()
    g, f = _workload(1024, h, "ellipses", 1, 0.005)
    iters = 50
    gd, fd = dev(g), dev(f)
    x, tr, best = ar.ar_restore(gd, h, 0.3, 1.0, iters, True, f_true=fd, stencil="f16x2")
    ks = (1, 2, 7, 20, iters)
    xs = {k: ar.ar_restore(gd, h, 0.3, 1.0, k, True, stencil="f16x2")[0].cpu().numpy()
          for k in ks if k != iters}
    xs[iters] = x.cpu().numpy()
    errs = {}

    def each(k, xk):
        if k in xs:
            errs[k] = rel_l2(xs[k], xk)

    xo, to, bo = O.restore(g.astype(np.float64), h, 0.3, 1.0, iters, True,
                           f_true=f.astype(np.float64), each=each)
    print({"tc_stencil_bench_rel_l2": errs})
    assert len(errs) == len(ks)
    assert max(errs.values()) <= 1e-5, errs
    assert np.all(np.abs(np.asarray(tr) - to) <= 1e-5 * (1.0 + to))
    assert best == bo


@pytest.mark.parametrize("pc,alpha", [(True, 0.3), (False, 0.0)])
def test_restore_tc_stencil_past_one_wave(ar, pc, alpha):
    """1104 x 1536: 216 blur tiles and 108 folding units, more than the SMs and
    the co-resident clusters, so the persistent loops take several tiles (units)
    each; two iterations against the oracle."""
    rng = np.random.default_rng(1104)
    n1, n2 = 1104, 1536
    h = rand_psf(rng, 7, 6)
    f = rng.uniform(0, 1, (n1, n2))
    g = (O.ar_blur(f, h) + 0.005 * rng.standard_normal((n1, n2))).astype(np.float32)
    f32 = f.astype(np.float32)
    x, tr, _ = ar.ar_restore(dev(g), h, alpha, 1.0, 2, pc, f_true=dev(f32), stencil="f16x2")
    xo, to, _ = O.restore(g.astype(np.float64), h, alpha, 1.0, 2, pc,
                          f_true=f32.astype(np.float64))
    tol = tol_alpha(alpha) if pc else 1e-5
    assert rel_l2(x.cpu().numpy(), xo) <= tol
    assert np.all(np.abs(np.asarray(tr) - to) <= tol * (1.0 + to))



@pytest.mark.parametrize("n,q", [(1024, 7), (4096, 7), (512, 1)])
def test_auto_stencil_is_one_of_the_two(ar, n, q):
    """AR_STENCIL_AUTO runs one of the two arithmetics, chosen by a timing the
    first time the shape is seen: its result equals one of theirs bit for bit,
    and a second call makes the same choice."""
    rng = np.random.default_rng(n + q)
    x = dev(rng.uniform(0, 1, (n, n)))
    h = dev(rand_psf(rng, q, q))
    a32 = ar.ar_blur_apply(x, h)
    atc = ar.ar_blur_apply(x, h, stencil="f16x2")
    got1 = ar.ar_blur_apply(x, h, stencil="auto")
    got2 = ar.ar_blur_apply(x, h, stencil="auto")
    assert torch.equal(got1, a32) or torch.equal(got1, atc)
    assert torch.equal(got1, got2)


def test_restore_auto_stencil_is_one_of_the_two(ar):
    h = W.psf_config1()
    g, f = _workload(64, h, "blocks", 0, 0.01)
    gd, fd = dev(g), dev(f)
    outs = [ar.ar_restore(gd, h, 0.03, 1.0, 5, True, f_true=fd, stencil=st)[0].clone()
            for st in ("fp32", "f16x2", "auto")]
    assert torch.equal(outs[2], outs[0]) or torch.equal(outs[2], outs[1])
