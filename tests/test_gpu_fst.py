"""The FFT-style AR transform (AR_PRECISION_FFT) against the FP64 oracle.

Every 1D transform of Theorem 1 is its boundary terms plus a DST-I taken from
one real DFT of length n - 1, split by Good and Thomas into two small dense
DFTs (n = 64: 63 = 7 x 9; 256: 15 x 17; 1024: 31 x 33; 2048: 23 x 89; 65: one
64-point DFT).  All sums are float32 (A_0 and the odd coefficients' prefix
float64).  The odd DST coefficients are prefix sums of up to m/2 DFT outputs, so
their rounding errors add like a random walk (sqrt(m/2) ~ 32 at m = 2048, cut by
the mean removal and the bridge correction to about twice the dense path's):
a float32 emulation of one 1D analysis at m = 2048 gives 1.8e-6 (random rows) and
2.3e-6 (smooth rows) against 0.7e-6 and 1.2e-6 for a dense float32 product.  The
bound is therefore tol_fft(alpha) = 2 tol(alpha)."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1211_0393_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def tol_alpha(alpha):
    return max(1e-5, 3 * U32 / alpha)


def tol_fft(alpha):
    return 2 * tol_alpha(alpha)


@pytest.fixture(scope="module")
def ar():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0393_gb300 import ar as mod

    mod.lib()
    return mod


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def rand_psf(rng, q1, q2):
    h = rng.uniform(0.0, 1.0, size=(2 * q1 + 1, 2 * q2 + 1))
    return h / h.sum()


@pytest.mark.parametrize("n1,n2,q,alpha", [(64, 64, 4, 0.03), (65, 256, 3, 0.1), (256, 64, 7, 0.3),
                                           (1024, 1024, 7, 0.3), (2048, 2048, 10, 0.1)])
def test_fft_solve_matches_oracle(ar, n1, n2, q, alpha):
    rng = np.random.default_rng(n1 + n2 + q)
    h = rand_psf(rng, q, q)
    y = rng.standard_normal((n1, n2)).astype(np.float32)
    P = ar.ar_symprec_setup(h, n1, n2, alpha, precision="fft")
    assert ar.ar_symprec_precision(P) == "fft"
    yd = torch.from_numpy(y).cuda()
    z = ar.ar_symprec_solve(P, yd).cpu().numpy()
    want = O.symprec_solve(O.symprec_setup(h, n1, n2, alpha), y.astype(np.float64))
    assert rel(z, want) <= tol_fft(alpha)
    ar.ar_symprec_solve(P, yd, yd)                           # in place
    assert rel(yd.cpu().numpy(), want) <= tol_fft(alpha)
    P.close()


@pytest.mark.parametrize("n,psf,scene,cidx,nu,alpha,iters", [
    (64, "config1", "blocks", 0, 0.01, 0.03, 20),
    (1024, "config2", "ellipses", 1, 0.005, 0.3, 5),
])
def test_fft_restore_matches_oracle(ar, n, psf, scene, cidx, nu, alpha, iters):
    h = W.psf_named(psf)
    q1, q2 = O.psf_support(h)
    ext, f, e = W.make_inputs(n, n, h, scene, cidx)
    g = W.add_noise(W.crop(O.ar_blur(ext, h), q1, q2), e, nu).astype(np.float32)
    f = f.astype(np.float32)
    x, tr, best = ar.ar_restore(torch.from_numpy(g).cuda(), h, alpha, 1.0, iters, True,
                                f_true=torch.from_numpy(f).cuda(), precision="fft")
    xo, to, bo = O.restore(g.astype(np.float64), h, alpha, 1.0, iters, True,
                           f_true=f.astype(np.float64))
    assert rel(x.cpu().numpy(), xo) <= tol_fft(alpha)
    assert np.all(np.abs(tr - to) <= tol_fft(alpha) * (1 + to))


def test_auto_picks_a_measured_transform(ar):
    h = W.psf_config2()
    for n in (2048, 1024):
        P = ar.ar_symprec_setup(h, n, n, 0.3, precision="auto")
        assert ar.ar_symprec_precision(P) in ("fft", "fp32")
        P.close()
    # no Good-Thomas split (527 - 1 = 2 x 263): the dense transform
    P = ar.ar_symprec_setup(h, 527, 64, 0.3, precision="auto")
    assert ar.ar_symprec_precision(P) == "fp32"
    P.close()
    # comparison BCs keep their dense transforms
    P = ar.ar_symprec_setup(h, 64, 64, 0.3, precision="auto", bc="reflective")
    assert ar.ar_symprec_precision(P) == "fp32"
    P.close()


def test_fft_rejects_what_it_cannot_do(ar):
    h = W.psf_config2()
    for kw in ({"n1": 527, "n2": 64}, {"n1": 64, "n2": 64, "bc": "reflective"}):
        with pytest.raises(ar.ARError) as ei:
            ar.ar_symprec_setup(h, kw["n1"], kw["n2"], 0.3, precision="fft", bc=kw.get("bc", "ar"))
        assert ei.value.name == "AR_ERR_UNSUPPORTED"
