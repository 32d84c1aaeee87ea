"""Precision modes on the 2048^2 workload (ellipses, 21x21 asymmetric Gaussian
PSF, 1% noise; alpha 0.1, the smallest half-decade value for which tau = 1 is
stable with this PSF): the error of each of the first ten iterates against the
FP64 oracle, for the float32-grade contractions (bf16x3, six products) and the
fast mode (bf16x2, three products).  Bounds as in test_gpu_parity:
tol(alpha) = max(1e-5, 3 * 2^-24 / alpha), tol_fast(alpha) = max(1e-4, 3 * 2^-16 / alpha)."""

import json

import numpy as np
import pytest
import torch

import oracle as O
from paper_1211_0393_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ALPHA = 0.1
STEPS = 10


@pytest.fixture(scope="module")
def ar():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0393_gb300 import ar as mod

    mod.lib()
    return mod


@pytest.fixture(scope="module")
def config4():
    wl = W.WORKLOADS["ellipses2048_gauss21"]
    n1, n2 = wl["n"]
    h = W.psf_config4()
    q1, q2 = O.psf_support(h)
    ext, f, e = W.make_inputs(n1, n2, h, "ellipses", wl["config_idx"])
    g = W.add_noise(W.crop(O.ar_blur(ext, h), q1, q2), e, wl["nu"]).astype(np.float32)
    # the oracle's first iterates (eq. DLandweberMeth, x_0 = 0)
    prec = O.symprec_setup(h, n1, n2, ALPHA)
    x = np.zeros((n1, n2))
    xs = []
    g64 = g.astype(np.float64)
    for _ in range(STEPS):
        x = x + O.symprec_solve(prec, O.ar_reblur(g64 - O.ar_blur(x, h), h))
        xs.append(x.copy())
    return h, g, f.astype(np.float32), xs


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision,tol", [
    ("fp32", max(1e-5, 3 * 2.0 ** -24 / ALPHA)),
    ("bf16x2", max(1e-4, 3 * 2.0 ** -16 / ALPHA)),
])
def test_config4_error_per_step(ar, config4, precision, tol):
    h, g, f, xs = config4
    gd = torch.from_numpy(g).cuda()
    errs = []
    for k in range(1, STEPS + 1):
        x, _, _ = ar.ar_restore(gd, h, ALPHA, 1.0, k, True, precision=precision)
        errs.append(rel_l2(x.cpu().numpy(), xs[k - 1]))
    print(json.dumps({"workload": "ellipses2048_gauss21", "precision": precision,
                      "alpha": ALPHA, "rel_l2_vs_oracle_per_step": errs}))
    assert max(errs) <= tol
