"""Batched restoration (one CUDA graph over many uneven images) against
per-image ar_restore_ex calls and, for one image, the FP64 oracle."""

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


def _images(sides, seed):
    rng = np.random.default_rng(seed)
    ims = []
    for n1, n2, q in sides:
        h = W.psf_random(q, q, rng)
        f = rng.uniform(0, 1, (n1, n2))
        g = O.ar_blur(f, h) + 0.005 * rng.standard_normal((n1, n2))
        ims.append({"g": torch.from_numpy(g.astype(np.float32)).cuda(), "psf": h, "alpha": 1.0,
                    "f_true": torch.from_numpy(f.astype(np.float32)).cuda(),
                    "x_out": torch.empty(n1, n2, device="cuda"), "f64": f, "g64": g.astype(np.float32)})
    return ims


SIDES = [(64, 96, 2), (128, 128, 7), (37, 53, 3), (200, 120, 10), (96, 64, 15), (130, 257, 4),
         (3, 5, 0), (64, 64, 4)]


@pytest.mark.parametrize("precondition,precision", [(True, "fp32"), (True, "bf16x2"), (False, "fp32")])
def test_batch_equals_per_image_restore(ar, precondition, precision):
    if not precondition:
        sides = SIDES
    else:
        sides = [s for s in SIDES if min(s[0], s[1]) >= 2 * s[2] + 3 and min(s[0], s[1]) >= 3]
    ims = _images(sides, 11)
    iters = 7
    B = ar.Batch(ims, tau=1.0, iters=iters, precondition=precondition, precision=precision,
                 concurrency=3)
    for run in range(2):                      # replays must reproduce the same result
        B.run()
        tr, best, kpr = B.results()
        assert kpr > 0
        for j, im in enumerate(ims):
            x, trj, bj = ar.ar_restore(im["g"], im["psf"], im["alpha"], 1.0, iters, precondition,
                                       f_true=im["f_true"], precision=precision)
            xb = im["x_out"].cpu().numpy()
            np.testing.assert_array_equal(xb, x.cpu().numpy())
            np.testing.assert_allclose(tr[j], trj, rtol=1e-12)
            assert best[j] == bj
    B.close()


def test_batch_image_matches_oracle(ar):
    ims = _images([(96, 80, 5), (64, 64, 4)], 12)
    B = ar.Batch(ims, iters=5, precondition=True, concurrency=2)
    B.run()
    tr, best, _ = B.results()
    im = ims[0]
    xo, to, _ = O.restore(im["g64"].astype(np.float64), im["psf"], 1.0, 1.0, 5, True,
                          f_true=im["f_true"].cpu().numpy().astype(np.float64))
    x = im["x_out"].cpu().numpy().astype(np.float64)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-5
    np.testing.assert_allclose(tr[0], to, rtol=1e-5)
    B.close()


def test_batch_rejects_aliasing_outputs(ar):
    ims = _images([(32, 32, 2), (32, 32, 2)], 13)
    ims[1]["x_out"] = ims[0]["x_out"]
    with pytest.raises(ar.ARError) as ei:
        ar.Batch(ims, iters=2)
    assert ei.value.name == "AR_ERR_ALIAS"
