"""Batched restoration (one persistent stencil launch and four grouped
contractions per iteration for many uneven images) against per-image
ar_restore_ex calls and the FP64 oracle.

The stencils of the batch are the single-image stencils' code, so plain
Landweber (stencils only) is bit-identical to per-image calls.  Preconditioned,
the batch always runs the last product in parity-paired clusters (the
single-image loop only where they fit in one wave), a different float32
rounding of the same transform: both are within the per-iterate bound
tol(alpha) of the exact iterate, so within 2 tol(alpha) of each other (bf16x2:
2 tol_fast)."""

import numpy as np
import pytest
import torch

import oracle as O
from paper_1211_0393_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def tol_alpha(alpha):
    return max(1e-5, 3 * U32 / alpha)


def tol_fast(alpha):
    return max(1e-4, 3 * 2.0 ** -16 / alpha)


@pytest.fixture(scope="module")
def ar():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1211_0393_gb300 import ar as mod

    mod.lib()
    return mod


def _images(sides, seed, alpha=0.5):
    rng = np.random.default_rng(seed)
    ims = []
    for n1, n2, q in sides:
        h = W.psf_random(q, q, rng)
        f = rng.uniform(0, 1, (n1, n2))
        g = O.ar_blur(f, h) + 0.005 * rng.standard_normal((n1, n2))
        ims.append({"g": torch.from_numpy(g.astype(np.float32)).cuda(), "psf": h, "alpha": alpha,
                    "f_true": torch.from_numpy(f.astype(np.float32)).cuda(),
                    "x_out": torch.empty(n1, n2, device="cuda"), "f64": f, "g64": g.astype(np.float32)})
    return ims


# n2 % 4 == 0 (TMA rows), q <= 15; sizes from one tile to several waves of tiles,
# supports from 3x3 to 31x31, a small image whose tiles are all border tiles
SIDES = [(64, 96, 2), (128, 128, 7), (37, 52, 3), (200, 120, 10), (96, 64, 15), (130, 256, 4),
         (5, 8, 1), (64, 64, 4), (300, 196, 12)]


def rel(a, b):
    return float(np.linalg.norm(a.astype(np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precondition,precision", [(True, "fp32"), (True, "bf16x2"), (False, "fp32")])
def test_batch_matches_per_image_restore(ar, precondition, precision):
    sides = SIDES if not precondition else [s for s in SIDES if min(s[0], s[1]) >= 2 * s[2] + 3]
    ims = _images(sides, 11)
    iters = 7
    B = ar.Batch(ims, tau=1.0, iters=iters, precondition=precondition, precision=precision)
    tol = (tol_fast(0.5) if precision == "bf16x2" else tol_alpha(0.5)) if precondition else 0.0
    first = None
    for run in range(2):                      # replays must reproduce the same result
        B.run()
        tr, best, kpr = B.results()
        assert 0 < kpr <= 2 * len(ims) + 5 * iters + 1
        xs = [im["x_out"].clone() for im in ims]
        if first is None:
            first = xs
        else:
            assert all(torch.equal(a, b) for a, b in zip(first, xs))
        for j, im in enumerate(ims):
            x, trj, bj = ar.ar_restore(im["g"], im["psf"], im["alpha"], 1.0, iters, precondition,
                                       f_true=im["f_true"], precision=precision)
            xb = xs[j].cpu().numpy()
            if precondition:
                assert rel(xb, x.cpu().numpy().astype(np.float64)) <= 2 * tol, j
                assert np.all(np.abs(tr[j] - trj) <= 2 * tol * (1 + trj)), j
            else:
                np.testing.assert_array_equal(xb, x.cpu().numpy())
                # the RRE sums group float32 partials of a thread's rows (at most 18
                # squares, relative error <= 18 2^-24) by the tile geometry
                np.testing.assert_allclose(tr[j], trj, rtol=18 * U32)
                assert best[j] == bj
    B.close()


def test_batch_images_match_oracle(ar):
    sides = [(96, 80, 5), (64, 64, 4), (130, 100, 9), (48, 200, 2)]
    ims = _images(sides, 12)
    iters = 5
    B = ar.Batch(ims, iters=iters, precondition=True)
    B.run()
    tr, best, _ = B.results()
    for j, im in enumerate(ims):
        xo, to, _ = O.restore(im["g64"].astype(np.float64), im["psf"], im["alpha"], 1.0, iters,
                              True, f_true=im["f_true"].cpu().numpy().astype(np.float64))
        x = im["x_out"].cpu().numpy()
        assert rel(x, xo) <= tol_alpha(im["alpha"]), j
        assert np.all(np.abs(tr[j] - to) <= tol_alpha(im["alpha"]) * (1 + to)), j
    B.close()


def test_batch_autotuner_reports_its_candidates(ar):
    ims = _images([(128, 128, 7), (256, 192, 3), (64, 64, 15)], 14)
    B = ar.Batch(ims, iters=4, precondition=True, tuning=0)
    t = B.tuning()
    assert len(t["candidates"]) >= 2
    best = min(t["candidates"], key=lambda c: c["ms_3_iters"])
    assert (best["geometry"], best["ctas_per_sm"]) == (t["geometry"], t["ctas_per_sm"])
    B.run()
    B.results()
    assert t["folded_input"] and t["paired_last_product"]
    B2 = ar.Batch(ims, iters=4, precondition=True, tuning=1)
    t2 = B2.tuning()
    assert (t2["geometry"], t2["ctas_per_sm"], t2["candidates"]) == ("64-row", 1, [])
    B2.close()
    B.close()


def test_batch_rejects_aliasing_outputs(ar):
    ims = _images([(32, 32, 2), (32, 32, 2)], 13)
    ims[1]["x_out"] = ims[0]["x_out"]
    with pytest.raises(ar.ARError) as ei:
        ar.Batch(ims, iters=2)
    assert ei.value.name == "AR_ERR_ALIAS"


def test_batch_rejects_unsupported_shapes(ar):
    ims = _images([(32, 30, 2)], 15)           # n2 % 4 != 0: the batched stencil's TMA rows
    with pytest.raises(ar.ARError) as ei:
        ar.Batch(ims, iters=2)
    assert ei.value.name == "AR_ERR_UNSUPPORTED"


def test_full_batch_configuration_sampled_images_match_oracle(ar):
    """The benchmarked batch configuration itself: all 96 images (sides from
    {128..1024} per axis, own PSF 5x5..31x31, 0.5% noise, each PSF's alpha the
    smallest stable half-decade value), 50 iterations, autotuned, in one batch.
    The three smallest images are compared with the FP64 oracle's 50-iteration
    restorations (inputs blurred by the oracle), iterate and RRE trace."""
    import importlib.util
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_for_alpha", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    argv, sys.argv = sys.argv, ["bench.py"]
    try:
        spec.loader.exec_module(bench)
    finally:
        sys.argv = argv
    iters = 50
    ims = []
    for sp in W.batch_specs(96):
        ext, f, e = W.batch_inputs(sp)
        h = sp["psf"]
        q1, q2 = O.psf_support(h)
        n = sp["n1"] * sp["n2"]
        small = n <= 128 * 192
        # the oracle blurs the small images it checks; the rest only need to be run
        if small:
            gc = W.crop(O.ar_blur(ext, h), q1, q2)
        else:
            gc = W.crop(ar.ar_blur_apply(torch.from_numpy(ext.astype(np.float32)).cuda(),
                                         torch.from_numpy(h.astype(np.float32)).cuda())
                        .cpu().numpy().astype(np.float64), q1, q2)
        g = W.add_noise(gc, e, 0.005).astype(np.float32)
        ims.append({"g": torch.from_numpy(g).cuda(), "psf": h, "alpha": bench.stable_alpha(h),
                    "f_true": torch.from_numpy(f.astype(np.float32)).cuda(),
                    "x_out": torch.empty(sp["n1"], sp["n2"], device="cuda"), "g64": g,
                    "f64": f.astype(np.float32).astype(np.float64), "n": n, "small": small})
    B = ar.Batch(ims, iters=iters, precondition=True, tuning=0)
    B.run()
    tr, best, _ = B.results()
    order = sorted((j for j, im in enumerate(ims) if im["small"]), key=lambda j: ims[j]["n"])[:3]
    assert len(order) == 3
    for j in order:
        im = ims[j]
        xo, to, bo = O.restore(im["g64"].astype(np.float64), im["psf"], im["alpha"], 1.0, iters,
                               True, f_true=im["f64"])
        tol = tol_alpha(im["alpha"])
        assert rel(im["x_out"].cpu().numpy(), xo) <= tol, (j, im["alpha"])
        assert np.all(np.abs(tr[j] - to) <= tol * (1 + to)), j
    B.close()
