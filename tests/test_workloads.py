"""Seeded input generators: determinism, PSF normalisation, the noise-level rule."""

import numpy as np
import pytest

from paper_1211_0393_gb300 import workloads as W


def test_noise_level_is_exact():
    rng = np.random.default_rng(1)
    gc = rng.uniform(0, 1, (40, 33))
    e = W.noise_field(40, 33, rng)
    for nu in (0.01, 0.005, 0.001):
        g = W.add_noise(gc, e, nu)
        assert np.linalg.norm(g - gc) / np.linalg.norm(gc) == pytest.approx(nu, rel=1e-12)


@pytest.mark.parametrize("fn,shape", [(W.psf_config1, (9, 9)), (W.psf_config2, (15, 15)),
                                      (W.psf_config4, (21, 21))])
def test_named_psfs_are_normalized_nonnegative_odd(fn, shape):
    h = fn()
    assert h.shape == shape
    assert h.min() >= 0
    assert h.sum() == pytest.approx(1.0, abs=1e-14)


def _asym(h):
    s = (h + h[::-1, :] + h[:, ::-1] + h[::-1, ::-1]) / 4
    return np.linalg.norm(h - s) / np.linalg.norm(h)


def test_config_psf_asymmetry_ordering():
    # config 1 is "slightly" and config 2 "highly" non-symmetric
    assert 0.05 < _asym(W.psf_config1()) < _asym(W.psf_config2())
    assert _asym(W.psf_config2()) > 0.5


def test_motion_psf_is_centrally_symmetric_segment():
    h = W.psf_motion(7, 7, 11.0, 30.0)
    np.testing.assert_allclose(h, h[::-1, ::-1], atol=1e-12)
    # points up-right: more mass at (row<0, col>0) than at (row<0, col<0)
    assert h[:7, 8:].sum() > 10 * h[:7, :7].sum()


def test_generators_are_deterministic_and_in_range():
    h = W.psf_config1()
    a = W.make_inputs(64, 64, h, "blocks", 0)
    b = W.make_inputs(64, 64, h, "blocks", 0)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    ext, f, e = a
    assert ext.shape == (72, 72) and f.shape == (64, 64) and e.shape == (64, 64)
    assert f.min() >= 0 and f.max() <= 1
    ext2, f2, _ = W.make_inputs(96, 80, W.psf_config2(), "ellipses", 1)
    assert ext2.shape == (110, 94) and 0 <= f2.min() and f2.max() <= 1
    np.testing.assert_array_equal(W.crop(ext2, 7, 7), f2)


def test_random_psf_mixture():
    rng = np.random.default_rng(3)
    for _ in range(10):
        q = int(rng.integers(2, 16))
        h = W.psf_random(q, q, rng)
        assert h.shape == (2 * q + 1, 2 * q + 1)
        assert h.min() >= 0 and h.sum() == pytest.approx(1.0, abs=1e-13)
