"""Seeded synthetic workloads: scenes, PSFs and noise.

This module holds no arithmetic of the restoration method (no boundary
condition, no blur, no transform, no iteration).  It only draws inputs, so
that the FP64 oracle and the CUDA library can be fed identical data:

* a scene larger than the field of view by ``q`` pixels on every side (the
  data model of eq. modello_discreto_sistema blurs a scene wider than the FOV;
  the caller blurs it and crops the centre),
* a PSF mask of odd sides, non-negative, summing to one (eq.
  coefficienti_psf),
* a standard normal noise field and the rule that scales it to a relative
  level ``nu`` (the paper adds "about 0.1%" white Gaussian noise; the level is
  read as ``||eta||_F = nu ||g_clean||_F``).

Recipes (see the workload table of the design notes):

* ``scene_blocks``: piecewise-constant rectangles and disks on a smooth linear
  gradient, clipped to [0, 1] (stands in for the paper's Cameraman image).
* ``scene_ellipses``: 8-16 random ellipses plus a smooth multi-octave texture
  (sum of four bilinearly interpolated random lattices), in [0, 1] (stands in
  for the Bridge image).
* ``psf_gaussian``: sampled anisotropic, rotated, off-centre Gaussian.
* ``psf_motion``: a bilinearly rasterised line segment.
* ``psf_config2``: motion length 11 at 30 degrees plus a 0.2-weight Gaussian
  offset by (2, -1) px, 15x15 (highly non-symmetric).
"""

from __future__ import annotations

import numpy as np

SEED_BASE = 12110393


def rng_for(config_idx: int, salt: int = 0) -> np.random.Generator:
    """Generator seeded with ``SEED_BASE + config_idx`` (plus an optional salt)."""
    return np.random.default_rng(SEED_BASE + config_idx + 1000 * salt)


# --------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------

def scene_blocks(m1: int, m2: int, rng: np.random.Generator) -> np.ndarray:
    """Rectangles and disks on a linear gradient, clipped to [0, 1]."""
    i1 = np.arange(m1)[:, None] / max(m1 - 1, 1)
    i2 = np.arange(m2)[None, :] / max(m2 - 1, 1)
    a, b = rng.uniform(-0.3, 0.3, size=2)
    img = 0.35 + a * i1 + b * i2
    img = np.broadcast_to(img, (m1, m2)).copy()
    for _ in range(int(rng.integers(4, 9))):
        r0, r1 = sorted(rng.uniform(0, 1, size=2))
        c0, c1 = sorted(rng.uniform(0, 1, size=2))
        mask = (i1 >= r0) & (i1 <= r1) & (i2 >= c0) & (i2 <= c1)
        img[np.broadcast_to(mask, img.shape)] = rng.uniform(0, 1)
    for _ in range(int(rng.integers(3, 7))):
        cy, cx = rng.uniform(0, 1, size=2)
        rad = rng.uniform(0.05, 0.25)
        mask = (i1 - cy) ** 2 + (i2 - cx) ** 2 <= rad ** 2
        img[np.broadcast_to(mask, img.shape)] = rng.uniform(0, 1)
    return np.clip(img, 0.0, 1.0)


def _lattice_texture(m1: int, m2: int, cells: int, rng: np.random.Generator) -> np.ndarray:
    """One octave: a random ``(cells+1)^2`` lattice bilinearly interpolated to ``m1 x m2``."""
    lat = rng.uniform(-1.0, 1.0, size=(cells + 1, cells + 1))
    u = np.linspace(0.0, cells, m1)
    v = np.linspace(0.0, cells, m2)
    iu = np.minimum(u.astype(int), cells - 1)
    iv = np.minimum(v.astype(int), cells - 1)
    fu = (u - iu)[:, None]
    fv = (v - iv)[None, :]
    l00 = lat[iu][:, iv]
    l10 = lat[iu + 1][:, iv]
    l01 = lat[iu][:, iv + 1]
    l11 = lat[iu + 1][:, iv + 1]
    return (1 - fu) * (1 - fv) * l00 + fu * (1 - fv) * l10 + (1 - fu) * fv * l01 + fu * fv * l11


def scene_ellipses(m1: int, m2: int, rng: np.random.Generator) -> np.ndarray:
    """8-16 random ellipses plus a four-octave smooth texture, rescaled into [0, 1]."""
    tex = np.zeros((m1, m2))
    for octave in range(4):
        tex += 0.5 ** octave * _lattice_texture(m1, m2, 4 * 2 ** octave, rng)
    img = 0.5 + 0.25 * tex / 1.875
    y = np.arange(m1)[:, None] / max(m1 - 1, 1)
    x = np.arange(m2)[None, :] / max(m2 - 1, 1)
    for _ in range(int(rng.integers(8, 17))):
        cy, cx = rng.uniform(0.05, 0.95, size=2)
        ry, rx = rng.uniform(0.03, 0.25, size=2)
        th = rng.uniform(0, np.pi)
        c, s = np.cos(th), np.sin(th)
        dy, dx = y - cy, x - cx
        u = (c * dx + s * dy) / rx
        v = (-s * dx + c * dy) / ry
        mask = u * u + v * v <= 1.0
        img = np.where(mask, 0.6 * rng.uniform(0, 1) + 0.4 * img, img)
    return np.clip(img, 0.0, 1.0)


# --------------------------------------------------------------------------
# PSFs
# --------------------------------------------------------------------------

def normalize(h: np.ndarray) -> np.ndarray:
    """Scale a non-negative mask to unit sum (eq. coefficienti_psf)."""
    h = np.asarray(h, dtype=np.float64)
    return h / h.sum()


def psf_gaussian(q1: int, q2: int, sigma1: float, sigma2: float | None = None,
                 theta_deg: float = 0.0, mu1: float = 0.0, mu2: float = 0.0) -> np.ndarray:
    """Sampled Gaussian on offsets ``-q..q`` with axis sigmas, rotation and mean offset."""
    sigma2 = sigma1 if sigma2 is None else sigma2
    t = np.deg2rad(theta_deg)
    a1 = np.arange(-q1, q1 + 1)[:, None] - mu1
    a2 = np.arange(-q2, q2 + 1)[None, :] - mu2
    u = np.cos(t) * a1 + np.sin(t) * a2
    v = -np.sin(t) * a1 + np.cos(t) * a2
    return normalize(np.exp(-0.5 * ((u / sigma1) ** 2 + (v / sigma2) ** 2)))


def psf_motion(q1: int, q2: int, length: float, angle_deg: float,
               samples: int = 400) -> np.ndarray:
    """A centred line segment of the given length and angle, rasterised with bilinear weights.

    ``angle`` is measured from the column axis towards decreasing row index
    (image convention: 30 degrees points up and to the right).
    """
    h = np.zeros((2 * q1 + 1, 2 * q2 + 1))
    t = np.deg2rad(angle_deg)
    for k in range(samples):
        r = (k + 0.5) / samples - 0.5
        p1 = -r * length * np.sin(t)     # row offset
        p2 = r * length * np.cos(t)      # column offset
        f1, f2 = np.floor(p1), np.floor(p2)
        w1, w2 = p1 - f1, p2 - f2
        for d1, c1 in ((0, 1 - w1), (1, w1)):
            for d2, c2 in ((0, 1 - w2), (1, w2)):
                a, b = int(f1) + d1 + q1, int(f2) + d2 + q2
                if 0 <= a <= 2 * q1 and 0 <= b <= 2 * q2:
                    h[a, b] += c1 * c2
    return normalize(h)


def psf_config1() -> np.ndarray:
    """9x9 Gaussian, sigma 1.5, centre shifted by (+0.5, +0.5) px (slightly non-symmetric)."""
    return psf_gaussian(4, 4, 1.5, 1.5, 0.0, 0.5, 0.5)


def psf_config2() -> np.ndarray:
    """15x15: motion length 11 at 30 degrees plus 0.2 x Gaussian(sigma 1.5) at (2, -1) px."""
    m = psf_motion(7, 7, 11.0, 30.0)
    g = psf_gaussian(7, 7, 1.5, 1.5, 0.0, 2.0, -1.0)
    return normalize(0.8 * m + 0.2 * g)


def psf_config4() -> np.ndarray:
    """21x21 asymmetric Gaussian, sigmas 2.0 / 3.5, rotated 40 degrees, mean offset 1 px."""
    return psf_gaussian(10, 10, 2.0, 3.5, 40.0, 1.0 / np.sqrt(2), 1.0 / np.sqrt(2))


def psf_random(q1: int, q2: int, rng: np.random.Generator) -> np.ndarray:
    """A random mixture (Gaussian / motion / asymmetric Gaussian) of the given support."""
    kind = int(rng.integers(0, 3))
    qm = min(q1, q2)
    s_hi = max(0.61, 0.5 + qm / 2)       # the bounds only bite for q = 0
    a_hi = max(0.61, 0.4 + qm / 2)
    if kind == 0:
        return psf_gaussian(q1, q2, rng.uniform(0.6, s_hi), None, 0.0,
                            rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5))
    if kind == 1:
        m = psf_motion(q1, q2, rng.uniform(1.5, max(1.51, 2 * qm)), rng.uniform(0, 180))
        g = psf_gaussian(q1, q2, 1.0, None, 0.0, 0.0, 0.0)
        return normalize(0.85 * m + 0.15 * g)
    return psf_gaussian(q1, q2, rng.uniform(0.6, a_hi), rng.uniform(0.6, a_hi),
                        rng.uniform(0, 180), rng.uniform(-1, 1), rng.uniform(-1, 1))


# --------------------------------------------------------------------------
# noise
# --------------------------------------------------------------------------

def noise_field(n1: int, n2: int, rng: np.random.Generator) -> np.ndarray:
    """Standard normal ``e`` of shape ``n1 x n2``."""
    return rng.standard_normal((n1, n2))


def add_noise(g_clean: np.ndarray, e: np.ndarray, nu: float) -> np.ndarray:
    """``g = g_clean + eta``, ``eta = nu ||g_clean||_F e / ||e||_F`` (noise level ``nu``)."""
    return g_clean + nu * np.linalg.norm(g_clean) / np.linalg.norm(e) * e


def crop(scene: np.ndarray, q1: int, q2: int) -> np.ndarray:
    """The field of view: drop ``q1`` rows and ``q2`` columns on every side."""
    m1, m2 = scene.shape
    return scene[q1:m1 - q1, q2:m2 - q2]


# --------------------------------------------------------------------------
# the named workloads
# --------------------------------------------------------------------------

WORKLOADS = {
    "blocks64_gauss9": dict(config_idx=0, n=(64, 64), scene="blocks", psf="config1",
                            nu=0.01, iters=20, alpha=None),
    "ellipses1024_motion15": dict(config_idx=1, n=(1024, 1024), scene="ellipses", psf="config2",
                                  nu=0.005, iters=50, alpha=None),
    "ellipses2048_gauss21": dict(config_idx=3, n=(2048, 2048), scene="ellipses", psf="config4",
                                 nu=0.01, iters=50, alpha=None),
}


def make_inputs(n1: int, n2: int, h: np.ndarray, scene: str, config_idx: int):
    """Extended scene, its FOV crop ``f`` and a noise field, all seeded.

    Returns ``(scene_ext, f, e)`` with ``scene_ext`` of shape
    ``(n1 + 2 q1) x (n2 + 2 q2)``; ``f = crop(scene_ext)``.
    """
    q1, q2 = (h.shape[0] - 1) // 2, (h.shape[1] - 1) // 2
    rng = rng_for(config_idx)
    gen = scene_blocks if scene == "blocks" else scene_ellipses
    ext = gen(n1 + 2 * q1, n2 + 2 * q2, rng)
    e = noise_field(n1, n2, rng)
    return ext, crop(ext, q1, q2), e


BATCH_SIDES = (128, 192, 256, 384, 512, 768, 1024)


def batch_specs(count: int = 96, config_idx: int = 2, sides=BATCH_SIDES, qmin: int = 2,
                qmax: int = 15):
    """Uneven batch: per image, sides drawn independently from ``sides`` and an
    own random PSF (Gaussian / motion / asymmetric Gaussian) of odd size
    5x5..31x31.  Returns a list of dicts with n1, n2, psf and a per-image seed."""
    rng = rng_for(config_idx)
    out = []
    for j in range(count):
        n1, n2 = int(rng.choice(sides)), int(rng.choice(sides))
        q = int(rng.integers(qmin, qmax + 1))
        out.append({"n1": n1, "n2": n2, "psf": psf_random(q, q, rng), "seed": int(rng.integers(1 << 30))})
    return out


def batch_inputs(spec: dict):
    """Extended scene, FOV crop and noise field of one batch image (seeded)."""
    h = spec["psf"]
    q1, q2 = (h.shape[0] - 1) // 2, (h.shape[1] - 1) // 2
    rng = np.random.default_rng(spec["seed"])
    ext = scene_ellipses(spec["n1"] + 2 * q1, spec["n2"] + 2 * q2, rng)
    e = noise_field(spec["n1"], spec["n2"], rng)
    return ext, crop(ext, q1, q2), e


def psf_named(name: str) -> np.ndarray:
    return {"config1": psf_config1, "config2": psf_config2, "config4": psf_config4}[name]()


# --------------------------------------------------------------------------
# the spectral-correction model: seeded PSF sets and initial parameters
# --------------------------------------------------------------------------

CORR_SHAPES = ((225, 256), (256,), (256, 256), (256,), (256, 1089), (1089,))


def corr_psfs(count: int, salt: int, config_idx: int = 4) -> np.ndarray:
    """``count`` random 15 x 15 PSFs (Gaussian / motion / asymmetric-Gaussian mixtures)."""
    rng = rng_for(config_idx, salt)
    return np.stack([psf_random(7, 7, rng) for _ in range(count)])


def corr_init_params(seed: int) -> np.ndarray:
    """Initial parameters W1 b1 W2 b2 W3 b3 (float32, flattened): He-uniform
    weights (row-major in x out), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for shape in CORR_SHAPES:
        if len(shape) == 2:
            lim = np.sqrt(6.0 / shape[0])
            parts.append(rng.uniform(-lim, lim, size=shape).reshape(-1))
        else:
            parts.append(np.zeros(shape))
    return np.concatenate(parts).astype(np.float32)
