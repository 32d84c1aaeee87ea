"""FP64 oracle of the spectral correction of the symmetrized preconditioner
and of the small MLP that predicts it.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's optimal preconditioner (Theorem 4) replaces the PSF h by its
symmetrized part s (eq. simmetrizzata2d); with a = h - s the antisymmetric
part, the AR eigenvalue of frequency x is the symbol of s (eq.
funzione_generatrice), lambda_s(x) = s^(x).  Iterating with A' A (Section 4),
the quantity a preconditioner should invert per frequency is the response of
A' A there.  For large images its value at an AR grid point is the average of
|h^|^2 over the four sign flips of the frequency, and since the flip average
of a^ is zero,

    avg_flips |h^(+-x1, +-x2)|^2 = lambda_s(x)^2 + delta(x),
    delta(x1, x2) = (|a^(x1, x2)|^2 + |a^(-x1, x2)|^2) / 2,

where a^(w) = sum_s a_s exp(-i s.w).  delta >= 0 depends only on the
antisymmetric part, and vanishes for strongly symmetric PSFs.  The corrected
filter is d = 1/(lambda_s^2 + delta + alpha) (eq. TikFilter with the refined
eigenvalue).  The paper has no such correction: it is the learned form's
target, the per-frequency refinement of the symmetrized eigenvalues.

The learned form predicts delta on a G x G grid of [0, pi]^2 (G = 33) from the
antisymmetric part of a 15 x 15 PSF with a three-layer perceptron (ReLU,
width 256), trained by mean squared error with Adam; the image's AR grid
reads the prediction by bilinear interpolation.
"""

from __future__ import annotations

import numpy as np

from .ar_oracle import (ar_analysis, ar_blur, ar_grid, ar_reblur, ar_synthesis, eigenvalues,
                        psf_support, rre, symmetrize, symprec_setup)

CORR_GRID = 33                 # points per axis of the predicted table on [0, pi]
CORR_Q = 7                     # the model takes 15 x 15 PSFs
CORR_IN = (2 * CORR_Q + 1) ** 2
CORR_HIDDEN = 256
CORR_OUT = CORR_GRID * CORR_GRID
CORR_IN_SCALE = 16.0           # inputs are 16 (h - s): O(1) entries for typical PSFs


def antisymmetric_part(h: np.ndarray) -> np.ndarray:
    """``a = h - s`` with ``s`` the symmetrized PSF of eq. simmetrizzata2d."""
    h = np.asarray(h, dtype=np.float64)
    return h - symmetrize(h)


def spectral_energy(a: np.ndarray, x1: np.ndarray, x2: np.ndarray) -> np.ndarray:
    """``delta(x1, x2) = (|a^(x1, x2)|^2 + |a^(-x1, x2)|^2) / 2`` on the grid ``x1 x x2``,
    ``a^(w) = sum_s a_s exp(-i (s1 w1 + s2 w2))``, summed term by term."""
    a = np.asarray(a, dtype=np.float64)
    q1, q2 = psf_support(a)
    x1 = np.asarray(x1, dtype=np.float64)[:, None]
    x2 = np.asarray(x2, dtype=np.float64)[None, :]
    ap = np.zeros((x1.shape[0], x2.shape[1]), dtype=complex)
    am = np.zeros_like(ap)
    for s1 in range(-q1, q1 + 1):
        for s2 in range(-q2, q2 + 1):
            v = a[s1 + q1, s2 + q2]
            ap += v * np.exp(-1j * (s1 * x1 + s2 * x2))
            am += v * np.exp(-1j * (-s1 * x1 + s2 * x2))
    return 0.5 * (np.abs(ap) ** 2 + np.abs(am) ** 2)


def corr_grid() -> np.ndarray:
    """The model's frequency grid ``j pi / (G - 1)``, ``j = 0..G-1``."""
    return np.arange(CORR_GRID) * np.pi / (CORR_GRID - 1)


def corr_target(h: np.ndarray) -> np.ndarray:
    """Training target: ``delta`` of the PSF's antisymmetric part on the model grid."""
    g = corr_grid()
    return spectral_energy(antisymmetric_part(h), g, g)


def corr_input(h: np.ndarray) -> np.ndarray:
    """Model input: ``16 (h - s)`` of a 15 x 15 PSF, row-major, length 225."""
    h = np.asarray(h, dtype=np.float64)
    if h.shape != (2 * CORR_Q + 1, 2 * CORR_Q + 1):
        raise ValueError("the correction model takes 15 x 15 PSFs")
    return CORR_IN_SCALE * antisymmetric_part(h).reshape(-1)


def bilinear(table: np.ndarray, x1: np.ndarray, x2: np.ndarray) -> np.ndarray:
    """Bilinear interpolation of a ``G x G`` table on ``[0, pi]^2`` at ``x1 x x2``."""
    G = table.shape[0]

    def cell(x):
        u = np.asarray(x, dtype=np.float64) / np.pi * (G - 1)
        i = np.minimum(np.floor(u).astype(int), G - 2)
        return i, u - i

    i, t = cell(x1)
    j, w = cell(x2)
    out = np.zeros((len(i), len(j)))
    for r in range(len(i)):
        for c in range(len(j)):
            a, b = i[r], j[c]
            out[r, c] = ((1 - t[r]) * (1 - w[c]) * table[a, b] + (1 - t[r]) * w[c] * table[a, b + 1]
                         + t[r] * (1 - w[c]) * table[a + 1, b] + t[r] * w[c] * table[a + 1, b + 1])
    return out


# ------------------------------------------------------------------ model --

def mlp_init(rng: np.random.Generator) -> dict:
    """He-uniform weights (row-major ``in x out``) and zero biases."""
    def layer(i, o):
        lim = np.sqrt(6.0 / i)
        return rng.uniform(-lim, lim, size=(i, o)), np.zeros(o)

    W1, b1 = layer(CORR_IN, CORR_HIDDEN)
    W2, b2 = layer(CORR_HIDDEN, CORR_HIDDEN)
    W3, b3 = layer(CORR_HIDDEN, CORR_OUT)
    return {"W1": W1, "b1": b1, "W2": W2, "b2": b2, "W3": W3, "b3": b3}


PARAM_ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def mlp_forward(P: dict, X: np.ndarray):
    """``Y = relu(relu(X W1 + b1) W2 + b2) W3 + b3``; returns ``(Y, cache)``."""
    X = np.asarray(X, dtype=np.float64)
    Z1 = X @ P["W1"] + P["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ P["W2"] + P["b2"]
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ P["W3"] + P["b3"]
    return Y, (X, Z1, H1, Z2, H2)


def mse_loss(Y: np.ndarray, T: np.ndarray):
    """``L = mean (Y - T)^2`` over the batch and the outputs, and ``dL/dY``."""
    D = Y - T
    return float(np.mean(D * D)), 2.0 * D / D.size


def mlp_backward(P: dict, cache, dY: np.ndarray) -> dict:
    """Gradients of the loss with respect to every parameter (chain rule)."""
    X, Z1, H1, Z2, H2 = cache
    g = {"W3": H2.T @ dY, "b3": dY.sum(axis=0)}
    dH2 = dY @ P["W3"].T
    dZ2 = dH2 * (Z2 > 0)
    g["W2"] = H1.T @ dZ2
    g["b2"] = dZ2.sum(axis=0)
    dH1 = dZ2 @ P["W2"].T
    dZ1 = dH1 * (Z1 > 0)
    g["W1"] = X.T @ dZ1
    g["b1"] = dZ1.sum(axis=0)
    return g


def adam_step(P: dict, G: dict, state: dict, lr: float, beta1=0.9, beta2=0.999, eps=1e-8) -> None:
    """One Adam update (Kingma and Ba) of every parameter, in place.
    ``state`` holds ``t`` and the first / second moment estimates."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in PARAM_ORDER:
        m = state.setdefault("m_" + k, np.zeros_like(P[k]))
        v = state.setdefault("v_" + k, np.zeros_like(P[k]))
        m[:] = beta1 * m + (1 - beta1) * G[k]
        v[:] = beta2 * v + (1 - beta2) * G[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)


def mlp_predict_table(P: dict, h: np.ndarray) -> np.ndarray:
    """The model's ``delta`` table for one PSF (entries may be negative where the
    symmetrized eigenvalue overstates the response; the filter clamps)."""
    Y, _ = mlp_forward(P, corr_input(h)[None, :])
    return Y[0].reshape(CORR_GRID, CORR_GRID)


# ------------------------------------------------------ corrected filter --

def symprec_setup_corrected(h: np.ndarray, n1: int, n2: int, alpha: float,
                            table: np.ndarray | None = None) -> dict:
    """AR preconditioner with the refined eigenvalues:
    ``d = 1/(max(lambda_s^2 + delta, 0) + alpha)``.

    ``delta`` is the exact spectral energy of ``h - s`` on the AR grid when
    ``table`` is None, else the bilinear reading of a ``G x G`` table.  A
    refined eigenvalue of A'A is a response energy, never negative: a table
    entry below ``-lambda_s^2`` (a restoration-fitted departure, or a model's
    prediction of one) is clamped there."""
    s = symmetrize(h)
    lam = eigenvalues(s, n1, n2)
    x1, x2 = ar_grid(n1), ar_grid(n2)
    if table is None:
        delta = spectral_energy(antisymmetric_part(h), x1, x2)
    else:
        delta = bilinear(np.asarray(table, dtype=np.float64), x1, x2)
    return {"s": s, "lam": lam, "delta": delta,
            "d": 1.0 / (np.maximum(lam ** 2 + delta, 0.0) + alpha), "n1": n1, "n2": n2}


def restore_corrected(g, h, alpha, tau=1.0, iters=20, table=None, f_true=None):
    """D-Landweber (eq. DLandweberMeth) with the corrected filter."""
    g = np.asarray(g, dtype=np.float64)
    n1, n2 = g.shape
    prec = symprec_setup_corrected(h, n1, n2, alpha, table)
    x = np.zeros((n1, n2))
    trace = [] if f_true is not None else None
    for _ in range(iters):
        z = ar_synthesis(prec["d"] * ar_analysis(ar_reblur(g - ar_blur(x, h), h)))
        x = x + tau * z
        if trace is not None:
            trace.append(rre(x, f_true))
    best = int(np.argmin(trace)) + 1 if trace else None
    return x, (np.asarray(trace) if trace is not None else None), best


# ------------------------------------- targets from the method's restorations --
#
# The learned form's training targets come from restorations the plain method
# itself produces.  Section 4's iteration x_{k+1} = x_k + tau D z_k, with
# z_k = A'(g - A x_k), updates the reblurred residual as
#     z_{k+1} = z_k - tau A'A D z_k,
# so in the AR spectral basis of Theorem 1 (z^ = T~ z, D = T diag(d) T~)
#     z^_{k+1} = z^_k - tau (T~ A'A T) (d o z^_k).
# Were T~ A'A T diagonal with entries mu, every frequency would obey
# z^_{k+1} = (1 - tau mu d) z^_k.  The per-frequency mu the iterates of the
# symmetrized D-Landweber actually show is the least-squares fit over the pairs
# of consecutive iterates,
#     mu^ = sum_k w_k v_k / sum_k w_k^2,   w_k = tau d z^_k,   v_k = z^_k - z^_{k+1},
# and the target is its departure from the symmetrized eigenvalue,
#     delta^ = mu^ - lambda_s^2,
# pooled onto the model's G x G grid: each interior AR frequency adds its
# delta^ with weight (bilinear weight of the node) x (sum_k w_k^2 / tau^2) to the
# four nodes around it, and a node takes the weighted mean.  Where the image
# has almost no content the fit divides two differences of tiny spectral values
# and is set by rounding, so each frequency's departure is shrunk towards 0 by
# a prior weight rho = theta x (the mean weight of the interior frequencies),
# theta = CORR_FIT_PRIOR: delta^ = (mu^ - lambda_s^2) w / (w + rho) (a Tikhonov
# fit of mu towards lambda_s^2).  A perturbation e of the spectral values then
# moves delta^ by at most about e sqrt(K) / (tau d sqrt(rho)): frequencies with
# real weight keep their fit, the others stay near 0.  (The mean, not the
# largest weight, keeps the rule independent of the image size: a natural
# scene's largest weight grows faster with the size than its typical one.)
# Frequencies on the
# boundary lines of the AR basis (index 0 or m - 1 on either axis, the unit
# columns of T_m) are left out.  For a strongly symmetric PSF T~ A'A T =
# diag(lambda^2) (Theorem 2, and A' = A), so mu^ = lambda^2 and the target is
# zero.

CORR_FIT_PRIOR = 5.0

def fit_spectral_response(zhat, d: np.ndarray, tau: float):
    """``(mu^, weight)`` per frequency from the spectra ``z^_0 .. z^_K`` of the
    reblurred residuals: ``mu^ = sum_k w_k v_k / sum_k w_k^2`` over k = 0..K-1,
    ``w_k = tau d z^_k``, ``v_k = z^_k - z^_{k+1}``; weight ``sum_k (d z^_k)^2``
    (mu^ = 0 where the weight is 0)."""
    num = np.zeros_like(d)
    den = np.zeros_like(d)
    for k in range(len(zhat) - 1):
        w = tau * d * zhat[k]
        v = zhat[k] - zhat[k + 1]
        num += w * v
        den += w * w
    mu = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
    return mu, den / (tau * tau)


def pool_to_grid(field: np.ndarray, weight: np.ndarray, x1: np.ndarray, x2: np.ndarray,
                 G: int = CORR_GRID, prior: float = 0.0) -> np.ndarray:
    """Weighted bilinear pooling of a field sampled at ``x1 x x2`` onto the ``G x G``
    grid ``j pi / (G - 1)``: node value = sum(b w f) / (sum(b w) + prior) over the
    samples of its four cells, b the bilinear weight of the node at the sample
    (0 where no weight falls)."""
    num = np.zeros((G, G))
    wsum = np.zeros((G, G))
    u1 = np.asarray(x1, dtype=np.float64) / np.pi * (G - 1)
    u2 = np.asarray(x2, dtype=np.float64) / np.pi * (G - 1)
    for r in range(len(u1)):
        i = min(int(np.floor(u1[r])), G - 2)
        t = u1[r] - i
        for c in range(len(u2)):
            if weight[r, c] <= 0:
                continue
            j = min(int(np.floor(u2[c])), G - 2)
            w = u2[c] - j
            for (a, b, bw) in ((i, j, (1 - t) * (1 - w)), (i, j + 1, (1 - t) * w),
                               (i + 1, j, t * (1 - w)), (i + 1, j + 1, t * w)):
                num[a, b] += bw * weight[r, c] * field[r, c]
                wsum[a, b] += bw * weight[r, c]
    return np.where(wsum > 0, num / np.where(wsum > 0, wsum + prior, 1.0), 0.0)


def restoration_target(h: np.ndarray, f: np.ndarray, e: np.ndarray, nu: float, alpha: float,
                       tau: float = 1.0, iters: int = 8) -> np.ndarray:
    """The learned form's training target for PSF ``h`` from a restoration of the
    scene ``f`` by the symmetrized D-Landweber (eq. DLandweberMeth, x_0 = 0):
    g = A f + nu ||A f|| e / ||e||, ``iters`` iterations, the spectra
    ``z^_k = T~ z_k`` (k = 0 .. iters - 1) fitted per frequency as above,
    ``delta^ = mu^ - lambda_s^2`` on the interior AR frequencies pooled onto the
    model grid, each shrunk by the prior weight CORR_FIT_PRIOR x the mean weight."""
    f = np.asarray(f, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    n1, n2 = f.shape
    gc = ar_blur(f, h)
    g = gc + nu * np.linalg.norm(gc) / np.linalg.norm(e) * e
    prec = symprec_setup(h, n1, n2, alpha)
    d = prec["d"]
    x = np.zeros((n1, n2))
    zhat = []
    for _ in range(iters):
        z = ar_reblur(g - ar_blur(x, h), h)
        zh = ar_analysis(z)
        zhat.append(zh)
        x = x + tau * ar_synthesis(d * zh)
    mu, wgt = fit_spectral_response(zhat, d, tau)
    inner = (slice(1, n1 - 1), slice(1, n2 - 1))
    x1, x2 = ar_grid(n1)[1:n1 - 1], ar_grid(n2)[1:n2 - 1]
    w = wgt[inner]
    rho = CORR_FIT_PRIOR * float(np.mean(w))
    delta = (mu[inner] - prec["lam"][inner] ** 2) * w / (w + rho)
    return pool_to_grid(delta, w, x1, x2)
