"""Pins of the spectral-correction oracle (the learned form's target, model
and corrected filter) against things other than itself: numpy's FFT, a dense
assembly of A' A in the AR basis, finite differences, Adam's closed-form
first step, exact interpolation identities and dense brute force."""

import numpy as np
import pytest

import oracle as O
from paper_1211_0393_gb300 import workloads as W


def rand_psf(rng, q1, q2):
    h = rng.random((2 * q1 + 1, 2 * q2 + 1))
    return h / h.sum()


@pytest.mark.parametrize("q1,q2", [(2, 2), (3, 1), (7, 7)])
def test_lambda2_plus_delta_is_flip_averaged_fft_energy(q1, q2):
    """lambda_s^2 + delta = (|h^(w1, w2)|^2 + |h^(-w1, w2)|^2) / 2 with h^ from numpy's FFT."""
    rng = np.random.default_rng(q1 * 10 + q2)
    h = rand_psf(rng, q1, q2)
    N = 64
    F = np.fft.fft2(h, s=(N, N))          # |F[k]| = |h^(2 pi k / N)| (the offset is a phase)
    k = np.arange(N // 2 + 1)
    x = 2 * np.pi * k / N
    E = np.abs(F) ** 2
    want = 0.5 * (E[np.ix_(k, k)] + E[np.ix_((-k) % N, k)])
    lam = O.symbol(O.symmetrize(h), x, x)
    got = lam ** 2 + O.spectral_energy(O.antisymmetric_part(h), x, x)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def test_delta_vanishes_exactly_for_strongly_symmetric_psfs_only():
    rng = np.random.default_rng(3)
    h = rand_psf(rng, 3, 2)
    s = O.symmetrize(h)
    x = O.corr_grid()
    assert np.max(np.abs(O.antisymmetric_part(s))) < 1e-17
    assert np.max(O.spectral_energy(O.antisymmetric_part(s), x, x)) < 1e-30
    d = O.spectral_energy(O.antisymmetric_part(h), x, x)
    assert d.min() >= 0 and d.max() > 1e-4


def test_corrected_eigenvalue_tracks_the_diagonal_of_AtA_in_the_AR_basis():
    """diag(T~ A'A T) at interior frequencies is matched by lambda_s^2 + delta far
    better than by lambda_s^2 alone (boundary terms are O(q/n))."""
    rng = np.random.default_rng(1)
    n = 40
    h = rand_psf(rng, 2, 2)
    A = O.ar_matrix_dense(h, n, n)
    Ap = O.ar_matrix_dense(h[::-1, ::-1], n, n)
    T = np.kron(O.ar_T(n), O.ar_T(n))
    Tt = np.kron(O.ar_Ttilde(n), O.ar_Ttilde(n))
    diag = np.diag(Tt @ Ap @ A @ T).reshape(n, n)[1:-1, 1:-1]
    lam = O.eigenvalues(O.symmetrize(h), n, n)[1:-1, 1:-1]
    x = O.ar_grid(n)[1:-1]
    corr = lam ** 2 + O.spectral_energy(O.antisymmetric_part(h), x, x)
    err_corr = np.max(np.abs(diag - corr))
    err_sym = np.max(np.abs(diag - lam ** 2))
    assert err_corr < 1e-2
    assert err_corr < 0.25 * err_sym


def test_bilinear_is_exact_on_nodes_and_for_bilinear_functions():
    G = O.CORR_GRID
    x = O.corr_grid()
    rng = np.random.default_rng(0)
    T = rng.random((G, G))
    np.testing.assert_allclose(O.bilinear(T, x, x), T, rtol=0, atol=1e-12)
    f = lambda u, v: 0.3 + 1.7 * u - 0.4 * v + 0.25 * u * v  # noqa: E731
    tab = f(x[:, None], x[None, :])
    y = rng.uniform(0, np.pi, 17)
    np.testing.assert_allclose(O.bilinear(tab, y, y[::-1]), f(y[:, None], y[::-1][None, :]),
                               atol=1e-12)


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(5)
    P = O.mlp_init(rng)
    for k in O.PARAM_ORDER:
        if k.startswith("b"):
            P[k] = rng.normal(0, 0.1, P[k].shape)
    X = rng.normal(0, 1, (4, O.CORR_IN))
    T = rng.normal(0, 1, (4, O.CORR_OUT))
    Y, cache = O.mlp_forward(P, X)
    _, dY = O.mse_loss(Y, T)
    G = O.mlp_backward(P, cache, dY)
    eps = 1e-6
    for k in O.PARAM_ORDER:
        flat = P[k].reshape(-1)
        for idx in rng.choice(flat.size, 4, replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _ = O.mse_loss(O.mlp_forward(P, X)[0], T)
            flat[idx] = old - eps
            lm, _ = O.mse_loss(O.mlp_forward(P, X)[0], T)
            flat[idx] = old
            num = (lp - lm) / (2 * eps)
            assert abs(G[k].reshape(-1)[idx] - num) <= 1e-6 * max(1.0, abs(num)), (k, idx)


def test_adam_first_step_closed_form():
    """After one step m^ = g and v^ = g^2, so the update is -lr g / (|g| + eps)."""
    rng = np.random.default_rng(2)
    P = O.mlp_init(rng)
    G = {k: rng.normal(0, 1e-3, P[k].shape) for k in O.PARAM_ORDER}
    before = {k: P[k].copy() for k in O.PARAM_ORDER}
    st = {}
    O.adam_step(P, G, st, lr=1e-3)
    for k in O.PARAM_ORDER:
        want = before[k] - 1e-3 * G[k] / (np.abs(G[k]) + 1e-8)
        np.testing.assert_allclose(P[k], want, rtol=1e-12, atol=1e-15)


def test_corrected_setup_reads_exact_delta_on_grid_nodes():
    """For n = 33 every AR grid point is a table node, so the table reading is exact."""
    rng = np.random.default_rng(9)
    h = rand_psf(rng, 7, 7)
    exact = O.symprec_setup_corrected(h, 33, 33, 0.1)
    tab = O.symprec_setup_corrected(h, 33, 33, 0.1, table=O.corr_target(h))
    np.testing.assert_allclose(tab["d"], exact["d"], rtol=1e-11)
    assert np.all(exact["d"] <= 1.0 / (exact["lam"] ** 2 + 0.1) + 1e-15)


def test_restore_corrected_reduces_to_restore_for_symmetric_psf_and_matches_dense():
    rng = np.random.default_rng(4)
    n = 12
    hs = O.symmetrize(rand_psf(rng, 2, 2))
    g = rng.random((n, n))
    x1, _, _ = O.restore(g, hs, 0.05, 1.0, 5, True)
    x2, _, _ = O.restore_corrected(g, hs, 0.05, 1.0, 5)
    np.testing.assert_allclose(x2, x1, rtol=0, atol=1e-14)
    # asymmetric PSF against a dense iteration with D = T diag(d) inv(T)
    h = rand_psf(rng, 2, 1)
    prec = O.symprec_setup_corrected(h, n, n, 0.05)
    A = O.ar_matrix_dense(h, n, n)
    Ap = O.ar_matrix_dense(h[::-1, ::-1], n, n)
    T = np.kron(O.ar_T(n), O.ar_T(n))
    D = T @ np.diag(prec["d"].reshape(-1)) @ np.linalg.inv(T)
    x = np.zeros(n * n)
    for _ in range(5):
        x = x + D @ (Ap @ (g.reshape(-1) - A @ x))
    x3, _, _ = O.restore_corrected(g, h, 0.05, 1.0, 5)
    np.testing.assert_allclose(x3.reshape(-1), x, rtol=0, atol=1e-11)


# ---------------------------------------- targets from the method's restorations

def test_fit_recovers_a_known_spectral_response():
    """A sequence that obeys z^_{k+1} = (1 - tau mu d) z^_k exactly at every
    frequency: the least-squares fit returns mu, and the weight sum_k (d z^_k)^2."""
    rng = np.random.default_rng(3)
    shape = (9, 7)
    mu = rng.uniform(0.0, 1.5, shape)
    d = rng.uniform(0.5, 3.0, shape)
    z = [rng.standard_normal(shape)]
    tau = 0.7
    for _ in range(5):
        z.append((1.0 - tau * mu * d) * z[-1])
    got, wgt = O.fit_spectral_response(z, d, tau)
    np.testing.assert_allclose(got, mu, rtol=1e-12, atol=1e-12)
    want_w = sum((d * zk) ** 2 for zk in z[:-1])
    np.testing.assert_allclose(wgt, want_w, rtol=1e-13)


def test_pool_of_a_constant_field_is_that_constant():
    rng = np.random.default_rng(4)
    x1 = np.sort(rng.uniform(0, np.pi, 40))
    x2 = np.sort(rng.uniform(0, np.pi, 50))
    w = rng.uniform(0.1, 2.0, (40, 50))
    T = O.pool_to_grid(np.full((40, 50), -0.375), w, x1, x2)
    covered = np.zeros_like(T, dtype=bool)
    G = T.shape[0]
    for a in x1:
        for b in x2:
            i = min(int(a / np.pi * (G - 1)), G - 2)
            j = min(int(b / np.pi * (G - 1)), G - 2)
            covered[i:i + 2, j:j + 2] = True
    np.testing.assert_allclose(T[covered], -0.375, rtol=1e-13)
    assert np.all(T[~covered] == 0.0)


def test_pool_is_a_weighted_mean_of_the_samples_around_a_node():
    """One sample per cell at known places: every node equals the bilinear-and-weight
    weighted mean of the field values of the samples in its (up to) four cells."""
    G = 5
    x = (np.arange(G - 1) + 0.3) * np.pi / (G - 1)       # one sample per cell, t = 0.3
    f = np.arange(16.0).reshape(4, 4)
    w = np.ones((4, 4))
    T = O.pool_to_grid(f, w, x, x, G)
    # node (1, 1): samples (0,0) b = .3*.3, (0,1) b = .3*.7, (1,0) .7*.3, (1,1) .7*.7
    b = np.array([[0.09, 0.21], [0.21, 0.49]])
    assert T[1, 1] == pytest.approx(np.sum(b * f[0:2, 0:2]) / np.sum(b), rel=1e-13)
    assert T[0, 0] == pytest.approx(f[0, 0], rel=1e-13)


def test_restoration_target_vanishes_for_a_strongly_symmetric_psf():
    """For h = s, T~ A'A T = diag(lambda^2) (Theorem 2 with A' = A), so the
    iterates decay frequency by frequency exactly and the fitted response equals
    lambda^2: the target is zero up to rounding."""
    rng = np.random.default_rng(5)
    n = 24
    a = np.arange(-3, 4)
    h = np.exp(-0.5 * (a[:, None] ** 2 / 1.3 + a[None, :] ** 2 / 2.1))
    h /= h.sum()
    f = rng.uniform(0, 1, (n, n))
    e = rng.standard_normal((n, n))
    T = O.restoration_target(h, f, e, 0.01, 0.1, 1.0, 6)
    assert np.max(np.abs(T)) <= 1e-9


def test_restoration_target_is_not_zero_and_positive_where_the_image_has_content():
    """For the bench's strongly non-symmetric PSF the fitted departure is clearly
    nonzero, and at the low frequencies (where a natural-like scene carries its
    energy) it is positive, as the closed-form flip-averaged energy of h - s."""
    h = W.psf_config2()
    ext, f, e = W.make_inputs(128, 128, h, "ellipses", 5)
    T = O.restoration_target(h, f, e, 0.005, 0.3, 1.0, 8)
    c = O.corr_target(h)
    assert np.max(np.abs(T)) > 0.05
    low = (slice(1, 6), slice(1, 6))
    assert np.all(T[low] > 0)
    assert np.corrcoef(T[low].ravel(), c[low].ravel())[0, 1] > 0.5
