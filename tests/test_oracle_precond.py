"""Pins of the symmetrized preconditioner and the (D-)Landweber iteration.

* Theorem 4 (eq. simmetrizzata2d-bis): least squares over all strongly
  symmetric PSFs of ||A(h) - P(s)||_F returns the symmetrized PSF,
* closed forms: one preconditioned step with alpha -> 0 and a strongly
  symmetric PSF is A^{-1} g; the iteration's fixed point solves A'A x = A'g,
* brute force: the dense N x N iteration with D = T diag(d) inv(T), the
  eigenvalues taken from the diagonal of inv(T) A(s) T, equals the oracle.
"""

import numpy as np
import pytest

import oracle as O


def rand_psf(rng, q1, q2):
    h = rng.uniform(0.0, 1.0, size=(2 * q1 + 1, 2 * q2 + 1))
    return h / h.sum()


def sharp_psf(rng, q1, q2, centre=0.6):
    """Non-symmetric PSF with a heavy centre: well conditioned, for closed-form checks."""
    h = rand_psf(rng, q1, q2) * (1 - centre)
    h[q1, q2] += centre
    return h


@pytest.mark.parametrize("n1,n2,q1,q2", [(7, 8, 1, 2), (9, 9, 2, 2), (8, 11, 3, 1)])
def test_theorem4_symmetrized_psf_is_the_frobenius_optimum(n1, n2, q1, q2):
    rng = np.random.default_rng(n1 + n2 + q1 + q2)
    h = rand_psf(rng, q1, q2)
    A = O.ar_matrix_dense(h, n1, n2)
    cols, keys = [], []
    for a in range(q1 + 1):
        for b in range(q2 + 1):
            e = np.zeros_like(h)
            for sa in {a, -a}:
                for sb in {b, -b}:
                    e[q1 + sa, q2 + sb] = 1.0
            cols.append(O.ar_matrix_dense(e, n1, n2).ravel())
            keys.append((a, b))
    coef, *_ = np.linalg.lstsq(np.stack(cols, axis=1), A.ravel(), rcond=None)
    s = O.symmetrize(h)
    for (a, b), c in zip(keys, coef):
        assert c == pytest.approx(s[q1 + a, q2 + b], abs=1e-13)
    # symmetrization: idempotent, sum preserving, strongly symmetric
    np.testing.assert_allclose(O.symmetrize(s), s, atol=0)
    assert s.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(s, s[::-1, :], atol=0)
    np.testing.assert_allclose(s, s[:, ::-1], atol=0)


def test_one_step_with_vanishing_alpha_inverts_a_strongly_symmetric_blur():
    rng = np.random.default_rng(21)
    n1, n2 = 10, 9
    s = O.symmetrize(sharp_psf(rng, 2, 3))
    f = rng.uniform(0, 1, (n1, n2))
    g = O.ar_blur(f, s)
    x1, _, _ = O.restore(g, s, alpha=1e-13, tau=1.0, iters=1, precondition=True)
    want = np.linalg.solve(O.ar_matrix_dense(s, n1, n2), g.ravel()).reshape(n1, n2)
    np.testing.assert_allclose(x1, want, atol=1e-9)
    np.testing.assert_allclose(x1, f, atol=1e-9)


def test_fixed_point_solves_the_reblurred_normal_equations():
    rng = np.random.default_rng(22)
    n1, n2 = 8, 9
    h = sharp_psf(rng, 2, 2, centre=0.7)
    g = rng.uniform(0, 1, (n1, n2))
    x, _, _ = O.restore(g, h, alpha=0.05, tau=1.0, iters=300, precondition=True)
    A = O.ar_matrix_dense(h, n1, n2)
    Ar = O.ar_matrix_dense(h[::-1, ::-1], n1, n2)
    want = np.linalg.solve(Ar @ A, Ar @ g.ravel()).reshape(n1, n2)
    np.testing.assert_allclose(x, want, atol=1e-10)


@pytest.mark.parametrize("precondition", [True, False])
def test_brute_force_dense_iteration(precondition):
    rng = np.random.default_rng(23)
    n1, n2, q1, q2 = 9, 8, 2, 3
    h = rand_psf(rng, q1, q2)
    f = rng.uniform(0, 1, (n1, n2))
    g = O.ar_blur(f, h) + 1e-3 * rng.standard_normal((n1, n2))
    alpha, tau, iters = 0.05, 1.0, 12
    A = O.ar_matrix_dense(h, n1, n2)
    Ar = O.ar_matrix_dense(h[::-1, ::-1], n1, n2)
    if precondition:
        T = np.kron(O.ar_T(n1), O.ar_T(n2))
        Tinv = np.linalg.inv(T)
        lam = np.diag(Tinv @ O.ar_matrix_dense(O.symmetrize(h), n1, n2) @ T)
        D = T @ np.diag(1.0 / (lam ** 2 + alpha)) @ Tinv
    else:
        D = np.eye(n1 * n2)
    x = np.zeros(n1 * n2)
    trace = []
    for _ in range(iters):
        x = x + tau * D @ Ar @ (g.ravel() - A @ x)
        trace.append(np.linalg.norm(x - f.ravel()) / np.linalg.norm(f))
    xo, to, best = O.restore(g, h, alpha, tau, iters, precondition, f_true=f)
    np.testing.assert_allclose(xo.ravel(), x, rtol=0, atol=1e-12 * np.abs(x).max())
    np.testing.assert_allclose(to, trace, rtol=1e-11)
    assert best == int(np.argmin(trace)) + 1


def test_restore_warm_start_continues_the_iteration():
    rng = np.random.default_rng(24)
    h = rand_psf(rng, 2, 2)
    g = rng.uniform(0, 1, (11, 12))
    x6, _, _ = O.restore(g, h, 0.02, 1.0, 6, True)
    x3, _, _ = O.restore(g, h, 0.02, 1.0, 3, True)
    x33, _, _ = O.restore(g, h, 0.02, 1.0, 3, True, x0=x3)
    np.testing.assert_allclose(x33, x6, atol=1e-13)


def test_solve_applies_D_and_its_inverse_is_A2_plus_alpha_for_symmetric_psf():
    """For strongly symmetric s: D^{-1} = A(s)^2 + alpha I (Theorems 1-2, eq. TikFilter)."""
    rng = np.random.default_rng(25)
    n1, n2 = 9, 10
    h = rand_psf(rng, 2, 3)
    s = O.symmetrize(h)
    prec = O.symprec_setup(h, n1, n2, 0.03)
    y = rng.standard_normal((n1, n2))
    z = O.symprec_solve(prec, y)
    As = O.ar_matrix_dense(s, n1, n2)
    back = (As @ As + 0.03 * np.eye(n1 * n2)) @ z.ravel()
    np.testing.assert_allclose(back, y.ravel(), atol=1e-11)


def _max_symbol_ratio(h, alphas):
    """max over [0, pi]^2 of |h^(w)|^2 / (f_s(w)^2 + alpha), both sign flips of w."""
    q1, q2 = O.psf_support(h)
    x = np.linspace(0, np.pi, 181)
    x1, x2 = x[:, None], x[None, :]

    def energy(s1, s2):
        acc = np.zeros((x.size, x.size), dtype=complex)
        for a in range(-q1, q1 + 1):
            for b in range(-q2, q2 + 1):
                acc += h[a + q1, b + q2] * np.exp(-1j * (a * s1 * x1 + b * s2 * x2))
        return np.abs(acc) ** 2

    e = np.maximum(energy(1, 1), energy(-1, 1))
    fs2 = O.symbol(O.symmetrize(h), x, x) ** 2
    return {alpha: float((e / (fs2 + alpha)).max()) for alpha in alphas}


def test_2048_workload_alpha_is_the_smallest_stable_half_decade_value():
    """The same reading for the 21 x 21 asymmetric Gaussian of the 2048^2 precision
    workload: the ratio is below 2 at alpha = 0.1 and above 2 at 0.03."""
    from paper_1211_0393_gb300 import workloads as W
    ratio = _max_symbol_ratio(W.psf_config4(), (0.3, 0.1, 0.03))
    assert ratio[0.3] < ratio[0.1] < 2.0 < ratio[0.03]


def test_bench_alpha_is_the_smallest_stable_half_decade_value():
    """Reading of the unstated alpha (Section 4 leaves it to the user): with tau = 1
    a frequency of the D-Landweber iteration grows when |h^(w)|^2 / (f_s(w)^2 + alpha)
    exceeds 2 (|1 - tau r| > 1), f_s the symbol of the symmetrized PSF and h^ the
    Fourier series of the PSF over both sign flips of w.  For the bench's 15 x 15
    motion PSF the largest ratio over [0, pi]^2 is below 2 at alpha = 0.3 and above 2
    at 0.1, so 0.3 is the smallest stable value of the half-decade grid."""
    from paper_1211_0393_gb300 import workloads as W
    ratio = _max_symbol_ratio(W.psf_config2(), (1.0, 0.3, 0.1))
    assert ratio[1.0] < ratio[0.3] < 2.0 < ratio[0.1]
