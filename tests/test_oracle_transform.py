"""Pins of the oracle's transforms, symbol and eigenvalues.

* eq. Qn against scipy's orthonormal DST-I and against Q^2 = I,
* Theorem 1: T~_m T_m = I, unit first/last columns, T~_m = inv(T_m) (numpy),
* Theorem 2: T~ A(s) T is diagonal (dense A from the extension assembly),
  its diagonal is the symbol on the AR grid, the four corners equal sum(s),
  and the multiplicities match the theorem's four groups,
* the symbol of the symmetrized PSF equals the cosine sum over the raw PSF.
"""

import numpy as np
import pytest
import scipy.fft

import oracle as O


def rand_psf(rng, q1, q2):
    h = rng.uniform(0.0, 1.0, size=(2 * q1 + 1, 2 * q2 + 1))
    return h / h.sum()


@pytest.mark.parametrize("M", [1, 2, 5, 16, 33, 126])
def test_Q_is_scipy_orthonormal_dst1_and_an_involution(M):
    Q = O.dst1_matrix(M)
    ref = scipy.fft.dst(np.eye(M), type=1, norm="ortho", axis=0)
    np.testing.assert_allclose(Q, ref, atol=1e-14)
    np.testing.assert_allclose(Q, Q.T, atol=0)
    np.testing.assert_allclose(Q @ Q, np.eye(M), atol=1e-13)


def test_naive_dst_loop_matches_matrix():
    rng = np.random.default_rng(1)
    y = rng.standard_normal(23)
    np.testing.assert_allclose(O.dst1_naive(y), scipy.fft.dst(y, type=1, norm="ortho"), atol=1e-13)


@pytest.mark.parametrize("m", [3, 4, 7, 16, 65])
def test_theorem1_inverse_pair(m):
    T, Tt = O.ar_T(m), O.ar_Ttilde(m)
    np.testing.assert_allclose(Tt @ T, np.eye(m), atol=1e-13)
    np.testing.assert_allclose(np.linalg.inv(T), Tt, atol=1e-12)
    assert np.linalg.norm(T[:, 0]) == pytest.approx(1.0, abs=1e-15)
    assert np.linalg.norm(T[:, -1]) == pytest.approx(1.0, abs=1e-15)
    # the middle columns are the orthonormal tau eigenvectors padded with zeros
    np.testing.assert_allclose(T[1:-1, 1:-1].T @ T[1:-1, 1:-1], np.eye(m - 2), atol=1e-13)
    # first column is the linear ramp from 1 to 0 (times 1/alpha_m)
    a = O.ar_alpha(m)
    np.testing.assert_allclose(T[:, 0] * a, 1 - np.arange(m) / (m - 1), atol=1e-15)


@pytest.mark.parametrize("n1,n2,q1,q2", [(5, 5, 1, 1), (7, 9, 2, 3), (10, 8, 3, 2), (12, 11, 4, 4),
                                         (6, 13, 3, 5)])
def test_theorem2_transform_diagonalizes_symmetric_ar_matrix(n1, n2, q1, q2):
    rng = np.random.default_rng(n1 * n2 + q1 * 3 + q2)
    s = O.symmetrize(rand_psf(rng, q1, q2))
    A = O.ar_matrix_dense(s, n1, n2)
    T = np.kron(O.ar_T(n1), O.ar_T(n2))
    Tt = np.kron(O.ar_Ttilde(n1), O.ar_Ttilde(n2))
    L = Tt @ A @ T
    off = L - np.diag(np.diag(L))
    assert np.max(np.abs(off)) < 1e-13
    lam = O.eigenvalues(s, n1, n2)
    np.testing.assert_allclose(np.diag(L).reshape(n1, n2), lam, atol=1e-13)
    # corners: eigenvalue sum(s) = 1 with multiplicity 4
    for c in [(0, 0), (0, n2 - 1), (n1 - 1, 0), (n1 - 1, n2 - 1)]:
        assert lam[c] == pytest.approx(1.0, abs=1e-14)
    # first/last rows: the tau eigenvalues of the column-summed PSF h^{r}, twice
    hr = s.sum(axis=0)
    Ar1 = O.ar_matrix_dense(hr.reshape(1, -1), 1, n2)
    tau_r = np.sort(np.linalg.eigvals(Ar1[1:-1, 1:-1]).real)
    np.testing.assert_allclose(np.sort(lam[0, 1:-1]), tau_r, atol=1e-13)
    np.testing.assert_allclose(np.sort(lam[-1, 1:-1]), tau_r, atol=1e-13)
    hc = s.sum(axis=1)
    Ac1 = O.ar_matrix_dense(hc.reshape(1, -1), 1, n1)
    tau_c = np.sort(np.linalg.eigvals(Ac1[1:-1, 1:-1]).real)
    np.testing.assert_allclose(np.sort(lam[1:-1, 0]), tau_c, atol=1e-13)
    # the full spectrum agrees with a dense eigensolver
    np.testing.assert_allclose(np.sort(np.linalg.eigvals(A).real), np.sort(lam.ravel()), atol=1e-10)


def test_symbol_of_symmetrized_psf_is_cosine_sum_over_raw_psf():
    rng = np.random.default_rng(4)
    q1, q2 = 3, 5
    h = rand_psf(rng, q1, q2)
    x1 = rng.uniform(0, np.pi, 7)
    x2 = rng.uniform(0, np.pi, 9)
    raw = np.zeros((7, 9))
    for a in range(-q1, q1 + 1):
        for b in range(-q2, q2 + 1):
            raw += h[a + q1, b + q2] * np.cos(a * x1)[:, None] * np.cos(b * x2)[None, :]
    np.testing.assert_allclose(O.symbol(O.symmetrize(h), x1, x2), raw, atol=1e-14)


def test_symbol_at_origin_is_psf_sum_and_grid_layout():
    h = rand_psf(np.random.default_rng(9), 2, 2)
    assert O.symbol(O.symmetrize(h), [0.0], [0.0])[0, 0] == pytest.approx(1.0, abs=1e-15)
    g = O.ar_grid(6)
    np.testing.assert_allclose(g, [0, np.pi / 5, 2 * np.pi / 5, 3 * np.pi / 5, 4 * np.pi / 5, 0])


def test_analysis_synthesis_roundtrip_and_kronecker_order():
    rng = np.random.default_rng(12)
    y = rng.standard_normal((9, 6))
    np.testing.assert_allclose(O.ar_synthesis(O.ar_analysis(y)), y, atol=1e-12)
    Tt = np.kron(O.ar_Ttilde(9), O.ar_Ttilde(6))
    np.testing.assert_allclose(O.ar_analysis(y).ravel(), Tt @ y.ravel(), atol=1e-12)


def test_tikhonov_filter():
    lam = np.array([1.0, 0.5, -0.25, 0.0])
    np.testing.assert_allclose(O.tikhonov(lam, 0.01), [1 / 1.01, 1 / 0.26, 1 / 0.0725, 100.0])
