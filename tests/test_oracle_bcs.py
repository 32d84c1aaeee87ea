"""Pins of the oracle's comparison boundary conditions (Reflective, Periodic).

* extensions against numpy's 'symmetric' (half-sample) and 'wrap' padding,
* the blur against scipy's convolve2d on those paddings (and 'wrap' boundary),
* Reflective: R of eq. Rn is scipy's orthonormal DCT-II transposed, and
  R^T A(s) R is diagonal with the symbol on k pi/m (Section 2.1),
* Periodic: the circulant is diagonalised by the FFT with the PSF's own
  eigenvalues; A' equals A^T (periodic reblurring is the transpose, Section
  4), so the preconditioner is exactly (A^T A + alpha I)^{-1}.
"""

import numpy as np
import pytest
import scipy.fft
import scipy.signal

import oracle as O


def rand_psf(rng, q1, q2):
    h = rng.uniform(0.0, 1.0, size=(2 * q1 + 1, 2 * q2 + 1))
    return h / h.sum()


@pytest.mark.parametrize("n1,n2,q1,q2", [(9, 12, 3, 4), (16, 16, 7, 7), (5, 7, 4, 2)])
def test_reflective_and_periodic_pads_are_numpy_pads(n1, n2, q1, q2):
    rng = np.random.default_rng(n1 + q2)
    x = rng.standard_normal((n1, n2))
    np.testing.assert_allclose(O.pad_bc(x, q1, q2, O.BC_REFLECTIVE),
                               np.pad(x, ((q1, q1), (q2, q2)), mode="symmetric"), atol=0)
    np.testing.assert_allclose(O.pad_bc(x, q1, q2, O.BC_PERIODIC),
                               np.pad(x, ((q1, q1), (q2, q2)), mode="wrap"), atol=0)
    np.testing.assert_allclose(O.pad_bc(x, q1, q2, O.BC_AR), O.ar_pad(x, q1, q2), atol=0)


@pytest.mark.parametrize("bc,mode", [(O.BC_REFLECTIVE, "symm"), (O.BC_PERIODIC, "wrap")])
def test_blur_matches_scipy_boundary_modes(bc, mode):
    rng = np.random.default_rng(3)
    h = rand_psf(rng, 3, 4)
    x = rng.uniform(0, 1, (20, 17))
    ref = scipy.signal.convolve2d(x, h, mode="same", boundary=mode)
    np.testing.assert_allclose(O.blur_bc(x, h, bc), ref, atol=1e-13)
    np.testing.assert_allclose(O.matrix_dense_bc(h, 20, 17, bc) @ x.ravel(), ref.ravel(), atol=1e-13)


@pytest.mark.parametrize("m", [4, 7, 16, 33])
def test_dct_matrix_is_scipy_dct(m):
    R = O.dct_matrix(m)
    np.testing.assert_allclose(R.T, scipy.fft.dct(np.eye(m), type=2, norm="ortho", axis=0), atol=1e-14)
    np.testing.assert_allclose(R.T @ R, np.eye(m), atol=1e-13)


@pytest.mark.parametrize("n1,n2,q1,q2", [(8, 9, 2, 3), (11, 7, 3, 2)])
def test_reflective_symmetric_matrix_is_diagonalised_by_dct(n1, n2, q1, q2):
    rng = np.random.default_rng(n1 * n2)
    s = O.symmetrize(rand_psf(rng, q1, q2))
    A = O.matrix_dense_bc(s, n1, n2, O.BC_REFLECTIVE)
    R = np.kron(O.dct_matrix(n1), O.dct_matrix(n2))
    L = R.T @ A @ R
    assert np.max(np.abs(L - np.diag(np.diag(L)))) < 1e-13
    np.testing.assert_allclose(np.diag(L).reshape(n1, n2),
                               O.eigenvalues_bc(s, n1, n2, O.BC_REFLECTIVE), atol=1e-13)


def test_periodic_circulant_eigenvalues_and_reblur_transpose():
    rng = np.random.default_rng(5)
    n1, n2 = 8, 10
    h = rand_psf(rng, 2, 3)
    A = O.matrix_dense_bc(h, n1, n2, O.BC_PERIODIC)
    Ar = O.matrix_dense_bc(h[::-1, ::-1], n1, n2, O.BC_PERIODIC)
    np.testing.assert_allclose(Ar, A.T, atol=1e-15)
    # eigen-decomposition by the 2D DFT: A v_k = lambda_k v_k for Fourier modes
    lam_abs = O.eigenvalues_bc(h, n1, n2, O.BC_PERIODIC)
    x = rng.standard_normal((n1, n2))
    Ax = (A @ x.ravel()).reshape(n1, n2)
    # |FFT(Ax)| = |lambda| |FFT(x)|
    np.testing.assert_allclose(np.abs(np.fft.fft2(Ax)), lam_abs * np.abs(np.fft.fft2(x)), atol=1e-12)


def test_periodic_preconditioner_inverts_tikhonov_normal_matrix():
    """Periodic: A' = A^T, so D^{-1} = A^T A + alpha I exactly (FFT algebra)."""
    rng = np.random.default_rng(6)
    n1, n2 = 12, 9
    h = rand_psf(rng, 2, 2)
    prec = O.symprec_setup_bc(h, n1, n2, 0.05, O.BC_PERIODIC)
    y = rng.standard_normal((n1, n2))
    z = O.symprec_solve_bc(prec, y)
    A = O.matrix_dense_bc(h, n1, n2, O.BC_PERIODIC)
    np.testing.assert_allclose((A.T @ A + 0.05 * np.eye(n1 * n2)) @ z.ravel(), y.ravel(), atol=1e-11)


@pytest.mark.parametrize("bc", [O.BC_REFLECTIVE, O.BC_PERIODIC])
def test_restore_bc_brute_force(bc):
    rng = np.random.default_rng(7 + bc)
    n1, n2 = 8, 9
    h = rand_psf(rng, 2, 2)
    f = rng.uniform(0, 1, (n1, n2))
    g = O.blur_bc(f, h, bc) + 1e-3 * rng.standard_normal((n1, n2))
    A = O.matrix_dense_bc(h, n1, n2, bc)
    Ar = O.matrix_dense_bc(h[::-1, ::-1], n1, n2, bc)
    d = O.symprec_setup_bc(h, n1, n2, 0.1, bc)["d"]
    if bc == O.BC_REFLECTIVE:
        R = np.kron(O.dct_matrix(n1), O.dct_matrix(n2))
        D = R @ np.diag(d.ravel()) @ R.T
    else:
        F = np.kron(np.fft.fft(np.eye(n1)), np.fft.fft(np.eye(n2)))
        D = np.real(np.linalg.inv(F) @ np.diag(d.ravel()) @ F)
    x = np.zeros(n1 * n2)
    for _ in range(6):
        x = x + D @ Ar @ (g.ravel() - A @ x)
    xo, _, _ = O.restore_bc(g, h, 0.1, bc, 1.0, 6, True)
    np.testing.assert_allclose(xo.ravel(), x, atol=1e-12 * np.abs(x).max())
