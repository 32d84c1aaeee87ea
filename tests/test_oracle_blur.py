"""Pins of the oracle's AR blur against what the paper and the mathematics fix.

* the paper's printed q = 3 example of C = A - P (proof of Theorem 3),
* three independent assemblies of A_n (extension matrix E, eq. ARnosym1D,
  eqs. 2d_form / 2d_form_block),
* library routines: numpy odd-reflect padding + scipy 'valid' convolution,
* invariants of AR BCs (constants, bilinear images, interior of A' vs A^T).
"""

import numpy as np
import pytest
import scipy.signal

import oracle as O


def rand_psf(rng, q1, q2, normalized=True):
    h = rng.uniform(0.0, 1.0, size=(2 * q1 + 1, 2 * q2 + 1))
    return h / h.sum() if normalized else h


def dense_1d(h1d, n):
    """1D AR matrix via the oracle's 2D assembly with a single row."""
    return O.ar_matrix_dense(np.asarray(h1d).reshape(1, -1), 1, n)


# ---------------------------------------------------------------- golden ---

def _parse_golden(path):
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line.split())
    return rows


def _points(h, q):
    """Point coordinates defined in the proof of Theorem 3, evaluated on h (dict h[k] = h_k)."""
    H = lambda k: h.get(k, 0.0)  # noqa: E731
    pts = {}
    for i in range(0, q + 1):
        pts[f"theta{i}x"], pts[f"theta{i}y"] = H(-i), H(i)
        pts[f"omega{i}x"] = H(-i) + 2 * sum(H(-j) for j in range(i + 1, q + 1))
        pts[f"omega{i}y"] = H(i) + 2 * sum(H(j) for j in range(i + 1, q + 1))
        pts[f"nu{i}x"], pts[f"nu{i}y"] = H(-i) - H(i), H(i) - H(-i)
    pts["theta0"] = H(0)
    pts["zeta0x"], pts["zeta0y"] = H(0) - H(-2), H(0) - H(2)
    pts["zeta1x"], pts["zeta1y"] = H(-1) - H(-3), H(1) - H(3)
    pts["zeta2x"], pts["zeta2y"] = H(-1) - H(3), H(1) - H(-3)
    return pts


def test_golden_q3_example_of_theorem3(golden_dir):
    layout = _parse_golden(f"{golden_dir}/ar1d_q3_n7_C.txt")
    assert len(layout) == 7 and all(len(r) == 7 for r in layout)
    rng = np.random.default_rng(3)
    q, n = 3, 7
    h1d = rng.uniform(0, 1, size=2 * q + 1)
    h1d /= h1d.sum()
    s1d = (h1d + h1d[::-1]) / 2  # any strongly symmetric PSF would do; use eq. simmetrizzata1d
    hd = {k: h1d[k + q] for k in range(-q, q + 1)}
    sd = {k: s1d[k + q] for k in range(-q, q + 1)}
    A = dense_1d(h1d, n)
    P = dense_1d(s1d, n)
    ph, ps = _points(hd, q), _points(sd, q)
    for i in range(n):
        for j in range(n):
            name = layout[i][j]
            if name == ".":
                assert abs(A[i, j]) < 1e-15 and abs(P[i, j]) < 1e-15, (i, j)
                continue
            assert A[i, j] == pytest.approx(ph[name], abs=1e-15), (i, j, name)
            want_p = 0.0 if name.startswith("nu") else ps[name]
            assert P[i, j] == pytest.approx(want_p, abs=1e-15), (i, j, name)


# ------------------------------------------------------- assemblies (T1) ---

@pytest.mark.parametrize("n,q", [(5, 1), (7, 3), (9, 2), (12, 4), (16, 3)])
def test_1d_explicit_form_equals_extension_assembly(n, q):
    rng = np.random.default_rng(n * 10 + q)
    h1d = rng.uniform(0, 1, size=2 * q + 1)
    np.testing.assert_allclose(O.ar_matrix_1d_structured(h1d, n), dense_1d(h1d, n),
                               atol=1e-15, rtol=0)


@pytest.mark.parametrize("n1,n2,q1,q2", [(7, 9, 2, 3), (8, 7, 3, 1), (10, 9, 1, 4), (9, 11, 4, 2)])
def test_2d_block_form_equals_extension_assembly(n1, n2, q1, q2):
    rng = np.random.default_rng(n1 * 100 + n2 * 10 + q1)
    h = rand_psf(rng, q1, q2, normalized=False)
    np.testing.assert_allclose(O.ar_matrix_2d_block(h, n1, n2), O.ar_matrix_dense(h, n1, n2),
                               atol=1e-14, rtol=0)


@pytest.mark.parametrize("n1,n2,q1,q2", [(5, 6, 1, 2), (8, 7, 3, 3), (9, 12, 4, 1), (6, 6, 5, 5),
                                         (11, 10, 0, 3)])
def test_structured_blur_equals_dense_matrix(n1, n2, q1, q2):
    rng = np.random.default_rng(n1 + 7 * n2 + 49 * q1 + q2)
    h = rand_psf(rng, q1, q2)
    x = rng.standard_normal((n1, n2))
    A = O.ar_matrix_dense(h, n1, n2)
    np.testing.assert_allclose(O.ar_blur(x, h).ravel(), A @ x.ravel(), atol=1e-13, rtol=0)
    Ar = O.ar_matrix_dense(h[::-1, ::-1], n1, n2)
    np.testing.assert_allclose(O.ar_reblur(x, h).ravel(), Ar @ x.ravel(), atol=1e-13, rtol=0)


def test_pad_equals_kronecker_of_1d_extensions():
    rng = np.random.default_rng(11)
    n1, n2, q1, q2 = 9, 7, 4, 3
    x = rng.standard_normal((n1, n2))
    E1, E2 = O.ar_extension_1d(n1, q1), O.ar_extension_1d(n2, q2)
    np.testing.assert_allclose(O.ar_pad(x, q1, q2), E1 @ x @ E2.T, atol=1e-14, rtol=0)


# ---------------------------------------------------- library check (T2) ---

@pytest.mark.parametrize("n1,n2,q1,q2", [(33, 40, 4, 4), (64, 64, 7, 7), (20, 17, 7, 2), (8, 9, 7, 8),
                                         (3, 3, 1, 1), (5, 4, 0, 3)])
def test_blur_equals_numpy_odd_reflect_plus_scipy_valid(n1, n2, q1, q2):
    rng = np.random.default_rng(n1 * n2 + q1)
    h = rand_psf(rng, q1, q2)
    x = rng.uniform(0, 1, size=(n1, n2))
    xp = np.pad(x, ((q1, q1), (q2, q2)), mode="reflect", reflect_type="odd")
    np.testing.assert_allclose(O.ar_pad(x, q1, q2), xp, atol=1e-14, rtol=0)
    ref = scipy.signal.convolve2d(xp, h, mode="valid")
    np.testing.assert_allclose(O.ar_blur(x, h), ref, atol=1e-13, rtol=0)
    ref_r = scipy.signal.convolve2d(xp, h[::-1, ::-1], mode="valid")
    np.testing.assert_allclose(O.ar_reblur(x, h), ref_r, atol=1e-13, rtol=0)


# ------------------------------------------------------- invariants (T8) ---

def test_constants_are_preserved_by_any_normalized_psf():
    rng = np.random.default_rng(5)
    h = rand_psf(rng, 3, 5)
    x = np.full((20, 23), 0.37)
    np.testing.assert_allclose(O.ar_blur(x, h), x, atol=1e-14)
    np.testing.assert_allclose(O.ar_reblur(x, h), x, atol=1e-14)


def test_strongly_symmetric_psf_fixes_bilinear_images():
    rng = np.random.default_rng(6)
    s = O.symmetrize(rand_psf(rng, 4, 3))
    i1 = np.arange(17)[:, None]
    i2 = np.arange(21)[None, :]
    x = 0.3 + 0.02 * i1 - 0.05 * i2 + 0.001 * i1 * i2
    np.testing.assert_allclose(O.ar_blur(x, s), x, atol=1e-13)


def test_nonsymmetric_psf_fixes_only_its_mean_shift_of_linear_images():
    """A linear image is mapped to itself shifted by the PSF's first moment."""
    rng = np.random.default_rng(7)
    h = rand_psf(rng, 3, 3)
    q = 3
    m1 = sum(h[a + q, b + q] * a for a in range(-q, q + 1) for b in range(-q, q + 1))
    m2 = sum(h[a + q, b + q] * b for a in range(-q, q + 1) for b in range(-q, q + 1))
    i1 = np.arange(15)[:, None] * np.ones((1, 16))
    i2 = np.ones((15, 1)) * np.arange(16)[None, :]
    x = 0.5 + 0.1 * i1 - 0.2 * i2
    # sum_s h_s x_{i-s} = x_i - 0.1 m1 + 0.2 m2 (linear data is its own AR extension)
    np.testing.assert_allclose(O.ar_blur(x, h), x - 0.1 * m1 + 0.2 * m2, atol=1e-13)


def test_reblur_is_not_the_transpose_but_agrees_in_the_interior():
    rng = np.random.default_rng(8)
    q1 = q2 = 2
    n1, n2 = 9, 10
    h = rand_psf(rng, q1, q2)
    A = O.ar_matrix_dense(h, n1, n2)
    Ar = O.ar_matrix_dense(h[::-1, ::-1], n1, n2)
    assert np.max(np.abs(Ar - A.T)) > 1e-2      # A' != A^T (Section 4, reblurring)
    inner = [i1 * n2 + i2 for i1 in range(2 * q1, n1 - 2 * q1) for i2 in range(2 * q2, n2 - 2 * q2)]
    idx = np.ix_(inner, inner)
    np.testing.assert_allclose(Ar[idx], A.T[idx], atol=1e-15)


def test_pad_rejects_support_wider_than_image():
    with pytest.raises(ValueError):
        O.ar_pad(np.zeros((4, 4)), 4, 1)
