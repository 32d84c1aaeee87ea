"""Host check of the algebra the GPU periodic preconditioner is built on.

The circulant solve D y = F* diag(d) F y (d real, d(-k) = d(k)) is applied on
the GPU in the real separable Hartley basis, as
    D y = H (d_e o Y^) H^T - H' (d_o o Y^) H'^T,   Y^ = H Y H^T,
with H[s, t] = cas(2 pi s t / m) / sqrt(m), H'[s, t] = cas(-2 pi s t / m) /
sqrt(m), d_e the part of d even in each frequency and d_o the part odd in
both.  This restates that identity in numpy and checks it against the
oracle's FFT solve, for PSFs with and without axis symmetry (d_o = 0 only in
the first case)."""

import numpy as np
import pytest

from oracle import ar_oracle as O


def _hartley(m, sign=1):
    s = np.arange(m)
    ang = 2.0 * np.pi * np.outer(s, s) / m
    return (np.cos(ang) + sign * np.sin(ang)) / np.sqrt(m)


def _even_odd(d):
    n1 = d.shape[0]
    dm = d[(-np.arange(n1)) % n1, :]
    return 0.5 * (d + dm), 0.5 * (d - dm)


@pytest.mark.parametrize("n1,n2,kind", [(8, 8, "motion"), (9, 12, "random"), (16, 7, "gauss")])
def test_hartley_split_equals_fft_solve(n1, n2, kind):
    rng = np.random.default_rng(7 + n1 * n2)
    if kind == "gauss":
        a = np.arange(-2, 3)
        h = np.exp(-0.3 * a[:, None] ** 2 - 0.7 * a[None, :] ** 2)
    elif kind == "motion":
        h = np.eye(5)[:, ::-1] + 0.1 * np.eye(5)
    else:
        h = rng.random((3, 5))
    h = h / h.sum()
    prec = O.symprec_setup_bc(h, n1, n2, 0.05, O.BC_PERIODIC)
    d = prec["d"]
    y = rng.standard_normal((n1, n2))
    H1, H2 = _hartley(n1), _hartley(n2)
    Hp1, Hp2 = _hartley(n1, -1), _hartley(n2, -1)
    de, do = _even_odd(d)
    Yh = H1 @ y @ H2.T
    z = H1 @ (de * Yh) @ H2.T - Hp1 @ (do * Yh) @ Hp2.T
    ref = O.symprec_solve_bc(prec, y)
    assert np.max(np.abs(z - ref)) <= 1e-12 * np.max(np.abs(ref))
    if kind == "gauss":
        assert np.max(np.abs(do)) <= 1e-15 * np.max(d)
    else:
        assert np.max(np.abs(do)) > 1e-6 * np.max(d)


def test_hartley_is_symmetric_orthogonal():
    for m in (1, 2, 7, 16):
        H = _hartley(m)
        assert np.allclose(H, H.T) and np.allclose(H @ H, np.eye(m), atol=1e-13)
