"""Plain FP64 NumPy oracle of the Anti-Reflective (AR) deblurring method.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  Nothing here is used by,
or shares code with, the CUDA library.

Everything is written from the paper (Dell'Acqua, Serra-Capizzano,
Tablino-Possio, "Optimal preconditioning for image deblurring with
Anti-Reflective boundary conditions"), step by step and in the paper's
notation, in float64, without blocking, fusion or reordering.  Conventions:

* Images are ``n1 x n2`` arrays indexed ``[i1, i2]`` (0-based; the paper is
  1-based), i.e. row-major ("row-wise ordering", Section 1).
* A PSF with support ``q = (q1, q2)`` is a ``(2q1+1) x (2q2+1)`` array with
  ``h[i1 + q1, i2 + q2] = h_{i1,i2}`` (eq. coefficienti_psf).
* The blur is a true convolution, ``g_i = sum_s h_s f_{i-s}`` (eq.
  modello_discreto).

Readings of silent or garbled passages (each one is pinned by a test):

* The bottom-right corner rule of Section 2.2 prints ``2 f_{n1, n1-i2}``; the
  double anti-reflection it describes gives ``2 f_{n1, n2-i2}``, which is what
  :func:`ar_pad` uses.
* The eigenvalue grid after Theorem 2 is garbled.  Theorem 1's ``T_m`` holds
  ``Q_{m-2}``, whose tau grid is ``r pi/(m-1)``, ``r = 1..m-2``; the first and
  last columns of ``T_m`` both take ``x = 0`` (:func:`ar_grid`).
* The iteration of Section 4 uses the reblurred matrix ``A'`` (PSF rotated by
  180 degrees) in place of ``A^H``.
* ``x_0 = 0`` unless given; ``IT`` is the first iteration attaining the
  minimum RRE.

Parity pins: every function is checked in ``tests/test_oracle_*.py`` against
something other than itself (an explicitly assembled matrix, the paper's
printed q = 3 example, library routines, closed forms, brute force).  No
function here is "parity unpinned".
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "BC_AR", "BC_REFLECTIVE", "BC_PERIODIC",
    "pad_bc", "blur_bc", "reblur_bc", "matrix_dense_bc", "extension_1d_bc",
    "dct_matrix", "eigenvalues_bc", "symprec_setup_bc", "symprec_solve_bc",
    "restore_bc",
    "psf_support",
    "ar_extension_1d",
    "ar_pad",
    "ar_blur",
    "ar_reblur",
    "toeplitz_extended_2d",
    "ar_matrix_dense",
    "ar_matrix_1d_structured",
    "ar_matrix_2d_block",
    "symmetrize",
    "symbol",
    "ar_grid",
    "eigenvalues",
    "tikhonov",
    "dst1_matrix",
    "dst1_naive",
    "ar_T",
    "ar_Ttilde",
    "ar_alpha",
    "ar_analysis",
    "ar_synthesis",
    "symprec_setup",
    "symprec_solve",
    "rre",
    "restore",
]


# --------------------------------------------------------------------------
# PSF and boundary conditions (Section 1, Section 2.2)
# --------------------------------------------------------------------------

def psf_support(h: np.ndarray) -> tuple[int, int]:
    """Return ``(q1, q2)`` of a ``(2q1+1) x (2q2+1)`` PSF mask (eq. coefficienti_psf)."""
    h = np.asarray(h)
    if h.ndim != 2 or h.shape[0] % 2 == 0 or h.shape[1] % 2 == 0:
        raise ValueError("PSF must be a 2D array with odd sides")
    return (h.shape[0] - 1) // 2, (h.shape[1] - 1) // 2


def ar_extension_1d(n: int, q: int) -> np.ndarray:
    """Matrix ``E`` of shape ``(n+2q, n)`` of the 1D anti-reflective extension.

    Section 3.1 (and the border rule of Section 2.2): ``f_{1-i} = 2 f_1 -
    f_{1+i}`` and ``f_{n+i} = 2 f_n - f_{n-i}``, ``i = 1..q``.  Row ``r`` of
    ``E`` gives the extended sample with 0-based index ``j = r - q``.
    """
    if q > n - 1:
        raise ValueError("anti-reflection needs q <= n-1")
    E = np.zeros((n + 2 * q, n))
    for r in range(n + 2 * q):
        j = r - q
        if 0 <= j < n:
            E[r, j] = 1.0
        elif j < 0:
            i = -j                      # f_{1-i} = 2 f_1 - f_{1+i}
            E[r, 0] += 2.0
            E[r, i] -= 1.0
        else:
            i = j - (n - 1)             # f_{n+i} = 2 f_n - f_{n-i}
            E[r, n - 1] += 2.0
            E[r, n - 1 - i] -= 1.0
    return E


def ar_pad(x: np.ndarray, q1: int, q2: int) -> np.ndarray:
    """Extend an ``n1 x n2`` image by ``q1`` rows and ``q2`` columns per side.

    Section 2.2, written entry by entry: the four border rules (anti-reflection
    about the first/last row and column) and the four corner rules (double
    anti-reflection ``4 f_c - 2 f - 2 f + f``).  The bottom-right corner uses
    ``f_{n1, n2-i2}`` (the printed ``f_{n1, n1-i2}`` is read as a typo).
    Returns ``xp`` with ``xp[j1 + q1, j2 + q2] = f_{j1, j2}`` (0-based).
    """
    x = np.asarray(x, dtype=np.float64)
    n1, n2 = x.shape
    if q1 > n1 - 1 or q2 > n2 - 1:
        raise ValueError("anti-reflection needs q_j <= n_j - 1")
    xp = np.zeros((n1 + 2 * q1, n2 + 2 * q2))
    f = x  # f[a, b] is the paper's f_{a+1, b+1}
    xp[q1:q1 + n1, q2:q2 + n2] = f
    # borders (Section 2.2, first display of the AR rules)
    for i1 in range(1, q1 + 1):
        for i2 in range(n2):
            xp[q1 - i1, q2 + i2] = 2 * f[0, i2] - f[i1, i2]                    # f_{1-i1, i2}
            xp[q1 + n1 - 1 + i1, q2 + i2] = 2 * f[n1 - 1, i2] - f[n1 - 1 - i1, i2]  # f_{n1+i1, i2}
    for i1 in range(n1):
        for i2 in range(1, q2 + 1):
            xp[q1 + i1, q2 - i2] = 2 * f[i1, 0] - f[i1, i2]                    # f_{i1, 1-i2}
            xp[q1 + i1, q2 + n2 - 1 + i2] = 2 * f[i1, n2 - 1] - f[i1, n2 - 1 - i2]  # f_{i1, n2+i2}
    # corners (Section 2.2, second display of the AR rules)
    for i1 in range(1, q1 + 1):
        for i2 in range(1, q2 + 1):
            # f_{1-i1, 1-i2} = 4 f_{1,1} - 2 f_{1, i2+1} - 2 f_{i1+1, 1} + f_{i1+1, i2+1}
            xp[q1 - i1, q2 - i2] = (4 * f[0, 0] - 2 * f[0, i2] - 2 * f[i1, 0]
                                    + f[i1, i2])
            # f_{1-i1, n2+i2} = 4 f_{1,n2} - 2 f_{1,n2-i2} - 2 f_{i1+1,n2} + f_{i1+1,n2-i2}
            xp[q1 - i1, q2 + n2 - 1 + i2] = (4 * f[0, n2 - 1] - 2 * f[0, n2 - 1 - i2]
                                             - 2 * f[i1, n2 - 1] + f[i1, n2 - 1 - i2])
            # f_{n1+i1, 1-i2} = 4 f_{n1,1} - 2 f_{n1,i2+1} - 2 f_{n1-i1,1} + f_{n1-i1,i2+1}
            xp[q1 + n1 - 1 + i1, q2 - i2] = (4 * f[n1 - 1, 0] - 2 * f[n1 - 1, i2]
                                             - 2 * f[n1 - 1 - i1, 0] + f[n1 - 1 - i1, i2])
            # f_{n1+i1, n2+i2} = 4 f_{n1,n2} - 2 f_{n1,n2-i2} - 2 f_{n1-i1,n2} + f_{n1-i1,n2-i2}
            xp[q1 + n1 - 1 + i1, q2 + n2 - 1 + i2] = (
                4 * f[n1 - 1, n2 - 1] - 2 * f[n1 - 1, n2 - 1 - i2]
                - 2 * f[n1 - 1 - i1, n2 - 1] + f[n1 - 1 - i1, n2 - 1 - i2])
    return xp


def ar_blur(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    """``y = A_n x``: AR extension (Section 2.2) then eq. modello_discreto.

    ``y_{i} = sum_{s=-q}^{q} h_s xt_{i-s}`` over the FOV, ``xt`` the extension.
    """
    h = np.asarray(h, dtype=np.float64)
    q1, q2 = psf_support(h)
    x = np.asarray(x, dtype=np.float64)
    n1, n2 = x.shape
    xp = ar_pad(x, q1, q2)
    y = np.zeros((n1, n2))
    for s1 in range(-q1, q1 + 1):
        for s2 in range(-q2, q2 + 1):
            # xt_{i - s} for all i in the FOV is xp[q1 - s1 + i1, q2 - s2 + i2]
            y += h[s1 + q1, s2 + q2] * xp[q1 - s1:q1 - s1 + n1, q2 - s2:q2 - s2 + n2]
    return y


def ar_reblur(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    """``y = A' x``: the AR matrix of the PSF rotated by 180 degrees (Section 4, reblurring)."""
    return ar_blur(x, np.asarray(h)[::-1, ::-1])


def toeplitz_extended_2d(h: np.ndarray, n1: int, n2: int) -> np.ndarray:
    """The rectangular two-level Toeplitz ``A~`` of eq. modello_discreto_sistema.

    Shape ``N(n) x N(n+2q)``; entry ``[(i1,i2), (r1,r2)] = h_{i - j}`` with
    ``j = r - q`` (0-based extended coordinates), row-wise ordering.
    """
    h = np.asarray(h, dtype=np.float64)
    q1, q2 = psf_support(h)
    m1, m2 = n1 + 2 * q1, n2 + 2 * q2
    At = np.zeros((n1 * n2, m1 * m2))
    for i1 in range(n1):
        for i2 in range(n2):
            for r1 in range(m1):
                s1 = i1 - (r1 - q1)
                if abs(s1) > q1:
                    continue
                for r2 in range(m2):
                    s2 = i2 - (r2 - q2)
                    if abs(s2) > q2:
                        continue
                    At[i1 * n2 + i2, r1 * m2 + r2] = h[s1 + q1, s2 + q2]
    return At


def ar_matrix_dense(h: np.ndarray, n1: int, n2: int) -> np.ndarray:
    """Explicitly assembled ``A_n = A~ (E_{n1} (x) E_{n2})`` (eqs. modello_discreto_sistema, sistema_quadrato)."""
    q1, q2 = psf_support(h)
    E = np.kron(ar_extension_1d(n1, q1), ar_extension_1d(n2, q2))
    return toeplitz_extended_2d(h, n1, n2) @ E


def ar_matrix_1d_structured(h1d: np.ndarray, n: int) -> np.ndarray:
    """1D AR matrix of a generic PSF in the explicit form of eq. ARnosym1D.

    ``A = [[v_0, u^T, 0], [v, B, w], [0, -(Ju)^T, w_0]]`` with
    ``u = [h_{-1}-h_1, ..., h_{-q}-h_q, 0...]``,
    ``v_k = h_k + 2 sum_{j>k} h_j``, ``w_k = h_{-k} + 2 sum_{j>k} h_{-j}`` and
    ``B = T([h_{-q}..h_q]) - H_TL([h_2..h_q]) - H_BR([h_{-2}..h_{-q}])``.
    """
    h1d = np.asarray(h1d, dtype=np.float64)
    q = (h1d.shape[0] - 1) // 2
    if n < 2 * q + 1 or n < 3:
        raise ValueError("the explicit form needs n >= 2q+1")

    def hh(k):  # h_k
        return h1d[k + q] if abs(k) <= q else 0.0

    m = n - 2
    A = np.zeros((n, n))
    v = [hh(k) + 2 * sum(hh(j) for j in range(k + 1, q + 1)) for k in range(q + 1)]
    w = [hh(-k) + 2 * sum(hh(-j) for j in range(k + 1, q + 1)) for k in range(q + 1)]
    u = np.array([hh(-k) - hh(k) for k in range(1, m + 1)])
    # first row and last row
    A[0, 0] = v[0]
    A[0, 1:n - 1] = u
    A[n - 1, 1:n - 1] = -u[::-1]                 # -(J u)^T
    A[n - 1, n - 1] = w[0]
    # first and last columns of the middle block rows
    for k in range(1, q + 1):
        A[k, 0] = v[k]                           # v_1..v_q down the first column
        A[n - 1 - k, n - 1] = w[k]               # w_q..w_1 up the last column
    # B = Toeplitz - H_TL - H_BR, (n-2) x (n-2), 1-based (a, b) inside B
    B = np.zeros((m, m))
    for a in range(1, m + 1):
        for b in range(1, m + 1):
            val = hh(a - b)
            if a + b <= q:                       # top-left Hankel, first row [h_2..h_q]
                val -= hh(a + b)
            ar, br = m + 1 - a, m + 1 - b        # distances from the bottom-right corner
            if ar + br <= q:                     # bottom-right Hankel, last row [..h_{-3}, h_{-2}]
                val -= hh(-(ar + br))
            B[a - 1, b - 1] = val
    A[1:n - 1, 1:n - 1] = B
    return A


def ar_matrix_2d_block(h: np.ndarray, n1: int, n2: int) -> np.ndarray:
    """2D AR matrix in the block form of eqs. 2d_form / 2d_form_block.

    The outer level repeats the 1D pattern of eq. ARnosym1D with the scalar
    ``h_j`` replaced by the block ``H^_j``, the 1D AR matrix (eq. 2d_form_block)
    of PSF row ``j``: ``U = [H^_{-1}-H^_1, ...]``, ``V_j = H^_j + 2 sum_{i>j} H^_i``,
    ``W_j = H^_{-j} + 2 sum_{i>j} H^_{-i}``, ``B = T - H_TL - H_BR`` blockwise.
    """
    h = np.asarray(h, dtype=np.float64)
    q1, q2 = psf_support(h)
    Hb = {j: ar_matrix_1d_structured(h[j + q1, :], n2) for j in range(-q1, q1 + 1)}
    Z = np.zeros((n2, n2))

    def H(k):
        return Hb[k] if abs(k) <= q1 else Z

    m = n1 - 2
    blocks = [[Z for _ in range(n1)] for _ in range(n1)]
    V = [H(k) + 2 * sum((H(j) for j in range(k + 1, q1 + 1)), Z) for k in range(q1 + 1)]
    W = [H(-k) + 2 * sum((H(-j) for j in range(k + 1, q1 + 1)), Z) for k in range(q1 + 1)]
    blocks[0][0] = V[0]
    blocks[n1 - 1][n1 - 1] = W[0]
    for k in range(1, m + 1):
        blocks[0][k] = H(-k) - H(k)                     # U
        blocks[n1 - 1][n1 - 1 - k] = H(k) - H(-k)       # -J U
    for k in range(1, q1 + 1):
        blocks[k][0] = V[k]
        blocks[n1 - 1 - k][n1 - 1] = W[k]
    for a in range(1, m + 1):
        for b in range(1, m + 1):
            blk = H(a - b)
            if a + b <= q1:
                blk = blk - H(a + b)
            ar, br = m + 1 - a, m + 1 - b
            if ar + br <= q1:
                blk = blk - H(-(ar + br))
            blocks[a][b] = blk
    return np.block(blocks)


# --------------------------------------------------------------------------
# Symmetrized PSF, symbol, eigenvalues, Tikhonov filter
# --------------------------------------------------------------------------

def symmetrize(h: np.ndarray) -> np.ndarray:
    """Symmetrized PSF of eq. simmetrizzata2d (Theorem 4, the optimal preconditioner's PSF).

    ``s_{+-i1,+-i2} = (h_{-i1,-i2} + h_{-i1,i2} + h_{i1,-i2} + h_{i1,i2}) / 4``.
    """
    h = np.asarray(h, dtype=np.float64)
    q1, q2 = psf_support(h)
    s = np.zeros_like(h)
    for i1 in range(-q1, q1 + 1):
        for i2 in range(-q2, q2 + 1):
            s[i1 + q1, i2 + q2] = (h[-i1 + q1, -i2 + q2] + h[-i1 + q1, i2 + q2]
                                   + h[i1 + q1, -i2 + q2] + h[i1 + q1, i2 + q2]) / 4.0
    return s


def symbol(s: np.ndarray, x1: np.ndarray, x2: np.ndarray) -> np.ndarray:
    """Generating function of eq. funzione_generatrice on the grid ``x1 x x2``.

    ``f = h00 + 2 sum h_{a,0} cos(a x1) + 2 sum h_{0,b} cos(b x2)
    + 4 sum sum h_{a,b} cos(a x1) cos(b x2)`` (``a, b >= 1``), for a strongly
    symmetric mask (only the ``a, b >= 0`` quadrant is read).
    """
    s = np.asarray(s, dtype=np.float64)
    q1, q2 = psf_support(s)
    x1 = np.asarray(x1, dtype=np.float64)[:, None]
    x2 = np.asarray(x2, dtype=np.float64)[None, :]
    f = np.full((x1.shape[0], x2.shape[1]), s[q1, q2])
    for a in range(1, q1 + 1):
        f = f + 2 * s[q1 + a, q2] * np.cos(a * x1)
    for b in range(1, q2 + 1):
        f = f + 2 * s[q1, q2 + b] * np.cos(b * x2)
    for a in range(1, q1 + 1):
        for b in range(1, q2 + 1):
            f = f + 4 * s[q1 + a, q2 + b] * np.cos(a * x1) * np.cos(b * x2)
    return f


def ar_grid(m: int) -> np.ndarray:
    """Evaluation grid of Theorem 2 in the column order of ``T_m`` (Theorem 1).

    Column 0 and column ``m-1`` (the anti-reflection centres) take ``x = 0``;
    column ``r = 1..m-2`` takes the tau grid of ``Q_{m-2}``, ``r pi / (m-1)``.
    """
    x = np.zeros(m)
    x[1:m - 1] = np.arange(1, m - 1) * np.pi / (m - 1)
    return x


def eigenvalues(s: np.ndarray, n1: int, n2: int) -> np.ndarray:
    """Eigenvalues ``lambda[i1, i2]`` of ``A_n(s)`` in ``T_n`` order (Theorem 2)."""
    return symbol(s, ar_grid(n1), ar_grid(n2))


def tikhonov(lam: np.ndarray, alpha: float) -> np.ndarray:
    """Tikhonov filter eq. TikFilter: ``d = 1 / (|lambda|^2 + alpha)``."""
    lam = np.asarray(lam, dtype=np.float64)
    return 1.0 / (np.abs(lam) ** 2 + alpha)


# --------------------------------------------------------------------------
# tau (DST-I) transform and the AR transform (eq. Qn, Theorem 1)
# --------------------------------------------------------------------------

def dst1_matrix(M: int) -> np.ndarray:
    """``Q_M = sqrt(2/(M+1)) sin(s t pi / (M+1))``, ``s, t = 1..M`` (eq. Qn)."""
    st = np.outer(np.arange(1, M + 1), np.arange(1, M + 1))
    return np.sqrt(2.0 / (M + 1)) * np.sin(st * np.pi / (M + 1))


def dst1_naive(y: np.ndarray) -> np.ndarray:
    """``Q_M y`` by the O(M^2) double loop of eq. Qn (small inputs only)."""
    y = np.asarray(y, dtype=np.float64)
    M = y.shape[0]
    out = np.zeros(M)
    c = np.sqrt(2.0 / (M + 1))
    for s in range(1, M + 1):
        acc = 0.0
        for t in range(1, M + 1):
            acc += np.sin(s * t * np.pi / (M + 1)) * y[t - 1]
        out[s - 1] = c * acc
    return out


def _p(m: int) -> np.ndarray:
    """``p_j = 1 - j/(m-1)``, ``j = 1..m-2`` (Theorem 1)."""
    return 1.0 - np.arange(1, m - 1) / (m - 1)


def ar_alpha(m: int) -> float:
    """``alpha_m``: makes the first and last columns of ``T_m`` unit vectors (Theorem 1)."""
    p = _p(m)
    return float(np.sqrt(1.0 + p @ p))


def ar_T(m: int) -> np.ndarray:
    """``T_m = [[a^-1, 0, 0], [a^-1 p, Q_{m-2}, a^-1 J p], [0, 0, a^-1]]`` (Theorem 1)."""
    if m < 3:
        raise ValueError("T_m needs m >= 3")
    a = ar_alpha(m)
    p = _p(m)
    T = np.zeros((m, m))
    T[0, 0] = 1.0 / a
    T[m - 1, m - 1] = 1.0 / a
    T[1:m - 1, 0] = p / a
    T[1:m - 1, m - 1] = p[::-1] / a
    T[1:m - 1, 1:m - 1] = dst1_matrix(m - 2)
    return T


def ar_Ttilde(m: int) -> np.ndarray:
    """``T~_m = [[a, 0, 0], [-Q p, Q, -Q J p], [0, 0, a]]``, ``Q = Q_{m-2}`` (Theorem 1)."""
    if m < 3:
        raise ValueError("T~_m needs m >= 3")
    a = ar_alpha(m)
    p = _p(m)
    Q = dst1_matrix(m - 2)
    Tt = np.zeros((m, m))
    Tt[0, 0] = a
    Tt[m - 1, m - 1] = a
    Tt[1:m - 1, 0] = -Q @ p
    Tt[1:m - 1, m - 1] = -Q @ p[::-1]
    Tt[1:m - 1, 1:m - 1] = Q
    return Tt


def ar_analysis(y: np.ndarray) -> np.ndarray:
    """``T~_n y`` with ``T~_n = T~_{n1} (x) T~_{n2}`` (Theorem 1), as ``T~1 Y T~2^T``."""
    n1, n2 = y.shape
    return ar_Ttilde(n1) @ np.asarray(y, dtype=np.float64) @ ar_Ttilde(n2).T


def ar_synthesis(w: np.ndarray) -> np.ndarray:
    """``T_n w`` with ``T_n = T_{n1} (x) T_{n2}`` (Theorem 1), as ``T1 W T2^T``."""
    n1, n2 = w.shape
    return ar_T(n1) @ np.asarray(w, dtype=np.float64) @ ar_T(n2).T


# --------------------------------------------------------------------------
# Optimal preconditioner and the (D-)Landweber iteration (Section 4)
# --------------------------------------------------------------------------

def symprec_setup(h: np.ndarray, n1: int, n2: int, alpha: float) -> dict:
    """Preconditioner data: symmetrized PSF (eq. simmetrizzata2d), its AR
    eigenvalues (Theorem 2) and the Tikhonov-filtered ``d`` (eq. TikFilter)."""
    s = symmetrize(h)
    lam = eigenvalues(s, n1, n2)
    return {"s": s, "lam": lam, "d": tikhonov(lam, alpha), "n1": n1, "n2": n2}


def symprec_solve(prec: dict, y: np.ndarray) -> np.ndarray:
    """``z = D y = T_n diag(d) T~_n y`` (Theorem 1 with the eigenvalues ``d`` of ``D``)."""
    return ar_synthesis(prec["d"] * ar_analysis(y))


def rre(x: np.ndarray, f: np.ndarray) -> float:
    """Relative restoration error ``||x - f||_F / ||f||_F`` (Section 4)."""
    return float(np.linalg.norm(x - f) / np.linalg.norm(f))


def restore(g, h, alpha, tau=1.0, iters=20, precondition=True, x0=None, f_true=None,
            each=None):
    """(D-)Landweber with reblurring: eqs. LandweberMeth / DLandweberMeth.

    ``x_{k+1} = x_k + tau D A'(g - A x_k)``, ``D = I`` when ``precondition`` is
    false.  Returns ``(x, rre_trace, best_iter)``; ``rre_trace[k]`` is the RRE
    of ``x_{k+1}`` and ``best_iter`` the first ``k+1`` attaining the minimum
    (the tables' IT), both ``None`` without ``f_true``.  ``each(k, x_k)``, when
    given, is called with every iterate ``k = 1 .. iters`` (for per-iterate
    comparisons; it does not change the iteration).
    """
    g = np.asarray(g, dtype=np.float64)
    n1, n2 = g.shape
    prec = symprec_setup(h, n1, n2, alpha) if precondition else None
    x = np.zeros((n1, n2)) if x0 is None else np.array(x0, dtype=np.float64)
    trace = [] if f_true is not None else None
    for k in range(1, iters + 1):
        r = g - ar_blur(x, h)
        z = ar_reblur(r, h)
        if precondition:
            z = symprec_solve(prec, z)
        x = x + tau * z
        if trace is not None:
            trace.append(rre(x, f_true))
        if each is not None:
            each(k, x)
    best = None
    if trace is not None and trace:
        best = int(np.argmin(np.asarray(trace))) + 1
    return x, (np.asarray(trace) if trace is not None else None), best


# --------------------------------------------------------------------------
# Comparison boundary conditions (Section 2.1 Reflective; periodic, Section 2)
# --------------------------------------------------------------------------

BC_AR, BC_REFLECTIVE, BC_PERIODIC = 0, 1, 2


def extension_1d_bc(n: int, q: int, bc: int) -> np.ndarray:
    """``(n+2q) x n`` extension matrix of one axis for the three BCs.

    Reflective (Section 2.1): ``f_{1-i} = f_i``, ``f_{n+i} = f_{n+1-i}``.
    Periodic: ``f_{1-i} = f_{n+1-i}``, ``f_{n+i} = f_i``.  AR: Section 2.2.
    """
    if bc == BC_AR:
        return ar_extension_1d(n, q)
    E = np.zeros((n + 2 * q, n))
    for r in range(n + 2 * q):
        j = r - q
        if 0 <= j < n:
            E[r, j] = 1.0
        elif bc == BC_REFLECTIVE:
            E[r, -j - 1 if j < 0 else 2 * n - 1 - j] = 1.0
        else:
            E[r, j % n] = 1.0
    return E


def pad_bc(x: np.ndarray, q1: int, q2: int, bc: int) -> np.ndarray:
    """Extend an image by the rules of ``bc`` (rows first, then columns)."""
    if bc == BC_AR:
        return ar_pad(x, q1, q2)
    x = np.asarray(x, dtype=np.float64)
    n1, n2 = x.shape
    if q1 > n1 or q2 > n2:
        raise ValueError("extension needs q_j <= n_j")
    return extension_1d_bc(n1, q1, bc) @ x @ extension_1d_bc(n2, q2, bc).T


def blur_bc(x: np.ndarray, h: np.ndarray, bc: int) -> np.ndarray:
    """``y_i = sum_s h_s xt_{i-s}`` (eq. modello_discreto) over the ``bc`` extension."""
    h = np.asarray(h, dtype=np.float64)
    q1, q2 = psf_support(h)
    n1, n2 = np.asarray(x).shape
    xp = pad_bc(x, q1, q2, bc)
    y = np.zeros((n1, n2))
    for s1 in range(-q1, q1 + 1):
        for s2 in range(-q2, q2 + 1):
            y += h[s1 + q1, s2 + q2] * xp[q1 - s1:q1 - s1 + n1, q2 - s2:q2 - s2 + n2]
    return y


def reblur_bc(x: np.ndarray, h: np.ndarray, bc: int) -> np.ndarray:
    """The matrix of the PSF rotated by 180 degrees under the same BC (Section 4)."""
    return blur_bc(x, np.asarray(h)[::-1, ::-1], bc)


def matrix_dense_bc(h: np.ndarray, n1: int, n2: int, bc: int) -> np.ndarray:
    """Dense ``A_n = A~ (E_{n1} (x) E_{n2})`` for the BC."""
    q1, q2 = psf_support(h)
    E = np.kron(extension_1d_bc(n1, q1, bc), extension_1d_bc(n2, q2, bc))
    return toeplitz_extended_2d(h, n1, n2) @ E


def dct_matrix(m: int) -> np.ndarray:
    """Orthogonal ``R_m`` of eq. Rn with columns the DCT-III basis vectors:
    ``R[t, k] = sqrt((2 - delta_{k,0})/m) cos(k (t + 1/2) pi / m)`` (0-based);
    reflective matrices of strongly symmetric PSFs are ``R diag(lambda) R^T``."""
    t = np.arange(m)[:, None]
    k = np.arange(m)[None, :]
    R = np.sqrt(2.0 / m) * np.cos(k * (t + 0.5) * np.pi / m)
    R[:, 0] = np.sqrt(1.0 / m)
    return R


def eigenvalues_bc(h: np.ndarray, n1: int, n2: int, bc: int) -> np.ndarray:
    """Eigenvalue magnitudes used by the preconditioner of each BC (Section 4).

    AR and Reflective: the symbol of the symmetrized PSF (eq. simmetrizzata2d,
    eq. funzione_generatrice) on the AR grid (Theorem 2) or on ``k pi / m``
    (Section 2.1).  Periodic: ``|lambda|`` of the circulant of the PSF itself,
    ``lambda(w) = sum_s h_s exp(-i s . w)`` at ``w = 2 pi k / m``.
    """
    if bc == BC_AR:
        return eigenvalues(symmetrize(h), n1, n2)
    if bc == BC_REFLECTIVE:
        return symbol(symmetrize(h), np.arange(n1) * np.pi / n1, np.arange(n2) * np.pi / n2)
    h = np.asarray(h, dtype=np.float64)
    q1, q2 = psf_support(h)
    w1 = 2.0 * np.pi * np.arange(n1) / n1
    w2 = 2.0 * np.pi * np.arange(n2) / n2
    lam = np.zeros((n1, n2), dtype=complex)
    for a in range(-q1, q1 + 1):
        for b in range(-q2, q2 + 1):
            lam += h[a + q1, b + q2] * np.exp(-1j * (a * w1[:, None] + b * w2[None, :]))
    return np.abs(lam)


def symprec_setup_bc(h: np.ndarray, n1: int, n2: int, alpha: float, bc: int) -> dict:
    lam = eigenvalues_bc(h, n1, n2, bc)
    return {"lam": lam, "d": tikhonov(lam, alpha), "bc": bc, "n1": n1, "n2": n2}


def symprec_solve_bc(prec: dict, y: np.ndarray) -> np.ndarray:
    """``D y`` in the BC's algebra: AR ``T diag(d) T~`` (Theorem 1), Reflective
    ``R diag(d) R^T`` (eq. Rn), Periodic ``F^* diag(d) F`` (numpy FFT)."""
    bc, d = prec["bc"], prec["d"]
    y = np.asarray(y, dtype=np.float64)
    if bc == BC_AR:
        return symprec_solve(prec, y)
    if bc == BC_REFLECTIVE:
        R1, R2 = dct_matrix(y.shape[0]), dct_matrix(y.shape[1])
        return R1 @ (d * (R1.T @ y @ R2)) @ R2.T
    return np.real(np.fft.ifft2(d * np.fft.fft2(y)))


def restore_bc(g, h, alpha, bc, tau=1.0, iters=20, precondition=True, f_true=None):
    """(D-)Landweber with reblurring under the BC (eqs. LandweberMeth / DLandweberMeth)."""
    g = np.asarray(g, dtype=np.float64)
    n1, n2 = g.shape
    prec = symprec_setup_bc(h, n1, n2, alpha, bc) if precondition else None
    x = np.zeros((n1, n2))
    trace = [] if f_true is not None else None
    for _ in range(iters):
        z = reblur_bc(g - blur_bc(x, h, bc), h, bc)
        if precondition:
            z = symprec_solve_bc(prec, z)
        x = x + tau * z
        if trace is not None:
            trace.append(rre(x, f_true))
    best = int(np.argmin(trace)) + 1 if trace else None
    return x, (np.asarray(trace) if trace is not None else None), best
