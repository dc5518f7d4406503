"""Oracle: GPSS matrices and the nominal-band tapers (FP64, dense LAPACK).

Test infrastructure only.  Follows:
  * Sec. 2.1, Eq. (gpss_matrix_b): R(B|n,m) = sin(2 pi f_max (t_n-t_m)) / (pi (t_n-t_m)),
    with the diagonal equal to its limit 2 f_max.
  * Sec. 2.3, Eq. (gpss_matrix_a) and Sec. 3.2: R(A0|n,m) = sin(2 pi f_w dt)/(pi dt)
    * exp(i 2 pi f_c0 dt); here the nominal band sits at f_c0 = 0, so R(A0) is
    real and symmetric.
  * Sec. 3.2, Eq. (gep_at_A0): R(A0) w = lambda R(B) w; the K largest
    eigenpairs are kept (Sec. 2.3, end).
  * Sec. 2.2, Eq. (bg_norm_requirement): each taper is scaled so that
    w^* R(B) w = 2 f_w.
The signal band is B = {|f| <= f_max} with f_max = fs/2.

Sign of each eigenvector: the paper does not fix it.  The k-th taper
(0-based) is made to satisfy sum_n w_k(t_n) (t_n - tbar)^(k mod 2) > 0, tbar
being the mean sampling time.  P-hat does not depend on this choice.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def _differences(t: np.ndarray) -> np.ndarray:
    t = np.asarray(t, dtype=np.float64)
    return t[:, None] - t[None, :]


def gpss_matrix_b(t: np.ndarray, f_max: float) -> np.ndarray:
    """R(B) for the band |f| <= f_max (Eq. gpss_matrix_b)."""
    d = _differences(t)
    R = np.empty_like(d)
    off = d != 0.0
    R[off] = np.sin(2.0 * np.pi * f_max * d[off]) / (np.pi * d[off])
    R[~off] = 2.0 * f_max
    return R


def gpss_matrix_a(t: np.ndarray, f_w: float, f_c: float = 0.0) -> np.ndarray:
    """R(A) for the band |f - f_c| <= f_w (Eq. gpss_matrix_a)."""
    d = _differences(t)
    R = np.empty_like(d)
    off = d != 0.0
    R[off] = np.sin(2.0 * np.pi * f_w * d[off]) / (np.pi * d[off])
    R[~off] = 2.0 * f_w
    if f_c != 0.0:
        return R * np.exp(2j * np.pi * f_c * d)
    return R


def sign_convention(w: np.ndarray, t: np.ndarray) -> np.ndarray:
    """Flip rows of w [K, N] so sum_n w_k (t_n - tbar)^(k mod 2) > 0."""
    t = np.asarray(t, dtype=np.float64)
    tc = t - t.mean()
    w = np.array(w, copy=True)
    for k in range(w.shape[0]):
        s = np.sum(w[k] * (tc if (k % 2) else 1.0))
        if s < 0:
            w[k] = -w[k]
    return w


def nominal_tapers(t: np.ndarray, fs: float, f_w: float, K: int):
    """Solve Eq. (gep_at_A0) for the K largest eigenpairs and normalise.

    Returns (w [K, N] float64 in the order of t, lam [K] descending).
    """
    t = np.asarray(t, dtype=np.float64)
    N = t.shape[0]
    if not (1 <= K <= N):
        raise ValueError("need 1 <= K <= N")
    RB = gpss_matrix_b(t, fs / 2.0)
    RA = gpss_matrix_a(t, f_w)
    # LAPACK generalized symmetric-definite solver; eigenvectors satisfy V^T RB V = I
    lam, V = scipy.linalg.eigh(RA, RB, subset_by_index=[N - K, N - 1])
    order = np.argsort(lam)[::-1]
    lam = lam[order]
    V = V[:, order]
    # Eq. (bg_norm_requirement): w^T R(B) w = 2 f_w
    w = (V * np.sqrt(2.0 * f_w)).T
    return sign_convention(w, t), lam


def all_generalized_eigenvalues(t: np.ndarray, fs: float, f_w: float) -> np.ndarray:
    """Every eigenvalue of Eq. (gep), descending (small N only)."""
    RB = gpss_matrix_b(t, fs / 2.0)
    RA = gpss_matrix_a(t, f_w)
    return np.sort(scipy.linalg.eigh(RA, RB, eigvals_only=True))[::-1]


def gpss_rows(t: np.ndarray, rows, f_max: float) -> np.ndarray:
    """Selected rows of R for the band |f| <= f_max (same formula as
    gpss_matrix_b, evaluated only for the requested rows) -- lets tests
    check GEP residuals at sizes where the full N x N matrix is too large."""
    t = np.asarray(t, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    d = t[rows][:, None] - t[None, :]
    R = np.empty_like(d)
    off = d != 0.0
    R[off] = np.sin(2.0 * np.pi * f_max * d[off]) / (np.pi * d[off])
    R[~off] = 2.0 * f_max
    return R


# ---------------------------------------------------------------------------
# sub-bands (Sec. 2.3, Eq. gpss_matrix_b_q; Sec. 3.1 multiband partition)
# ---------------------------------------------------------------------------
def gpss_matrix_b_sub(t: np.ndarray, f_min: float, f_max: float) -> np.ndarray:
    """R(B^q) for the sub-band f_min <= |f| <= f_max (Eq. gpss_matrix_b_q):
    2 cos(pi (f_max + f_min) d) sin(pi (f_max - f_min) d) / (pi d), diagonal 2 (f_max - f_min)."""
    d = _differences(t)
    R = np.empty_like(d)
    off = d != 0.0
    dd = d[off]
    R[off] = 2.0 * np.cos(np.pi * (f_max + f_min) * dd) * np.sin(np.pi * (f_max - f_min) * dd) / (np.pi * dd)
    R[~off] = 2.0 * (f_max - f_min)
    return R


def phase_convention(w: np.ndarray, t: np.ndarray, f_c0: float) -> np.ndarray:
    """Complex tapers: rotate each row so that sum_n w_k(t_n) e^{-i 2 pi f_c0 t_n} (t_n - tbar)^(k mod 2)
    is real and positive (for f_c0 = 0 and real tapers this is sign_convention)."""
    t = np.asarray(t, dtype=np.float64)
    tc = t - t.mean()
    dem = np.exp(-2j * np.pi * f_c0 * t)
    w = np.array(w, dtype=np.complex128, copy=True)
    for k in range(w.shape[0]):
        s = np.sum(w[k] * dem * (tc if (k % 2) else 1.0))
        if abs(s) > 0:
            w[k] *= np.conj(s) / abs(s)
    return w


RANGE_TOL = 1e-9  # eigenvalues of R(B^q) below this fraction of the largest span its numerical null space


def subband_tapers(t: np.ndarray, f_w: float, K: int, f_c0: float, f_min: float, f_max: float):
    """Eq. (gep_at_A0) for the nominal band |f - f_c0| <= f_w inside the sub-band f_min <= |f| <= f_max:
    R(A0) (Hermitian, Eq. gpss_matrix_a with f_c0) w = lambda R(B^q) w, the K largest pairs,
    w^H R(B^q) w = 2 f_w.  Returns (w [K, N] complex128 in the order of t, lam [K] descending).

    R(B^q) is positive definite in exact arithmetic (Sec. 2.3) but numerically singular once N exceeds
    the sub-band's Shannon number 2 (f_max - f_min) T.  Reading: the GEP is solved on the numerical
    range of R(B^q): with R(B^q) = U S U^T and U_r the eigenvectors whose eigenvalues exceed
    RANGE_TOL times the largest, w = U_r S_r^{-1/2} y where y are the top eigenvectors of
    C = S_r^{-1/2} U_r^T R(A0) U_r S_r^{-1/2}; since A0 lies inside B^q, R(B^q) - R(A0) is positive
    semi-definite and the discarded directions carry no energy in A0 either."""
    t = np.asarray(t, dtype=np.float64)
    RB = gpss_matrix_b_sub(t, f_min, f_max)
    RA = gpss_matrix_a(t, f_w, f_c0)
    s, U = np.linalg.eigh(RB)
    keep = s > RANGE_TOL * s.max()
    M = U[:, keep] / np.sqrt(s[keep])[None, :]
    C = np.conj(M.T) @ RA @ M
    C = 0.5 * (C + np.conj(C.T))
    r = C.shape[0]
    if K > r:
        raise ValueError(f"K = {K} exceeds the numerical rank {r} of R(B^q)")
    lam, Y = scipy.linalg.eigh(C, subset_by_index=[r - K, r - 1])
    order = np.argsort(lam)[::-1]
    lam = lam[order]
    w = ((M @ Y[:, order]) * np.sqrt(2.0 * f_w)).T
    return phase_convention(w, t, f_c0), lam
