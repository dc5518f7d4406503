"""Oracle: eigencoefficients, eigenspectra and the multitaper estimate.

Test infrastructure only.  Follows:
  * Sec. 3.2, Eq. (eigencoefficients) and Table 1 step 4:
        J_k(A_i) = sum_n [w_k^*(t_n) x(t_n)] exp(-i 2 pi df_i t_n),
    with nominal centre f_c0 = 0 so that the shift df_i equals the band
    centre f_i = f_lo + i*df.  Evaluated as the direct sum (oracle/nudft.c).
  * Sec. 3.2, Eq. (power_spectrum_estimator) and Table 1 step 5:
        P(A_i) = (1/K) sum_k |J_k(A_i)|^2.
  * Eigenspectra |J_k(A_i)|^2 (the per-taper terms of that average).
"""
from __future__ import annotations

import numpy as np

from . import _native


def band_centres(f_lo: float, df: float, I: int) -> np.ndarray:
    return f_lo + np.arange(I) * df


def eigencoefficients(t, x, w, f_lo: float, df: float, I: int, idx=None,
                      nthreads: int = 0) -> np.ndarray:
    """J [K, len(idx)] complex128 for a single signal x [N]."""
    w = np.atleast_2d(np.asarray(w))
    x = np.asarray(x, dtype=np.float64 if not np.iscomplexobj(x) else np.complex128)
    c = np.conj(w) * x[None, :]
    if idx is None:
        idx = np.arange(I, dtype=np.int64)
    return _native.nudft(t, c, f_lo, df, np.asarray(idx, dtype=np.int64), nthreads)


def eigenspectra(J: np.ndarray) -> np.ndarray:
    return np.abs(J) ** 2


def psd(J: np.ndarray) -> np.ndarray:
    """Eq. (power_spectrum_estimator): mean over tapers of |J_k|^2."""
    return np.mean(np.abs(J) ** 2, axis=0)


def m2nufft(t, x, w, f_lo: float, df: float, I: int, idx=None, nthreads: int = 0):
    """Full hot path for one signal: returns (J [K, n], E [K, n], P [n])."""
    J = eigencoefficients(t, x, w, f_lo, df, I, idx, nthreads)
    E = eigenspectra(J)
    return J, E, psd(J)
