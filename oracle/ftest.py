"""Oracle: Thomson's F-statistic for nonuniformly sampled series.

Test infrastructure only (imported by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg, never by the product path).

Follows Sec. 3 (periodicity test), Eq. (f_stat) and the amplitude estimate
that follows it, in the paper's order:
  * W_k^0(0): the eigencoefficient transform of the nominal taper w_k^0 at
    zero shift, which is the plain sum of the taper weights over the samples;
  * C_i = sum_k J_k(A_i) W_k^0(0) / sum_k [W_k^0(0)]^2   (amplitude estimate);
  * F_i = |C_i|^2 (K - 1) sum_k [W_k^0(0)]^2 / sum_k |J_k(A_i) - C_i W_k^0(0)|^2,
    distributed as F(2, 2K - 2) when the band holds no spectral line.
The paper states the statistic for bands with 2 f_ci > f_w (away from zero
frequency); the formulas are evaluated as written everywhere.
"""
from __future__ import annotations

import numpy as np


def taper_dc(w: np.ndarray) -> np.ndarray:
    """W_k^0(0) = sum_n w_k^0(t_n), one value per taper [K]."""
    return np.asarray(w).sum(axis=1)


def line_amplitude(J: np.ndarray, W: np.ndarray) -> np.ndarray:
    """C_i for every band: J [K, nb] complex, W [K] -> [nb] complex."""
    W = np.asarray(W, dtype=np.float64)
    return (J * W[:, None]).sum(axis=0) / np.sum(W * W)


def f_statistic(J: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Eq. (f_stat) for every band: J [K, nb] eigencoefficients of one signal,
    w [K, N] the tapers they were computed with -> F [nb] (FP64)."""
    J = np.asarray(J, dtype=np.complex128)
    K = J.shape[0]
    W = taper_dc(w).astype(np.float64)
    C = line_amplitude(J, W)
    num = np.abs(C) ** 2 * (K - 1) * np.sum(W * W)
    den = np.sum(np.abs(J - C[None, :] * W[:, None]) ** 2, axis=0)
    return num / den
