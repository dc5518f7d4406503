"""Oracle: the suboptimality measure with the optimal per-band eigenvalues.

Test infrastructure only.  Follows Sec. 3 (bias of the shifted tapers),
Eq. (subopt_measure):
    E_i = (1/K) sum_k |lambda_k^i - lambda_k^0|,
where lambda_k^0 are the nominal eigenvalues (Eq. gep_at_A0) and lambda_k^i
the K largest eigenvalues of the GEP at the analysis band A_i itself,
    R(A_i) w = lambda R(B) w,
R(A_i | n, m) = sin(2 pi f_w d) / (pi d) e^{i 2 pi f_ci d} (Eq. gpss_matrix_a
centred at f_ci, Hermitian), i.e. the GEP the paper's adaptive baseline solves
once per band.  Dense LAPACK per band: small N only.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .gpss import gpss_matrix_a, gpss_matrix_b


def band_eigenvalues(t, fs: float, f_w: float, K: int, freqs) -> np.ndarray:
    """lambda_k^i [len(freqs), K], descending per band."""
    t = np.asarray(t, dtype=np.float64)
    N = t.size
    RB = gpss_matrix_b(t, fs / 2.0).astype(np.complex128)
    out = np.empty((len(freqs), K))
    for j, f in enumerate(np.asarray(freqs, dtype=np.float64)):
        RA = gpss_matrix_a(t, f_w, f)
        RA = RA if np.iscomplexobj(RA) else RA.astype(np.complex128)
        lam = scipy.linalg.eigh(RA, RB, eigvals_only=True, subset_by_index=[N - K, N - 1])
        out[j] = lam[::-1]
    return out


def true_suboptimality(lam0, lam_band) -> np.ndarray:
    """E_i [n] from the nominal eigenvalues lam0 [K] and the per-band ones [n, K]."""
    return np.mean(np.abs(np.asarray(lam_band) - np.asarray(lam0)[None, :]), axis=1)
