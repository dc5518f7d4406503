"""Oracle: sidelobe-leakage (suboptimality) estimate of the shifted tapers.

Test infrastructure only.  Follows App. B, Eq. (lambda_hat_ki):

    lambda_hat_k^i = lambda_k^0 * 2 f_w / D_k^i,
    D_k^i = (E_i w_k^0)^* R(B) (E_i w_k^0),   E_i = diag(exp(i 2 pi df_i t_n)),

and the leakage estimate L_k^i = |lambda_k^0 - lambda_hat_k^i| with its taper
average E_i = (1/K) sum_k L_k^i (the estimate of Eq. (subopt_measure)).
The paper's Theorem 1 writes the left side as L itself; the reading taken
here is the difference between the nominal eigenvalue and the Rayleigh
quotient of the shifted taper.

D is formed densely: D = v^H R(B) v with v_n = w_n exp(i 2 pi f t_n).  Cost
is O(N^2) per band, so callers pass a subset of bands for large N.  The
phases use times re-centred at their mean; D depends only on t_n - t_m.
For sub-band plans (complex tapers normalised to w^H R(B^q) w = 2 f_w) the
same estimate is taken with R(B^q) and the shift from the nominal centre.
"""
from __future__ import annotations

import numpy as np

from .gpss import gpss_matrix_b, gpss_matrix_b_sub


def leakage_denominator(t, w, fs: float, freqs) -> np.ndarray:
    """D [K, len(freqs)] real."""
    t = np.asarray(t, dtype=np.float64)
    tc = t - t.mean()
    w = np.atleast_2d(np.asarray(w, dtype=np.float64))
    RB = gpss_matrix_b(t, fs / 2.0)
    freqs = np.asarray(freqs, dtype=np.float64)
    D = np.empty((w.shape[0], freqs.shape[0]))
    for j, f in enumerate(freqs):
        e = np.exp(2j * np.pi * f * tc)
        V = w * e[None, :]                     # rows: E_i w_k
        RV = V @ RB                            # RB symmetric
        D[:, j] = np.real(np.sum(np.conj(V) * RV, axis=1))
    return D


def leakage(lam, D, f_w: float):
    """(L [K, n], Ehat [n]) from eigenvalues lam [K] and denominators D [K, n]."""
    lam = np.asarray(lam, dtype=np.float64)[:, None]
    lam_hat = lam * (2.0 * f_w) / D
    L = np.abs(lam - lam_hat)
    return L, L.mean(axis=0)


def leakage_at(t, w, lam, fs: float, f_w: float, freqs):
    return leakage(lam, leakage_denominator(t, w, fs, freqs), f_w)


def leakage_denominator_subband(t, w, f_min: float, f_max: float, dfreqs) -> np.ndarray:
    """D [K, len(dfreqs)] for a sub-band plan (Sec. 2.3 with App. B's estimate): the band of the
    analysis is B^q = {f_min <= |f| <= f_max} (R(B^q), Eq. gpss_matrix_b_q), the tapers w [K, N] are
    complex, and the shift is the offset from the nominal centre, dfreqs = f_ci - f_c0:
        D_k^i = (E_i w_k)^H R(B^q) (E_i w_k),   E_i = diag(exp(i 2 pi dfreqs_i t_n)).
    Formed densely, as leakage_denominator."""
    t = np.asarray(t, dtype=np.float64)
    tc = t - t.mean()
    w = np.atleast_2d(np.asarray(w, dtype=np.complex128))
    RB = gpss_matrix_b_sub(t, f_min, f_max)
    dfreqs = np.asarray(dfreqs, dtype=np.float64)
    D = np.empty((w.shape[0], dfreqs.shape[0]))
    for j, f in enumerate(dfreqs):
        e = np.exp(2j * np.pi * f * tc)
        V = w * e[None, :]
        RV = V @ RB
        D[:, j] = np.real(np.sum(np.conj(V) * RV, axis=1))
    return D


def leakage_subband_at(t, w, lam, f_w: float, f_min: float, f_max: float, dfreqs):
    """(L, Ehat) of a sub-band plan's tapers at the shifts dfreqs (w^H R(B^q) w = 2 f_w)."""
    return leakage(lam, leakage_denominator_subband(t, w, f_min, f_max, dfreqs), f_w)
