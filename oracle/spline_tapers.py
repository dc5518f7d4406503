"""Oracle: nominal tapers by interpolated DPSS (no GEP).

Test infrastructure only (imported by tests/, never by the product path).

Follows Table 1, step 3 (case f_c0 = 0), sub-steps (a)-(c), in the paper's
order, with the readings stated beside each:
  (a) DPSS of order k on a uniform grid of N nodes u_j = t_1 + j D spanning
      the sampling times.  Reading: D = (t_N - t_1) / (N - 1), so that the
      grid runs from t_1 to t_N (the table prints (t_N - t_1) / N); the DPSS
      half-bandwidth in cycles per grid step is W = f_w D.  The sequences are
      computed by the tridiagonal route of oracle/dpss.py (Percival & Walden
      1993, Sec. 8.3; the paper cites these fast algorithms);
  (b) the taper weights at the sampling times by cubic-spline interpolation
      of each sequence.  Reading: not-a-knot end conditions (the paper does
      not state them);
  (c) normalise each taper so that w^T R(B) w = 2 f_w (Eq. bg_norm_requirement).
The sign rule of the GEP tapers is applied, and the concentration used by the
leakage estimate is the Rayleigh quotient lambda_k = w^T R(A0) w / w^T R(B) w
(reading: the interpolated taper is not an eigenvector, so its eigenvalue is
taken as the concentration it attains).
"""
from __future__ import annotations

import numpy as np
import scipy.interpolate

from . import dpss as odpss
from . import gpss as ogpss


def grid(t: np.ndarray):
    """Uniform nodes u [N] and their spacing D for the sorted times t."""
    ts = np.sort(np.asarray(t, dtype=np.float64))
    N = ts.size
    D = (ts[-1] - ts[0]) / (N - 1)
    return ts[0] + D * np.arange(N), D


def spline_tapers(t: np.ndarray, fs: float, f_w: float, K: int, spacing_divisor=None):
    """(w [K, N] in the order of t, lambda [K]).  spacing_divisor overrides N - 1 in the grid
    interval (pins use it to show which reading the uniform-grid reduction fixes)."""
    t = np.asarray(t, dtype=np.float64)
    N = t.size
    ts = np.sort(t)
    div = (N - 1) if spacing_divisor is None else spacing_divisor
    D = (ts[-1] - ts[0]) / div
    u = ts[0] + D * np.arange(N)
    v, _ = odpss.dpss(N, f_w * D, K)                                        # (a)
    w = np.empty((K, N))
    for k in range(K):
        cs = scipy.interpolate.CubicSpline(u, v[k], bc_type="not-a-knot")  # (b)
        w[k] = cs(t)
    RB = ogpss.gpss_matrix_b(t, 0.5 * fs)
    q = np.einsum("kn,nm,km->k", w, RB, w)
    w *= np.sqrt(2.0 * f_w / q)[:, None]                                    # (c)
    w = ogpss.sign_convention(w, t)
    RA = ogpss.gpss_matrix_a(t, f_w)
    lam = np.einsum("kn,nm,km->k", w, RA, w) / np.einsum("kn,nm,km->k", w, RB, w)
    return w, lam
