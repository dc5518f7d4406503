"""Oracle pin helper: discrete prolate spheroidal sequences on a uniform grid.

Test infrastructure only.  Used to pin the GEP of Eq. (gep_at_A0): on a full
unit-rate grid with f_max = 1/2, R(B) is the identity, the GEP becomes the
ordinary eigenproblem of the prolate matrix, and the nominal tapers are the
DPSS scaled to w^T w = 2 f_w (Sec. 4: uniform sampling gives identical
tapers; Sec. 3.7: the f_c0 = 0 case reduces to the DPSS).

The sequences are computed here by an independent route: the symmetric
tridiagonal matrix that commutes with the prolate matrix (Slepian 1978;
Percival & Walden 1993, Sec. 8.3), solved by LAPACK's tridiagonal
eigensolver.  Its entries are
    diag_n = ((N - 1 - 2n) / 2)^2 cos(2 pi W),   offdiag_n = n (N - n) / 2,
for n = 0..N-1 (offdiag for n = 1..N-1).  The concentration of each
sequence is its Rayleigh quotient with the prolate (sinc) matrix.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def dpss(N: int, W: float, K: int):
    """(v [K, N] unit-norm, concentration [K]) sorted by concentration."""
    n = np.arange(N, dtype=np.float64)
    diag = ((N - 1 - 2.0 * n) / 2.0) ** 2 * np.cos(2.0 * np.pi * W)
    off = n[1:] * (N - n[1:]) / 2.0
    vals, vecs = scipy.linalg.eigh_tridiagonal(diag, off, select="i",
                                               select_range=(N - K, N - 1))
    order = np.argsort(vals)[::-1]
    v = vecs[:, order].T
    d = n[:, None] - n[None, :]
    A = np.where(d == 0, 2.0 * W, np.sin(2.0 * np.pi * W * d) / (np.pi * np.where(d == 0, 1.0, d)))
    conc = np.einsum("kn,nm,km->k", v, A, v)
    return v, conc
