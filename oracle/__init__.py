"""CPU oracle for the M2NuFFT hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 implementations of what the GPU path computes, written
from the paper (Cui, Brinkmann & Worrell, "Multiband-Multitaper NuFFT",
arXiv 2407.01943):

  gpss.py       R(B), R(A0) (Eqs. gpss_matrix_b, gpss_matrix_a), the nominal-band
                GEP (Eq. gep_at_A0) by LAPACK, normalisation (Eq. bg_norm_requirement)
  estimator.py  eigencoefficients by the direct sum (Eq. eigencoefficients, Table 1
                step 4), eigenspectra, P-hat (Eq. power_spectrum_estimator, step 5)
  leakage.py    lambda-hat, L-hat and E-hat (App. B, Eq. lambda_hat_ki)
  dpss.py       uniform-grid DPSS by the tridiagonal route (pin helper only)
  nudft.c       the direct NUDFT in plain C with exact phase reduction

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
leg may import this package.  The GPU product path never calls it, and it
shares no code with the CUDA sources.

Pins (tests/test_oracle_pins.py) tie each function to something other than
itself: DPSS on full uniform grids, closed forms for two samples, the trace
identity on integer grids, the bias-bound and variance-factor identities of
Sec. 3.3-3.5, exact FFTs on integer grids, Parseval, time-shift and
taper-rotation invariance, white-noise flatness, L-hat = 0 on integer grids
and at f = 0, and Theorem 1's bounds.
"""
from . import estimator, gpss, leakage  # noqa: F401
from ._native import build, nudft, num_threads  # noqa: F401
