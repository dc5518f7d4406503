"""Pins of the true suboptimality oracle (Sec. 3, Eq. subopt_measure, per-band GEPs).

  * integer grid: R(B) = I and R(A_i) = E_i R(A0) E_i^* with E_i unitary, so every band has the
    nominal eigenvalues and E_i = 0 (Sec. 3.7's statement for uniform sampling);
  * the nominal band itself (f_ci = f_c0 = 0): lambda^i = lambda^0, E = 0;
  * Courant-Fischer per band: the optimal leading eigenvalue at A_i is at least the
    concentration the shifted nominal taper attains there, lambda_0^i >= lambda_hat_0^i
    (the leakage oracle's Rayleigh quotient, App. B), and both lie in (0, 1);
  * (all bands inside the signal band, |f_ci| + f_w <= f_max, as the method requires;
    a band reaching past f_max can have lambda > 1)
  * conjugate symmetry: for real sampling times the bands at f and -f have equal eigenvalues
    (R(A at -f) is the complex conjugate of R(A at f), R(B) is real).
"""
import numpy as np

import synth
from oracle import gpss as ogpss
from oracle import leakage as oleak
from oracle import true_subopt as ots


def test_integer_grid_has_zero_suboptimality():
    t = synth.grid_bernoulli(48, 0.2, 3)
    fw, K = 3.0 / 48, 3
    _, lam0 = ogpss.nominal_tapers(t, 1.0, fw, K)
    freqs = np.linspace(-0.43, 0.43, 13)
    lb = ots.band_eigenvalues(t, 1.0, fw, K, freqs)
    np.testing.assert_allclose(ots.true_suboptimality(lam0, lb), 0.0, atol=1e-12)


def test_nominal_band_and_bounds_on_jittered_times():
    t = synth.jittered(40, 0.4, 5)
    fw, K = 3.0 / 40, 3
    w, lam0 = ogpss.nominal_tapers(t, 1.0, fw, K)
    freqs = np.array([0.0, 0.05, 0.17, 0.31, 0.42])  # analysis bands inside |f| <= 1/2
    lb = ots.band_eigenvalues(t, 1.0, fw, K, freqs)
    E = ots.true_suboptimality(lam0, lb)
    assert abs(E[0]) < 1e-12
    assert np.all((lb > 0) & (lb < 1))
    L, _ = oleak.leakage_at(t, w, lam0, 1.0, fw, freqs)
    lam_hat0 = lam0[0] * 2 * fw / oleak.leakage_denominator(t, w, 1.0, freqs)[0]
    assert np.all(lb[:, 0] >= lam_hat0 - 1e-12)
    assert np.any(E[1:] > 1e-6)  # jittered times: the shifted tapers are not optimal everywhere


def test_conjugate_band_symmetry():
    t = synth.jittered(36, 0.3, 9)
    fw, K = 2.0 / 36, 2
    f = np.array([0.12, 0.27])
    np.testing.assert_allclose(ots.band_eigenvalues(t, 1.0, fw, K, f), ots.band_eigenvalues(t, 1.0, fw, K, -f),
                               atol=1e-12)
