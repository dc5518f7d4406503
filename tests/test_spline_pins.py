"""Pins of the interpolated-DPSS tapers (Table 1, step 3 a-c) computed by the oracle.

  * uniform grid t_n = n: the spline nodes are the sampling times, so the
    tapers are sqrt(2 f_w) x DPSS, which the GEP route also gives there
    (Sec. 4: uniform sampling reduces the GPSS to the DPSS); the printed grid
    interval (t_N - t_1) / N moves the nodes off the samples and breaks this
    reduction (planted variant);
  * time-scale invariance: t -> c t with f_w -> f_w / c and fs -> fs / c
    leaves the tapers unchanged (catches a half-bandwidth not converted to
    cycles per grid step);
  * Courant-Fischer: the leading GEP taper maximises the concentration
    w^T R(A0) w / w^T R(B) w, so the interpolated leading taper's
    concentration cannot exceed the leading GEP eigenvalue (on jittered or
    gapped patterns it is clearly below it: R(B) is far from the identity
    there, and the GEP tapers exploit that, the interpolated DPSS do not);
  * normalisation: w^T R(B) w = 2 f_w for every taper (Eq. bg_norm_requirement).
"""
import numpy as np
import pytest

import synth
from oracle import dpss as odpss
from oracle import gpss as ogpss
from oracle import spline_tapers as ost


def test_uniform_grid_reduces_to_dpss_and_gep():
    N, K, NW = 512, 5, 3.5
    fw = NW / N
    t = np.arange(N, dtype=np.float64)
    w, lam = ost.spline_tapers(t, 1.0, fw, K)
    v, conc = odpss.dpss(N, fw, K)
    dp = ogpss.sign_convention(v * np.sqrt(2 * fw), t)
    np.testing.assert_allclose(w, dp, atol=1e-12 * np.abs(dp).max())
    np.testing.assert_allclose(lam, conc, rtol=1e-12)
    wg, lg = ogpss.nominal_tapers(t, 1.0, fw, K)
    np.testing.assert_allclose(w, wg, atol=1e-7 * np.abs(wg).max())
    np.testing.assert_allclose(lam, lg, atol=1e-12)
    # the printed interval (t_N - t_1) / N puts the nodes between the samples
    wn, _ = ost.spline_tapers(t, 1.0, fw, K, spacing_divisor=N)
    assert np.max(np.abs(wn - dp)) > 1e-6 * np.abs(dp).max()


def test_time_scale_invariance():
    N, K = 400, 4
    t = synth.jittered(N, 0.4, 3)
    w1, l1 = ost.spline_tapers(t, 1.0, 3.0 / N, K)
    c = 2.5
    w2, l2 = ost.spline_tapers(c * t, 1.0 / c, 3.0 / N / c, K)
    # R(B) and 2 f_w both scale by 1/c, and W = f_w D is unchanged, so the tapers are the same
    np.testing.assert_allclose(w2, w1, rtol=1e-9, atol=1e-12 * np.abs(w1).max())
    np.testing.assert_allclose(l2, l1, rtol=1e-10)


@pytest.mark.parametrize("kind", ["jitter", "bernoulli"])
def test_concentration_bounded_by_gep(kind):
    N, K = 600, 6
    fw = 4.0 / N
    t = synth.jittered(N, 0.4, 9) if kind == "jitter" else synth.grid_bernoulli(N, 0.15, 9)
    w, lam = ost.spline_tapers(t, 1.0, fw, K)
    _, lg = ogpss.nominal_tapers(t, 1.0, fw, K)
    assert lam[0] <= lg[0] + 1e-13
    assert np.all((lam > 0) & (lam < 1))


def test_normalisation():
    N, K = 500, 5
    t = synth.jittered(N, 0.3, 4)
    fw = 3.0 / N
    w, _ = ost.spline_tapers(t, 1.0, fw, K)
    RB = ogpss.gpss_matrix_b(t, 0.5)
    np.testing.assert_allclose(np.einsum("kn,nm,km->k", w, RB, w), 2 * fw, rtol=1e-12)
