"""Pins of the oracle's F-statistic (Sec. 3 periodicity test, Eq. f_stat).

Each check is fixed by the mathematics, not by retyping the formula:
  * null distribution: with white Gaussian noise and tapers that are
    orthogonal with equal norms (uniform grid: R(B) = I, so the R(B)
    normalisation makes w_k^T w_l = 2 f_w delta_kl), the eigencoefficients of
    a band away from 0 and 1/2 are independent circular complex Gaussians of
    equal variance, so F_i follows F(2, 2K - 2) exactly (a regression of J on
    one complex regressor W: 2 real degrees of freedom in the fit, 2K - 2 in
    the residual).  A wrong dof factor, a dropped sum of W^2 or a residual
    taken from the wrong amplitude shifts the distribution and fails the
    Kolmogorov-Smirnov check;
  * line amplitude: for a complex line A e^{i(2 pi f0 t + phi)} the
    eigencoefficients at f0 are A e^{i phi} W_k^0(0) exactly, so the amplitude
    estimate is A e^{i phi} on any sampling pattern (GPSS tapers, missing
    samples); for a real cosine on the full grid it is (A/2) e^{i phi} up to
    the DPSS spectrum at 2 f0;
  * invariances: F does not change when x is scaled or a taper flips sign.
"""
import numpy as np
import pytest

import synth
from oracle import dpss as odpss
from oracle import estimator as oest
from oracle import ftest as oft
from oracle import gpss as ogpss

scipy_stats = pytest.importorskip("scipy.stats")


def _null_sample(K, n_signals=40, N=2048, NW=4, seed=5):
    fw = NW / N
    v, _ = odpss.dpss(N, fw, K)
    w = v * np.sqrt(2 * fw)
    t = np.arange(N, dtype=np.float64)
    # bands on the Rayleigh grid, 16 bins apart (twice the 2 f_w = 8-bin bandwidth), away from 0 and 1/2
    idx = np.arange(40, N // 2 - 40, 16, dtype=np.int64)
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_signals):
        x = rng.standard_normal(N)
        J = oest.eigencoefficients(t, x, w, 0.0, 1.0 / N, N, idx)
        out.append(oft.f_statistic(J, w))
    return np.concatenate(out)


@pytest.mark.parametrize("K", [4, 6])
def test_ftest_null_distribution_is_F_2_2Km2(K):
    F = _null_sample(K)
    assert F.size > 2000
    ks = scipy_stats.kstest(F, scipy_stats.f(2, 2 * K - 2).cdf)
    assert ks.pvalue > 1e-3, ks
    # the same sample is far from the distributions a wrong dof count would give
    for d2 in (2 * K, 2 * K - 4):
        assert scipy_stats.kstest(F, scipy_stats.f(2, d2).cdf).pvalue < ks.pvalue
    # planted mistakes in the statistic: K in place of K - 1, or the factor dropped
    assert scipy_stats.kstest(F * K / (K - 1), scipy_stats.f(2, 2 * K - 2).cdf).pvalue < 1e-6
    assert scipy_stats.kstest(F / (K - 1), scipy_stats.f(2, 2 * K - 2).cdf).pvalue < 1e-6
    # and its mean matches (2K - 2) / (2K - 4)
    m = (2 * K - 2) / (2 * K - 4)
    assert abs(F.mean() - m) < 6 * m * np.sqrt(2.0 / F.size) * 2


def test_ftest_line_amplitude_nonuniform():
    """A complex line A e^{i(2 pi f0 t + phi)} sampled on a nonuniform pattern:
    J_k(f0) = A e^{i phi} W_k^0(0) for every taper, so the amplitude estimate is
    exactly A e^{i phi} and the residual vanishes (F unbounded)."""
    N, K = 2048, 6
    fw = 4.0 / N
    t = synth.grid_bernoulli(N, 0.2, 3)
    w, _ = ogpss.nominal_tapers(t, 1.0, fw, K)
    A, phi, f0 = 2.5, 0.7, 421.0 / N
    x = A * np.exp(1j * (2 * np.pi * f0 * t + phi))
    idx = np.array([421, 421 + 40], dtype=np.int64)
    J = oest.eigencoefficients(t, x, w, 0.0, 1.0 / N, N, idx)
    C = oft.line_amplitude(J, oft.taper_dc(w))
    assert abs(C[0] - A * np.exp(1j * phi)) < 1e-10 * A
    F = oft.f_statistic(J, w)
    crit = scipy_stats.f(2, 2 * K - 2).ppf(1 - 1.0 / N)  # p-value at the Rayleigh frequency 1/N
    assert F[0] > 1e12 * crit
    # with noise added, the line stays detected and an empty band 40 bins away does not
    rng = np.random.default_rng(1)
    xn = x + rng.standard_normal(t.size)
    Jn = oest.eigencoefficients(t, xn, w, 0.0, 1.0 / N, N, idx)
    Fn = oft.f_statistic(Jn, w)
    assert Fn[0] > crit and Fn[1] < crit


def test_ftest_line_amplitude_real_cosine_uniform():
    """A real cosine on the full grid with DPSS tapers: the amplitude estimate at f0
    is (A/2) e^{i phi} up to the taper spectrum at 2 f0, far outside the band."""
    N, K, NW = 2048, 6, 4
    fw = NW / N
    v, _ = odpss.dpss(N, fw, K)
    w = v * np.sqrt(2 * fw)
    t = np.arange(N, dtype=np.float64)
    A, phi, f0 = 2.5, 0.7, 421.0 / N
    x = A * np.cos(2 * np.pi * f0 * t + phi)
    J = oest.eigencoefficients(t, x, w, 0.0, 1.0 / N, N, np.array([421], dtype=np.int64))
    C = oft.line_amplitude(J, oft.taper_dc(w))
    assert abs(C[0] - 0.5 * A * np.exp(1j * phi)) < 1e-6 * A


def test_ftest_invariances():
    N, K = 600, 5
    t = synth.jittered(N, 0.4, 2)
    w, _ = ogpss.nominal_tapers(t, 1.0, 3.0 / N, K)
    x = synth.white(t, 1.0, 4)
    idx = np.arange(10, 300, 7, dtype=np.int64)
    J = oest.eigencoefficients(t, x, w, -0.5, 1.0 / N, N, idx)
    F = oft.f_statistic(J, w)
    J2 = oest.eigencoefficients(t, -3.5 * x, w, -0.5, 1.0 / N, N, idx)
    np.testing.assert_allclose(oft.f_statistic(J2, w), F, rtol=1e-10)
    s = np.array([1, -1, 1, -1, -1])[:, None]
    J3 = oest.eigencoefficients(t, x, w * s, -0.5, 1.0 / N, N, idx)
    np.testing.assert_allclose(oft.f_statistic(J3, w * s), F, rtol=1e-10)
