"""Pins of the sub-band oracle (Sec. 2.3 Eq. gpss_matrix_b_q; Sec. 3 multiband partition;
Eq. gep_at_A0 with f_c0 != 0).

  * partition: the sub-band matrices of a partition of the signal band add up to R(B) exactly
    (the integrals over disjoint pieces of |f| <= f_max add up);
  * definition: R(B^q | n, m) equals the integral of e^{i 2 pi f (t_n - t_m)} over
    f_min <= |f| <= f_max, evaluated by numerical quadrature;
  * shift theorem: on the full unit grid (R(B) = I), R(A0) at centre f_c0 is D R(A0 at 0) D^H with
    D = diag(e^{i 2 pi f_c0 t_n}), so the sub-band tapers are the DPSS modulated to f_c0 (with the
    same eigenvalues) -- catches a conjugated or missing modulation;
  * reduction: f_c0 = 0, f_min = 0, f_max = fs/2 gives the full-band (real) tapers;
  * the Hermitian GEP's invariants: w^H R(B^q) w = 2 f_w, R(B^q)-orthogonality, 0 < lambda < 1;
  * leakage estimate of sub-band tapers (App. B with R(B^q)): D equals the integral of the shifted
    taper spectrum |W(f - df)|^2 over f_min <= |f| <= f_max (quadrature; catches a conjugated phase
    or a dropped half of the band), it reduces to the full-band estimate for f_min = 0,
    f_max = fs/2 and real tapers, and it vanishes at the nominal centre (D = w^H R(B^q) w = 2 f_w).
"""
import numpy as np
import pytest

import synth
from oracle import dpss as odpss
from oracle import estimator as oest
from oracle import gpss as ogpss
from oracle import leakage as oleak

integrate = pytest.importorskip("scipy.integrate")


def test_partition_adds_up_to_full_band():
    t = synth.jittered(200, 0.4, 1)
    edges = [0.0, 0.11, 0.27, 0.5]
    R = sum(ogpss.gpss_matrix_b_sub(t, a, b) for a, b in zip(edges[:-1], edges[1:]))
    np.testing.assert_allclose(R, ogpss.gpss_matrix_b(t, 0.5), atol=1e-14)


def test_subband_matrix_matches_its_integral():
    t = synth.jittered(40, 0.4, 2)
    f_min, f_max = 0.13, 0.31
    R = ogpss.gpss_matrix_b_sub(t, f_min, f_max)
    for n, m in [(0, 0), (3, 7), (10, 2), (25, 39)]:
        d = t[n] - t[m]
        re = integrate.quad(lambda f: np.cos(2 * np.pi * f * d), f_min, f_max, epsabs=1e-14, epsrel=1e-13)[0]
        # the band is symmetric in f, so the imaginary parts cancel and both sides contribute re
        assert abs(R[n, m] - 2 * re) < 1e-12


def test_shift_theorem_on_uniform_grid():
    N, K, NW = 256, 4, 3.0
    fw, f_c0 = NW / N, 0.2
    t = np.arange(N, dtype=np.float64)
    w, lam = ogpss.subband_tapers(t, fw, K, f_c0, 0.0, 0.5)
    v, conc = odpss.dpss(N, fw, K)
    ref = ogpss.phase_convention((v * np.sqrt(2 * fw)) * np.exp(2j * np.pi * f_c0 * t)[None, :], t, f_c0)
    np.testing.assert_allclose(lam, conc, atol=1e-12)
    np.testing.assert_allclose(w, ref, atol=1e-7 * np.abs(ref).max())
    # the conjugate modulation is not a solution
    bad = ogpss.phase_convention((v * np.sqrt(2 * fw)) * np.exp(-2j * np.pi * f_c0 * t)[None, :], t, f_c0)
    assert np.max(np.abs(w - bad)) > 0.1 * np.abs(ref).max()


def test_full_band_reduction():
    t = synth.jittered(300, 0.4, 5)
    w, lam = ogpss.subband_tapers(t, 3.0 / 300, 4, 0.0, 0.0, 0.5)
    wr, lr = ogpss.nominal_tapers(t, 1.0, 3.0 / 300, 4)
    np.testing.assert_allclose(lam, lr, atol=1e-12)
    np.testing.assert_allclose(w, wr, atol=1e-8 * np.abs(wr).max())


def test_hermitian_gep_invariants():
    t = synth.grid_bernoulli(400, 0.2, 6)
    fw, f_c0, f_min, f_max = 4.0 / 400, 0.3, 0.2, 0.4
    w, lam = ogpss.subband_tapers(t, fw, 5, f_c0, f_min, f_max)
    RB = ogpss.gpss_matrix_b_sub(t, f_min, f_max)
    G = np.conj(w) @ RB @ w.T
    np.testing.assert_allclose(G, 2 * fw * np.eye(5), atol=1e-10)
    assert np.all((lam > 0) & (lam < 1)) and np.all(np.diff(lam) <= 0)
    RA = ogpss.gpss_matrix_a(t, fw, f_c0)
    res = RA @ w.T - (RB @ w.T) * lam[None, :]
    # exact on the kept range of R(B^q); the discarded directions (eigenvalues <= tau * max) leave a
    # residual of order sqrt(tau * max(eig R(B^q)) * 2 f_w)
    tau = ogpss.RANGE_TOL
    assert np.max(np.abs(res)) < np.sqrt(tau * 2 * (f_max - f_min) * 2 * fw)


def test_shifted_eigencoefficient_of_a_line_at_the_nominal_centre():
    """x = e^{i 2 pi f_c0 t}: J_k(A_0) = sum conj(w_k) x = conj(sum w_k e^{-i 2 pi f_c0 t}), which the
    phase rule makes real and positive for the even-order tapers."""
    t = synth.jittered(300, 0.4, 8)
    f_c0 = 0.17
    w, _ = ogpss.subband_tapers(t, 3.0 / 300, 3, f_c0, 0.1, 0.25)
    x = np.exp(2j * np.pi * f_c0 * t)
    J = oest.eigencoefficients(t, x, w, 0.0, 1.0, 1)  # delta f = 0 only
    assert J[0, 0].real > 0 and abs(J[0, 0].imag) < 1e-12 * abs(J[0, 0])


def test_subband_leakage_denominator_is_the_band_integral():
    t = synth.jittered(60, 0.4, 9)
    rng = np.random.default_rng(4)
    w = rng.standard_normal((2, 60)) + 1j * rng.standard_normal((2, 60))
    f_min, f_max = 0.12, 0.33
    dfs = np.array([-0.07, 0.0, 0.045])
    D = oleak.leakage_denominator_subband(t, w, f_min, f_max, dfs)
    tc = t - t.mean()
    xg, wg = np.polynomial.legendre.leggauss(400)
    for j, df in enumerate(dfs):
        for k in range(2):
            def spec(f):  # |W(f - df)|^2, W(f) = sum_n w_n e^{-i 2 pi f t_n}
                return np.abs(np.exp(-2j * np.pi * np.outer(f - df, tc)) @ w[k]) ** 2
            total = 0.0
            for a, b in ((f_min, f_max), (-f_max, -f_min)):
                # split each interval so 400 nodes resolve the oscillations (span ~60)
                for a2, b2 in zip(np.linspace(a, b, 9)[:-1], np.linspace(a, b, 9)[1:]):
                    f = 0.5 * (b2 - a2) * xg + 0.5 * (b2 + a2)
                    total += 0.5 * (b2 - a2) * np.sum(wg * spec(f))
            assert abs(D[k, j] - total) < 1e-10 * abs(total)


def test_subband_leakage_reduces_to_full_band():
    t = synth.jittered(120, 0.4, 10)
    w, lam = ogpss.nominal_tapers(t, 1.0, 3.0 / 120, 3)
    fr = np.linspace(-0.5, 0.5, 17)
    a = oleak.leakage_denominator_subband(t, w.astype(np.complex128), 0.0, 0.5, fr)
    b = oleak.leakage_denominator(t, w, 1.0, fr)
    np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)


def test_subband_leakage_vanishes_at_the_nominal_centre():
    t = synth.grid_bernoulli(300, 0.2, 11)
    fw, f_c0, f_min, f_max = 4.0 / 300, 0.3, 0.2, 0.4
    w, lam = ogpss.subband_tapers(t, fw, 4, f_c0, f_min, f_max)
    L, E = oleak.leakage_subband_at(t, w, lam, fw, f_min, f_max, np.array([0.0, 0.01]))
    assert np.max(L[:, 0]) < 1e-10 and E[0] < 1e-10
    assert np.max(L[:, 1]) > 1e-6  # a shift off the nominal centre leaks
