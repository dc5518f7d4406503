"""Pins for the CPU oracle: each check ties an oracle function to something
other than itself (closed forms, an independent DPSS route, exact FFTs on
integer grids, identities the paper states, invariances, brute force).

No GPU is used here.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import dpss as odpss
from oracle import estimator as oest
from oracle import gpss as ogpss
from oracle import leakage as oleak
from oracle import _native

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "e1_sampling_schemes.json")


def e1_times(scheme: str, seed: int = 0) -> np.ndarray:
    """Sampling times of the paper's Sec. 4 schemes (parameters in the fixture)."""
    g = json.load(open(GOLDEN))
    s = g["schemes"][scheme]
    rng = np.random.Generator(np.random.PCG64(seed))
    n = np.arange(1, g["N"] + 1, dtype=np.float64)
    if scheme == "uniform":
        return n
    if scheme == "jitter":
        return np.sort(n + s["sigma"] * rng.standard_normal(n.shape[0]))
    if scheme == "missing":
        return synth.scaled_missing(s["n_grid"], s["n_drop"], s["rate"], seed)
    if scheme == "arithmetic":
        a = s["a"]
        N = g["N"]
        b = (N - 1 - a * (N - 1)) / ((N - 1) * (N - 2) / 2.0)
        return 1.0 + a * (n - 1) + b * (n - 1) * (n - 2) / 2.0
    raise KeyError(scheme)


def projector(w, RB):
    """R(B)-orthogonal projector onto span(w^T) (basis-independent)."""
    W = np.atleast_2d(w).T
    G = W.T @ RB @ W
    return W @ np.linalg.solve(G, W.T @ RB)


# ---------------------------------------------------------------------------
# GEP / tapers
# ---------------------------------------------------------------------------
def test_two_sample_closed_form():
    """Two samples: R(B) and R(A0) share the eigenvectors (1,1) and (1,-1);
    lambda = (2fw +- a)/(1 +- s), and w^T R(B) w = 2 fw fixes the scale."""
    d, fw = 0.7, 0.11
    t = np.array([3.0, 3.0 + d])
    s = np.sin(np.pi * d) / (np.pi * d)           # R(B) off-diagonal, f_max = 1/2
    a = np.sin(2 * np.pi * fw * d) / (np.pi * d)  # R(A0) off-diagonal
    lp, lm = (2 * fw + a) / (1 + s), (2 * fw - a) / (1 - s)
    w, lam = ogpss.nominal_tapers(t, 1.0, fw, 2)
    exp_lam = sorted([lp, lm], reverse=True)
    np.testing.assert_allclose(lam, exp_lam, rtol=1e-13)
    for k in range(2):
        sym = (lp >= lm) == (k == 0)
        v = np.array([1.0, 1.0]) if sym else np.array([-1.0, 1.0])
        q = v @ np.array([[1, s], [s, 1]]) @ v
        np.testing.assert_allclose(np.abs(w[k]), np.abs(v) * np.sqrt(2 * fw / q), rtol=1e-12)
        assert np.sign(w[k, 0] * w[k, 1]) == (1 if sym else -1)


@pytest.mark.parametrize("N,NW,K", [(64, 3.0, 4), (128, 4.0, 6), (200, 2.5, 4)])
def test_uniform_grid_is_scaled_dpss(N, NW, K):
    """Full unit grid: the GEP tapers equal sqrt(2 f_w) * DPSS and the
    eigenvalues equal the DPSS concentrations (independent tridiagonal route)."""
    fw = NW / N
    t = np.arange(N, dtype=np.float64)
    w, lam = ogpss.nominal_tapers(t, 1.0, fw, K)
    v, conc = odpss.dpss(N, fw, K)
    np.testing.assert_allclose(lam, conc, atol=1e-12)
    v = ogpss.sign_convention(v, t)
    np.testing.assert_allclose(w, np.sqrt(2 * fw) * v, atol=2e-6 * np.sqrt(2 * fw))
    I = np.eye(N)
    np.testing.assert_allclose(projector(w, I), projector(v, I), atol=1e-10)


@pytest.mark.parametrize("scheme", ["uniform", "jitter", "missing", "arithmetic"])
def test_gep_invariants_on_paper_schemes(scheme):
    """0 < lambda < 1 descending; w^T R(B) w' = 2 f_w delta; the GEP residual;
    the bias-bound identity (Sec. 3.5) and the variance factor (Eq.
    bound_factor_approx) hold for the paper's Sec. 4 sampling schemes."""
    g = json.load(open(GOLDEN))
    t = e1_times(scheme)
    fw, K = g["f_w"], g["K"]
    w, lam = ogpss.nominal_tapers(t, 1.0, fw, K)
    RB = ogpss.gpss_matrix_b(t, 0.5)
    RA = ogpss.gpss_matrix_a(t, fw)
    assert np.all(lam < 1) and np.all(lam > 0)
    assert np.all(np.diff(lam) <= 0)
    G = w @ RB @ w.T
    np.testing.assert_allclose(G, 2 * fw * np.eye(K), atol=1e-10)
    res = RA @ w.T - RB @ w.T * lam[None, :]
    assert np.linalg.norm(res) / (np.linalg.norm(RA) * np.linalg.norm(w)) < 1e-10
    bias_lhs = (2 * fw / K) * np.sum(1 - lam)
    bias_rhs = np.mean([w[k] @ (RB - RA) @ w[k] for k in range(K)])
    np.testing.assert_allclose(bias_lhs, bias_rhs, rtol=1e-10, atol=1e-12)
    V = np.sum(np.abs(w @ RB @ w.T) ** 2) / K**2
    np.testing.assert_allclose(V, (2 * fw) ** 2 / K, rtol=1e-9)


def test_gep_against_cholesky_route():
    """Brute force on a small jittered set: reduce with an explicit Cholesky
    factor and a standard symmetric eigensolver; same eigenvalues, same
    K-dimensional subspace."""
    t = synth.jittered(48, 0.4, 5)
    fw, K = 4.0 / 48, 5
    RB = ogpss.gpss_matrix_b(t, 0.5)
    RA = ogpss.gpss_matrix_a(t, fw)
    L = np.linalg.cholesky(RB)
    Li = np.linalg.inv(L)
    vals, Y = np.linalg.eigh(Li @ RA @ Li.T)
    W2 = (Li.T @ Y[:, ::-1][:, :K]).T
    w, lam = ogpss.nominal_tapers(t, 1.0, fw, K)
    np.testing.assert_allclose(lam, vals[::-1][:K], atol=1e-13)
    np.testing.assert_allclose(projector(w, RB), projector(W2, RB), atol=1e-9)


def test_trace_identity_integer_grid():
    """Integer times with f_max = 1/2 give R(B) = I, so the generalized
    eigenvalues are those of R(A0) and sum to tr R(A0) = 2 f_w N."""
    t = synth.grid_bernoulli(80, 0.25, 3)
    fw = 3.0 / 80
    lam = ogpss.all_generalized_eigenvalues(t, 1.0, fw)
    np.testing.assert_allclose(lam.sum(), 2 * fw * t.shape[0], rtol=1e-12)
    RB = ogpss.gpss_matrix_b(t, 0.5)
    np.testing.assert_allclose(RB, np.eye(t.shape[0]), atol=1e-15)


def test_translation_invariance_of_tapers():
    t = synth.jittered(60, 0.3, 9)
    w0, l0 = ogpss.nominal_tapers(t, 1.0, 0.06, 4)
    w1, l1 = ogpss.nominal_tapers(t + 1234.0, 1.0, 0.06, 4)
    np.testing.assert_allclose(l0, l1, atol=1e-12)
    RB = ogpss.gpss_matrix_b(t, 0.5)
    np.testing.assert_allclose(projector(w0, RB), projector(w1, RB), atol=1e-8)


# ---------------------------------------------------------------------------
# eigencoefficients / P-hat
# ---------------------------------------------------------------------------
def test_nudft_brute_force_complex():
    """The C direct sum equals a dense numpy exponential matrix product
    for complex strengths, an arbitrary band grid and a band subset."""
    rng = np.random.default_rng(0)
    t = np.sort(rng.uniform(-5, 20, 37))
    c = rng.standard_normal((3, 37)) + 1j * rng.standard_normal((3, 37))
    f_lo, df = -0.31, 0.0173
    idx = np.array([0, 5, 17, 63, 100], dtype=np.int64)
    f = f_lo + idx * df
    ref = c @ np.exp(-2j * np.pi * np.outer(t, f))
    got = _native.nudft(t, c, f_lo, df, idx)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_integer_grid_equals_fft():
    """t_n integers, distinct mod I, f_i = -1/2 + i/I: J_k is the length-I FFT
    of c_k (-1)^t_n placed at t_n mod I (numpy pocketfft, FP64)."""
    wl = synth.workload("grid1024")
    t, x = wl.t, wl.x[0]
    w, lam = ogpss.nominal_tapers(t, wl.fs, wl.f_w, wl.K)
    J = oest.eigencoefficients(t, x, w, wl.f_lo, wl.df, wl.I)
    I = wl.I
    y = np.zeros((wl.K, I))
    ti = t.astype(np.int64)
    y[:, ti % I] = w * x[None, :] * np.where(ti % 2 == 0, 1.0, -1.0)[None, :]
    ref = np.fft.fft(y, axis=1)
    err = np.linalg.norm(J - ref) / np.linalg.norm(ref)
    assert err < 1e-13
    # discrete Parseval: (1/I) sum_i |J_k|^2 = sum_n |c_k[n]|^2
    np.testing.assert_allclose(np.sum(np.abs(J) ** 2, axis=1) / I,
                               np.sum((w * x[None, :]) ** 2, axis=1), rtol=1e-12)


def test_time_shift_exact_phase_large_t():
    """t -> t + t0 with a large integer t0 and dyadic band centres: P-hat is
    unchanged and J picks up exp(-i 2 pi f_i t0), whose phase is computed
    exactly in integers.  Exercises the oracle's exact phase reduction."""
    # times on a 2^-10 lattice so that t + t0 stays exactly representable
    t = np.round(synth.jittered(200, 0.4, 2) * 1024.0) / 1024.0
    rng = np.random.default_rng(4)
    x = rng.standard_normal(200)
    w, _ = ogpss.nominal_tapers(t, 1.0, 4.0 / 200, 4)
    I = 1 << 12
    f_lo, df = -0.5, 1.0 / I
    t0 = 987654321
    J0 = oest.eigencoefficients(t, x, w, f_lo, df, I)
    J1 = oest.eigencoefficients(t + t0, x, w, f_lo, df, I)
    # f_i t0 = (i - I/2) t0 / I  (exact integer arithmetic modulo I)
    m = (np.arange(I, dtype=np.int64) - I // 2)
    cyc = ((m * (t0 % I)) % I).astype(np.float64) / I
    ref = J0 * np.exp(-2j * np.pi * cyc)[None, :]
    assert np.linalg.norm(J1 - ref) / np.linalg.norm(ref) < 1e-12
    np.testing.assert_allclose(oest.psd(J1), oest.psd(J0), rtol=1e-10)


def test_psd_invariant_under_taper_rotation():
    """P-hat depends only on span(w): w -> Q w (Q orthogonal K x K) leaves it
    unchanged (Eq. power_spectrum_estimator is a sum of squares)."""
    t = synth.jittered(120, 0.4, 6)
    x = np.random.default_rng(1).standard_normal(120)
    w, _ = ogpss.nominal_tapers(t, 1.0, 5.0 / 120, 6)
    Q, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((6, 6)))
    P0 = oest.psd(oest.eigencoefficients(t, x, w, -0.5, 1 / 256, 256))
    P1 = oest.psd(oest.eigencoefficients(t, x, Q @ w, -0.5, 1 / 256, 256))
    np.testing.assert_allclose(P1, P0, rtol=1e-10, atol=1e-14)


def test_white_noise_expected_psd_is_flat():
    """For i.i.d. x with variance s2, E[|J_k(f)|^2] = s2 sum_n w_k(t_n)^2 at
    every f (Sec. 3.3).  Checked exactly via linearity (sum over the unit
    basis) and statistically by Monte Carlo."""
    t = e1_times("jitter")
    w, _ = ogpss.nominal_tapers(t, 1.0, 0.05, 4)
    I = 64
    N = t.shape[0]
    basis = np.eye(N)
    acc = np.zeros((4, I))
    for n in range(N):
        acc += np.abs(oest.eigencoefficients(t, basis[n], w, -0.5, 1 / I, I)) ** 2
    np.testing.assert_allclose(acc, np.sum(w**2, axis=1)[:, None] * np.ones((1, I)), rtol=1e-11)
    expected = np.mean(np.sum(w**2, axis=1))            # (1/K) sum_k ||w_k||^2, s2 = 1
    M = 400
    rng = np.random.default_rng(11)
    P = np.zeros(I)
    for _ in range(M):
        P += oest.psd(oest.eigencoefficients(t, rng.standard_normal(N), w, -0.5, 1 / I, I))
    P /= M
    # each bin's mean of M draws: relative SE about 1/sqrt(M K) (chi-square-like)
    assert abs(P.mean() / expected - 1) < 3.0 / np.sqrt(M * 4 * 8)
    assert np.all(np.abs(P / expected - 1) < 6.0 / np.sqrt(M * 4) + 0.05)


# ---------------------------------------------------------------------------
# leakage estimate (App. B)
# ---------------------------------------------------------------------------
def test_leakage_zero_on_integer_grid():
    """Missing data on the unit grid (f_max = 1/2): R(B) = I so lambda-hat =
    lambda and L-hat = 0 at every band (App. B)."""
    t = synth.grid_bernoulli(90, 0.2, 8)
    w, lam = ogpss.nominal_tapers(t, 1.0, 4.0 / 90, 5)
    f = np.linspace(-0.5, 0.5, 23, endpoint=False)
    L, E = oleak.leakage_at(t, w, lam, 1.0, 4.0 / 90, f)
    assert np.max(L) < 1e-12 and np.max(E) < 1e-12


def test_leakage_zero_at_nominal_band():
    """At f = 0, D = w^T R(B) w = 2 f_w by normalisation, so L-hat = 0."""
    t = e1_times("jitter")
    w, lam = ogpss.nominal_tapers(t, 1.0, 0.05, 4)
    L, E = oleak.leakage_at(t, w, lam, 1.0, 0.05, [0.0])
    assert np.max(L) < 1e-12


def test_leakage_denominator_by_spectral_integral():
    """Independent route: D_k(f) = integral over [f - f_max, f + f_max] of
    |W_k(phi)|^2 with W_k(phi) = sum_n w_k(t_n) exp(-i 2 pi phi t_n), by
    Gauss-Legendre quadrature (R(B) is the integral of exp(i 2 pi nu dt)
    over the signal band, Eq. gpss_matrix_b)."""
    t = e1_times("arithmetic")
    w, lam = ogpss.nominal_tapers(t, 1.0, 0.05, 4)
    freqs = np.array([-0.37, -0.1, 0.05, 0.21, 0.44])
    D = oleak.leakage_denominator(t, w, 1.0, freqs)
    x, wt = np.polynomial.legendre.leggauss(600)
    tc = t - t.mean()
    for j, f in enumerate(freqs):
        phi = f + 0.5 * x
        Wp = w @ np.exp(-2j * np.pi * np.outer(tc, phi))
        ref = 0.5 * np.sum(np.abs(Wp) ** 2 * wt[None, :], axis=1)
        np.testing.assert_allclose(D[:, j], ref, rtol=1e-11)


def test_theorem1_bounds_rate_mismatch():
    """Theorem 1 (App. B): missing-data sampling at actual rate 1.2 Hz with
    a nominal 1 Hz: 0 <= L-hat <= lambda (1 + f_w / (||w||^2 - f_w)) whenever
    f_w < ||w||^2 <= 2 f_w; and L-hat is not identically zero."""
    t = e1_times("missing")
    fw = 0.05
    w, lam = ogpss.nominal_tapers(t, 1.0, fw, 4)
    f = np.linspace(-0.5, 0.5, 41, endpoint=False)
    L, E = oleak.leakage_at(t, w, lam, 1.0, fw, f)
    nrm = np.sum(w**2, axis=1)
    assert np.all(L >= 0)
    assert np.max(L) > 1e-6
    ok = (nrm > fw) & (nrm <= 2 * fw)
    bound = lam * (1 + fw / (nrm - fw))
    for k in np.nonzero(ok)[0]:
        assert np.all(L[k] <= bound[k] + 1e-12)


def test_nudft_threads_agree():
    """The OpenMP split does not change any result bit."""
    t = synth.jittered(300, 0.4, 1)
    c = np.random.default_rng(3).standard_normal((2, 300))
    idx = np.arange(500, dtype=np.int64)
    a = _native.nudft(t, c, -0.5, 1 / 500, idx, nthreads=1)
    b = _native.nudft(t, c, -0.5, 1 / 500, idx, nthreads=4)
    assert np.array_equal(a, b)


def test_lambda_hat_is_rayleigh_quotient_of_shifted_taper():
    """App. B: lambda-hat is the generalized Rayleigh quotient of the shifted
    taper E_i w with the analysis-band matrix R(A_i) centred at f_i (Eq.
    gpss_matrix_a with f_c = f_i).  Built here from the complex matrix
    directly, not from the shift identity the oracle uses."""
    t = e1_times("missing")
    fw = 0.05
    w, lam = ogpss.nominal_tapers(t, 1.0, fw, 4)
    RB = ogpss.gpss_matrix_b(t, 0.5)
    freqs = [-0.41, -0.2, 0.13, 0.37]
    L, _ = oleak.leakage_at(t, w, lam, 1.0, fw, freqs)
    for j, f in enumerate(freqs):
        RAi = ogpss.gpss_matrix_a(t, fw, f_c=f)
        for k in range(4):
            v = w[k] * np.exp(2j * np.pi * f * t)
            lam_hat = np.real(np.conj(v) @ RAi @ v) / np.real(np.conj(v) @ RB @ v)
            np.testing.assert_allclose(L[k, j], abs(lam[k] - lam_hat), rtol=1e-9, atol=1e-13)


def test_gpss_rows_match_full_matrix():
    t = synth.jittered(70, 0.4, 12)
    rows = np.array([0, 5, 33, 69])
    np.testing.assert_array_equal(ogpss.gpss_rows(t, rows, 0.5), ogpss.gpss_matrix_b(t, 0.5)[rows])
    np.testing.assert_array_equal(ogpss.gpss_rows(t, rows, 0.07), ogpss.gpss_matrix_a(t, 0.07)[rows])
