"""The element-wise parity check itself (CPU): it accepts what a correct FP32 result looks like and
rejects a wrong value at a single band that the relative l2 norm over the array lets through.

The mistakes are planted in the oracle's own output, on the CPU."""
import numpy as np

import synth
from oracle import estimator as oest
from oracle import gpss as ogpss
from tests._util import TOL, elementwise_errors, packed_edge_bands, rel_l2, sample_bands, source_l1


def _case():
    # an AR(4) spectrum (poles 0.95 e^{+-i 0.1 pi}, 0.95 e^{+-i 0.3 pi}) on a jittered pattern:
    # tens of dB between the peaks and the band edges
    N, K, I = 2048, 4, 1 << 14
    t = synth.jittered(N, 0.4, 3)
    poles = [0.95 * np.exp(1j * a) for a in (0.1 * np.pi, -0.1 * np.pi, 0.3 * np.pi, -0.3 * np.pi)]
    x = synth.ar_process(np.arange(N), poles, 4)
    w, _ = ogpss.nominal_tapers(t, 1.0, 3.0 / N, K)
    idx = np.union1d(sample_bands(I, 256, 1), packed_edge_bands(I, 24))
    J, _, P = oest.m2nufft(t, x, w, -0.5, 1.0 / I, I, idx)
    return J[None], P[None], source_l1(w, x)


def test_fp32_rounded_result_passes():
    J, P, l1 = _case()
    Jg = J.astype(np.complex64)
    Pg = np.mean(np.abs(Jg.astype(np.complex128)) ** 2, axis=1).astype(np.float32)
    r = elementwise_errors(Jg, J, l1, TOL[32], Pg, P, (np.abs(Jg) ** 2).astype(np.float32))
    assert max(r.values()) < 0.05, r


def test_single_band_error_is_caught_where_the_norm_is_not():
    J, P, l1 = _case()
    aJ = np.abs(J[0])
    ratio = aJ / (TOL[32] * l1[0][:, None])
    # every compared entry is well above the bound, so a wrong value anywhere is visible
    assert np.min(ratio) > 10.0
    # a 100 % error (the value zeroed) at any single entry of J or of P-hat fails its check
    rng = np.random.default_rng(0)
    for k, i in zip(rng.integers(0, J.shape[1], 50), rng.integers(0, J.shape[2], 50)):
        Jf = J.copy()
        Jf[0, k, i] = 0.0
        assert elementwise_errors(Jf, J, l1, TOL[32])["J"] > 1.0
        Pf = P.copy()
        Pf[0, i] = 0.0
        assert elementwise_errors(None, J, l1, TOL[32], Pf, P)["P"] > 1.0
    # an 8 % error at one of the weakest entries: the norm over the array lets some through, the
    # bound none
    missed_by_norm = 0
    for flat in np.argsort(ratio.ravel())[:10]:
        k, i = np.unravel_index(flat, ratio.shape)
        Jf = J.copy()
        Jf[0, k, i] *= 1.08
        assert elementwise_errors(Jf, J, l1, TOL[32])["J"] > 1.0
        missed_by_norm += rel_l2(Jf, J) <= TOL[32]
    assert missed_by_norm >= 2
