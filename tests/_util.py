"""Small helpers shared by the tests (no method arithmetic).

Element-wise parity bound.  A type-1 NuFFT evaluates the finite sum
J_k(f_i) = sum_n c_k[n] exp(-i 2 pi f_i t_n), c_k = w_k x (Eq. eigencoefficients), with an error
that is bounded per output by the kernel's relative accuracy times the l1 norm of the sources:
|J_gpu - J| <= eps * sum_n |c_k[n]| (the window truncation and aliasing errors are bounded
source by source; FFT and spreading rounding add about u * (w + log2 nf) * sum_n |c_k[n]|, far
below eps for both precisions).  The tests assert it with eps = the path's tolerance (1e-5 FP32,
1e-10 FP64) and constant c = 1 at EVERY compared band, so a wrong value at one band fails no matter
how large the spectrum is elsewhere.  For the eigenspectra E = |J|^2 and P-hat = (1/K) sum_k |J_k|^2
(Eq. power_spectrum_estimator) the bound follows by |(a + d)^2 - a^2| <= 2|a||d| + |d|^2:
|dE_k| <= b_k (2 |J_k| + b_k),  |dP| <= (1/K) sum_k b_k (2 |J_k| + b_k),  b_k = eps * sum_n |c_k[n]|.
"""
import numpy as np


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


TOL = {32: 1e-5, 64: 1e-10}
C_BOUND = 1.0  # the constant of the element-wise bound (see the module docstring)

# measured errors of the current session (written out by conftest.py when M2_PARITY_LOG names a file)
PARITY_LOG = []
CURRENT_TEST = [""]


def seeded_tapers(K: int, N: int, seed: int) -> np.ndarray:
    from synth import taper_like
    return taper_like(K, N, seed)


def source_l1(w, X) -> np.ndarray:
    """sum_n |w_k(t_n) x_b(t_n)| as [B, K] (w [K, N] real or complex, X [B, N] or [N])."""
    X = np.atleast_2d(np.asarray(X))
    return (np.abs(np.asarray(w))[None, :, :] * np.abs(X)[:, None, :]).sum(axis=-1)


def elementwise_errors(Jg, Jr, l1, tol, Pg=None, Pr=None, Eg=None):
    """Worst ratio |error| / bound over the compared entries (<= 1 passes), per output.
    Jg (or None: J not checked), Jr [B, K, n]; l1 [B, K]; Pg, Pr [B, n]; Eg [B, K, n]."""
    b = C_BOUND * tol * np.asarray(l1)[:, :, None]  # [B, K, 1]
    out = {}
    if Jg is not None:
        Jg = np.asarray(Jg).reshape(np.shape(Jr))
        out["J"] = float(np.max(np.abs(Jg - Jr) / b))
    aJ = np.abs(Jr)
    if Pg is not None:
        bP = np.mean(b * (2 * aJ + b), axis=1)  # [B, n]
        out["P"] = float(np.max(np.abs(np.asarray(Pg).reshape(np.shape(Pr)) - Pr) / bP))
    if Eg is not None:
        bE = b * (2 * aJ + b)
        out["E"] = float(np.max(np.abs(np.asarray(Eg).reshape(aJ.shape) - aJ ** 2) / bE))
    return out


def assert_elementwise(Jg, Jr, l1, tol, Pg=None, Pr=None, Eg=None):
    """Assert the element-wise bound on J (and P-hat, eigenspectra) at every compared band."""
    r = elementwise_errors(Jg, Jr, l1, tol, Pg, Pr, Eg)
    entry = {"test": CURRENT_TEST[0], "tol": tol, "bands": int(np.shape(Jr)[-1]),
             "elem_over_bound": r}
    rel = {}
    if Jg is not None:
        rel["J"] = rel_l2(Jg, Jr)
    if Pg is not None:
        rel["P"] = rel_l2(Pg, Pr)
        rel["P_max_abs_over_max"] = float(np.max(np.abs(np.asarray(Pg) - Pr)) / np.max(Pr))
    entry["rel_l2"] = rel
    PARITY_LOG.append(entry)
    for k, v in r.items():
        assert v <= 1.0, f"{k}: element-wise error {v:.3g} x the bound {C_BOUND} * {tol:g} * sum|w x|"
    return r


def sample_bands(I: int, n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    edge = np.array([0, 1, I // 2 - 1, I // 2, I // 2 + 1, I - 2, I - 1], dtype=np.int64)
    edge = edge[(edge >= 0) & (edge < I)]
    idx = np.unique(np.concatenate([edge, rng.choice(I, size=min(n, I), replace=False)]))
    return idx.astype(np.int64)


def packed_edge_bands(I: int, n1: int, n2: int = 1024) -> np.ndarray:
    """Band indices at the packed path's special positions.  The packed FFT's spectrum index
    k = k1 + n1 k2 (k1 < n1, k2 < n2) gives band i = i_c + m with m = k (k < nf/2) or k - nf, and
    i_c = floor(I/2); an output thread writes m and -m together.  Covered: the first and last
    band; every k1 of the columns k2 = 0, 1 and the last two in-band columns k2max - 1, k2max
    (k2max = min(n2/2 - 1, ceil((I - i_c)/n1))), on both signs of m; row 0 (k1 = 0, whose
    partner column is n2 - k2 instead of n2 - 1 - k2) at every in-band column; the self-paired
    row k1 = n1/2."""
    i_c = I // 2
    k2max = min(n2 // 2 - 1, -(-(I - i_c) // n1))
    k1 = np.arange(n1)
    ms = [np.array([-i_c, I - 1 - i_c])]
    cols = sorted({c for c in (0, 1, k2max - 1, k2max) if 0 <= c <= k2max})
    for c in cols:
        ms.append(k1 + n1 * c)
    ms.append(n1 * np.arange(k2max + 1))
    if n1 % 2 == 0:
        ms.append(n1 // 2 + n1 * np.arange(0, k2max + 1, max(1, (k2max + 1) // 16)))
    m = np.concatenate(ms)
    m = np.concatenate([m, -m])
    i = m + i_c
    i = i[(i >= 0) & (i < I)]
    return np.unique(i).astype(np.int64)
