"""Seeded synthetic inputs for the M2NuFFT hot path.

This module produces sampling patterns and signals only.  It contains none of
the estimator's arithmetic (no GPSS matrices, tapers, transforms or spectra),
so both the CPU oracle's tests and the CUDA path can draw the same inputs
from it without sharing any method code.

Every generator takes an explicit seed and uses numpy's PCG64 generator.

Workloads (sizes and distributions follow the paper's problem statement:
samples x(t_n) at arbitrary times t_n, a signal band |f| <= fs/2, analysis
bands of half-width f_w and K tapers; Sec. 2 and Table 1 steps 1-2):

  grid_bernoulli   : unit-rate grid 0..G-1 with i.i.d. Bernoulli missing samples
  jittered         : t_n = n + U(-a, a), sorted
  markov_missing   : unit grid with bursty gaps from a 2-state Markov chain
  periodic_missing : unit grid, each block of `beta` samples drops its last `drop`
  scaled_missing   : t_n = r*n on a kept subset (sampling-rate mismatch example,
                     Sec. 4's missing-data scheme with t_n = 5n/6)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Workload",
    "grid_bernoulli",
    "jittered",
    "markov_missing",
    "periodic_missing",
    "scaled_missing",
    "tones",
    "ar_process",
    "chirp_plus_pink",
    "white",
    "workload",
    "batched_uneven",
    "serving_patterns",
    "poisson_arrivals",
    "taper_like",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ---------------------------------------------------------------------------
# sampling patterns
# ---------------------------------------------------------------------------
def grid_bernoulli(G: int, missing: float, seed: int) -> np.ndarray:
    """Integer times 0..G-1 keeping each sample with probability 1-missing."""
    keep = _rng(seed).random(G) >= missing
    return np.nonzero(keep)[0].astype(np.float64)


def jittered(N: int, amp: float, seed: int) -> np.ndarray:
    """t_n = n + U(-amp, amp), n = 0..N-1, returned sorted."""
    t = np.arange(N, dtype=np.float64) + _rng(seed).uniform(-amp, amp, N)
    t.sort()
    return t


def markov_missing(G: int, p_gap_gap: float, missing: float, seed: int) -> np.ndarray:
    """Unit grid with gaps from a 2-state Markov chain.

    P(gap -> gap) = p_gap_gap; P(obs -> gap) is set so the stationary gap
    rate equals `missing`:  pi_gap = p_og / (p_og + 1 - p_gg).
    """
    p_og = missing * (1.0 - p_gap_gap) / (1.0 - missing)
    r = _rng(seed).random(G)
    gap = np.zeros(G, dtype=bool)
    state = r[0] < missing
    for n in range(G):
        if n > 0:
            state = (r[n] < p_gap_gap) if state else (r[n] < p_og)
        gap[n] = state
    if gap.all():
        gap[0] = False
    return np.nonzero(~gap)[0].astype(np.float64)


def periodic_missing(G: int, beta: int, drop: int) -> np.ndarray:
    """Unit grid where every block of `beta` samples loses its last `drop`."""
    n = np.arange(G)
    return n[(n % beta) < (beta - drop)].astype(np.float64)


def scaled_missing(G: int, n_drop: int, rate: float, seed: int) -> np.ndarray:
    """t_n = rate * n for n = 1..G with n_drop samples removed at random."""
    n = np.arange(1, G + 1, dtype=np.float64)
    drop = _rng(seed).choice(G, size=n_drop, replace=False)
    keep = np.ones(G, dtype=bool)
    keep[drop] = False
    return rate * n[keep]


# ---------------------------------------------------------------------------
# signals (values at the given times)
# ---------------------------------------------------------------------------
def white(t: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    return sigma * _rng(seed).standard_normal(t.shape[0])


def tones(t: np.ndarray, freqs, amps, noise_sigma: float, seed: int) -> np.ndarray:
    """Sum of real sinusoids with random phases plus white Gaussian noise."""
    rng = _rng(seed)
    x = noise_sigma * rng.standard_normal(t.shape[0])
    for f, a in zip(freqs, amps):
        x += a * np.cos(2.0 * np.pi * f * t + rng.uniform(0.0, 2.0 * np.pi))
    return x


def ar_process(n_index: np.ndarray, poles, seed: int, burn_in: int = 1000) -> np.ndarray:
    """AR process driven by unit-variance innovations, run on the integer
    index and read at the given indices.  `poles` are complex; conjugate
    pairs give real coefficients."""
    from scipy.signal import lfilter
    a = np.real(np.poly(poles))                  # x[n] + a1 x[n-1] + ... = e[n]
    L = int(n_index.max()) + 1 + burn_in
    e = _rng(seed).standard_normal(L)
    x = lfilter([1.0], a, e)
    return x[burn_in + n_index.astype(np.int64)]


def chirp_plus_pink(t: np.ndarray, f0: float, f1: float, T: float, pink_sigma: float,
                    seed: int) -> np.ndarray:
    """Linear chirp f0 -> f1 over [0, T] plus 1/f noise scaled to pink_sigma.

    The pink noise is white noise filtered by 1/sqrt(f) on the integer grid
    covering t and then read at round(t)."""
    rng = _rng(seed)
    G = int(math.ceil(t.max())) + 1
    w = rng.standard_normal(G)
    Wf = np.fft.rfft(w)
    f = np.fft.rfftfreq(G)
    f[0] = f[1]
    pink = np.fft.irfft(Wf / np.sqrt(f), n=G)
    pink *= pink_sigma / pink.std()
    chirp = np.cos(2.0 * np.pi * (f0 * t + (f1 - f0) * t * t / (2.0 * T)))
    return chirp + pink[np.rint(t).astype(np.int64).clip(0, G - 1)]


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    t: np.ndarray            # sampling times (float64, as given to the plan)
    x: np.ndarray            # [B, N] float64 signals at those times
    fs: float                # nominal sampling rate; signal band |f| <= fs/2
    f_w: float               # half-bandwidth of the analysis bands
    K: int                   # number of tapers
    f_lo: float              # first band centre
    df: float                # band-centre spacing
    I: int                   # number of band centres
    grid_len: int            # nominal grid length that f_w and I are defined from
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.t.shape[0])

    @property
    def B(self) -> int:
        return int(self.x.shape[0])


def workload(name: str, batch: int = 1, seed: int = 0) -> Workload:
    """Synthetic stand-ins for the paper's workloads at scale.

    name:
      'grid1024'     N=1024 unit grid, 20% Bernoulli missing, 3 tones + noise,
                     f_w = 4/1024, K = 6, I = 1024 band centres on [-0.5, 0.5)
      'jitter16k'    N=16384 jittered (+-0.4), AR(4), f_w = 5/N, K = 8, I = 2^18
      'periodic16k'  N=16384 grid, blocks of 8 drop 2, chirp + pink noise,
                     f_w = 6/N, K = 10, I = 2^20
    `batch` signals are drawn on the same sampling pattern (seeds seed..seed+B-1).
    """
    if name == "grid1024":
        G = 1024
        t = grid_bernoulli(G, 0.2, seed)
        x = np.stack([tones(t, (0.11, 0.23, 0.37), (1.0, 1.0, 1.0), 1.0, 1000 + seed + b)
                      for b in range(batch)])
        return Workload(name, t, x, 1.0, 4.0 / G, 6, -0.5, 1.0 / 1024, 1024, G)
    if name == "jitter16k":
        G = 16384
        t = jittered(G, 0.4, seed)
        poles = [0.95 * np.exp(s * 1j * a * np.pi) for a in (0.1, 0.3) for s in (1, -1)]
        idx = np.arange(G)
        x = np.stack([ar_process(idx, poles, 2000 + seed + b) for b in range(batch)])
        I = 1 << 18
        return Workload(name, t, x, 1.0, 5.0 / G, 8, -0.5, 1.0 / I, I, G)
    if name == "periodic16k":
        G = 16384
        t = periodic_missing(G, 8, 2)
        x = np.stack([chirp_plus_pink(t, 0.05, 0.45, float(G), 0.5, 3000 + seed + b)
                      for b in range(batch)])
        I = 1 << 20
        return Workload(name, t, x, 1.0, 6.0 / G, 10, -0.5, 1.0 / I, I, G)
    raise ValueError(f"unknown workload {name!r}")


def batched_uneven(n_signals: int, seed: int = 0, n_min: int = 1024, n_max: int = 16384):
    """Uneven batch: grid length log-uniform in [n_min, n_max], Markov gaps
    (P(gap->gap)=0.9, 15% missing), white noise plus 1-4 tones at 0-20 dB SNR,
    K in {4, 6, 8}, f_w = (K/2+1)/G, I = 4G band centres on [-0.5, 0.5)."""
    rng = _rng(seed)
    out = []
    for s in range(n_signals):
        G = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        t = markov_missing(G, 0.9, 0.15, seed * 100003 + s)
        ntone = int(rng.integers(1, 5))
        freqs = rng.uniform(-0.5, 0.5, ntone)
        snr = rng.uniform(0.0, 20.0, ntone)
        amps = np.sqrt(2.0 * 10.0 ** (snr / 10.0))
        x = tones(t, freqs, amps, 1.0, seed * 100003 + s + 7)[None, :]
        K = int(rng.choice([4, 6, 8]))
        I = 4 * G
        out.append(Workload(f"uneven{s}", t, x, 1.0, (K / 2 + 1) / G, K, -0.5, 1.0 / I, I, G))
    return out


def serving_patterns(n_patterns: int = 64, seed: int = 0, n_min: int = 2048,
                     n_max: int = 16384):
    """Fixed sampling patterns for the request stream: grid length uniform in
    [n_min, n_max], jittered (+-0.4) or Bernoulli-missing at 10-30%."""
    rng = _rng(seed)
    pats = []
    for p in range(n_patterns):
        G = int(rng.integers(n_min, n_max + 1))
        if p % 2 == 0:
            t = jittered(G, 0.4, 7919 * (p + 1) + seed)
            kind = "jitter"
        else:
            t = grid_bernoulli(G, float(rng.uniform(0.1, 0.3)), 7919 * (p + 1) + seed)
            kind = "bernoulli"
        pats.append({"t": t, "G": G, "kind": kind, "K": 8, "f_w": 5.0 / G,
                     "f_lo": -0.5, "I": 4 * G, "df": 1.0 / (4 * G)})
    return pats


def poisson_arrivals(rate_hz: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process."""
    return np.cumsum(_rng(seed).exponential(1.0 / rate_hz, n))


def taper_like(K: int, N: int, seed: int) -> np.ndarray:
    """Arbitrary real taper-shaped rows [K, N] (sine windows times cosines
    plus 1% noise, scaled like unit-energy tapers).  Used as inputs where
    the dense GEP would be too slow to run beside the check: the
    eigencoefficient sum is linear in the taper, so any real sequence is a
    valid input to it."""
    rng = _rng(seed)
    n = np.arange(N)
    base = np.sin(np.pi * (n + 0.5) / N)
    return np.stack([base * np.cos(np.pi * k * (n + 0.5) / N) + 0.01 * rng.standard_normal(N)
                     for k in range(K)]) * np.sqrt(2.0 / N)
