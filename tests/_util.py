"""Small helpers shared by the tests (no method arithmetic)."""
import numpy as np


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


TOL = {32: 1e-5, 64: 1e-10}


def seeded_tapers(K: int, N: int, seed: int) -> np.ndarray:
    from synth import taper_like
    return taper_like(K, N, seed)


def sample_bands(I: int, n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    edge = np.array([0, 1, I // 2 - 1, I // 2, I // 2 + 1, I - 2, I - 1], dtype=np.int64)
    edge = edge[(edge >= 0) & (edge < I)]
    idx = np.unique(np.concatenate([edge, rng.choice(I, size=min(n, I), replace=False)]))
    return idx.astype(np.int64)
