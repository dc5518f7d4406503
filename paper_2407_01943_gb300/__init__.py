"""GB300 (sm_103a) multitaper NuFFT power-spectrum path.

Implements the per-signal hot path of the Multiband-Multitaper NuFFT
(Cui, Brinkmann & Worrell, arXiv 2407.01943): FP64 nominal-band GPSS tapers
solved once per sampling pattern (Sec. 3.2, Eq. gep_at_A0), then, per signal,
eigencoefficients by a hand-written nonuniform FFT (Eq. eigencoefficients),
eigenspectra and the multitaper estimate (Eq. power_spectrum_estimator), and
the leakage estimates of App. B.

The compute lives in libm2nufft.so (csrc/, C ABI in include/m2nufft.h);
`binding` marshals arguments to it.
"""
from ._build_lib import build as build_library  # noqa: F401
from .binding import BatchCall, M2Error, Plan, exec_batch, load, lib_path, version  # noqa: F401


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a (in-tree) and load it."""
    path = build_library(force=force)
    return path
