"""Thin Python binding of libm2nufft (include/m2nufft.h) via ctypes.

Argument marshalling only: every step of the path runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams; numpy supplies
host arrays.  If the shared library is missing or fails to load, every
entry point raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

from . import _build_lib

M2_OK = 0
M2_OUT_J, M2_OUT_E, M2_OUT_P = 1, 2, 4
STATUS_NAMES = {0: "M2_OK", 1: "M2_ERR_ARG", 2: "M2_ERR_NOMEM", 3: "M2_ERR_BUDGET", 4: "M2_ERR_GEP",
                5: "M2_ERR_CUDA", 6: "M2_ERR_TIMEOUT", 7: "M2_ERR_CANCELLED"}


class M2Error(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")


class m2_fgrid(ctypes.Structure):
    _fields_ = [("f_lo", ctypes.c_double), ("df", ctypes.c_double), ("I", ctypes.c_int64)]


class m2_subband(ctypes.Structure):
    _fields_ = [("f_c0", ctypes.c_double), ("f_min", ctypes.c_double), ("f_max", ctypes.c_double)]


class m2_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double), ("mem_budget", ctypes.c_size_t),
                ("device", ctypes.c_int), ("max_batch", ctypes.c_int), ("path", ctypes.c_int),
                ("tapers", ctypes.c_int), ("sigma", ctypes.c_double), ("tune", ctypes.c_int)]


class m2_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("K", ctypes.c_int), ("I", ctypes.c_int64), ("precision", ctypes.c_int),
                ("width", ctypes.c_int), ("beta", ctypes.c_double), ("nf", ctypes.c_int64),
                ("n1", ctypes.c_int64), ("n2", ctypes.c_int64), ("rows", ctypes.c_int64), ("wrap", ctypes.c_int),
                ("real_taper", ctypes.c_int), ("integer_grid", ctypes.c_int), ("chunk", ctypes.c_int),
                ("path", ctypes.c_int),
                ("device_bytes", ctypes.c_size_t), ("gep_seconds", ctypes.c_double),
                ("spread_entries", ctypes.c_int64)]


# (name, restype, argtypes) of every exported entry point of include/m2nufft.h
_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
EXPORTS = [
    ("m2nufft_plan", ctypes.c_int, [_DP, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.POINTER(m2_fgrid), ctypes.POINTER(m2_opts), ctypes.POINTER(_VP)]),
    ("m2nufft_plan_with_tapers", ctypes.c_int,
     [_DP, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.POINTER(m2_fgrid), _DP, _DP,
      ctypes.POINTER(m2_opts), ctypes.POINTER(_VP)]),
    ("m2nufft_exec", ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP, _VP, _VP, _VP, _VP]),
    ("m2nufft_exec_ftest", ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP, _VP, _VP, _VP]),
    ("m2nufft_exec_batch", ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.c_int64,
                                          ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]),
    ("m2nufft_exec_batch_ftest", ctypes.c_int,
     [ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.c_int64, ctypes.POINTER(_VP), ctypes.POINTER(_VP),
      ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]),
    ("m2nufft_set_batch_mode", ctypes.c_int, [ctypes.c_int]),
    ("m2nufft_get_batch_tuning", ctypes.c_int, [ctypes.POINTER(ctypes.c_int), _VP, _DP]),
    ("m2nufft_get_tuning", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), _VP, _DP]),
    ("m2nufft_get_tapers", ctypes.c_int, [_VP, _DP, _DP]),
    ("m2nufft_get_tapers_complex", ctypes.c_int, [_VP, _DP, _DP]),
    ("m2nufft_plan_subband", ctypes.c_int, [_DP, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                            ctypes.POINTER(m2_subband), ctypes.POINTER(m2_fgrid), _DP, _DP,
                                            ctypes.POINTER(m2_opts), ctypes.POINTER(_VP)]),
    ("m2nufft_get_leakage", ctypes.c_int, [_VP, _DP, _DP]),
    ("m2nufft_get_info", ctypes.c_int, [_VP, ctypes.POINTER(m2_info)]),
    ("m2nufft_set_timing", ctypes.c_int, [_VP, ctypes.c_int]),
    ("m2nufft_get_timing", ctypes.c_int, [_VP, _DP, ctypes.POINTER(ctypes.c_int64)]),
    ("m2nufft_leakage_static", ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                              ctypes.POINTER(m2_fgrid), _VP, _VP, _VP, _VP, _VP]),
    ("m2nufft_pipe_selftest", ctypes.c_int, [ctypes.c_int, _VP]),
    ("m2nufft_true_suboptimality", ctypes.c_int, [_VP, _DP, _DP]),
    ("m2nufft_get_pipe_profile", ctypes.c_int, [_VP, _DP, _DP, ctypes.POINTER(ctypes.c_int64)]),
    ("m2nufft_destroy", ctypes.c_int, [_VP]),
    ("m2nufft_last_error", ctypes.c_char_p, []),
    ("m2nufft_version", ctypes.c_char_p, []),
]

# entry points of include/m2serve.h
SERVE_EXPORTS = [
    ("m2serve_create", ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_uint, ctypes.POINTER(_VP)]),
    ("m2serve_run_trace", ctypes.c_int, [_VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    ("m2serve_stats", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    ("m2serve_destroy", ctypes.c_int, [_VP]),
]

_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None


def lib_path() -> str:
    return _build_lib.LIB_PATH


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libm2nufft.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing and _build_lib.is_stale():
                _build_lib.build()
            if not os.path.exists(_build_lib.LIB_PATH):
                raise RuntimeError("libm2nufft.so is not built; run paper_2407_01943_gb300.build()")
            L = ctypes.CDLL(_build_lib.LIB_PATH)
            for name, res, args in EXPORTS + SERVE_EXPORTS:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status: int, where: str):
    if status != M2_OK:
        raise M2Error(status, where, load().m2nufft_last_error().decode())


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _tptr(x) -> Optional[int]:
    """Device pointer of a torch tensor (None -> NULL)."""
    if x is None:
        return None
    if not x.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return x.data_ptr()


def _optr(x) -> Optional[int]:
    """Pointer of an output tensor: device memory, or page-locked host memory that the device
    addresses directly (the kernels then write the results straight to host memory)."""
    if x is None:
        return None
    if not (x.is_cuda or x.is_pinned()):
        raise ValueError("expected a CUDA tensor or a pinned host tensor")
    if not x.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return x.data_ptr()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """A cached M2NuFFT plan for one sampling pattern and one band grid."""

    def __init__(self, t, fs: float, f_w: float, K: int, f_lo: float, df: float, I: int,
                 precision: int = 32, tol: float = 0.0, mem_budget: int = 0, device: int = -1,
                 max_batch: int = 0, tapers=None, lam=None, path: int = 0, taper_design: str = "gep",
                 subband=None, sigma: float = 0.0, tune: bool = False):
        """subband = (f_c0, f_min, f_max) makes a sub-band plan (m2nufft_plan_subband): band centres
        f_lo + i df are absolute, tapers (if given) complex [K, N].  sigma > 0 asks for an
        oversampling factor of at least sigma; tune = True times the packed configurations at plan
        time and keeps the fastest (report: tuning())."""
        L = load()
        self._t = np.ascontiguousarray(t, dtype=np.float64)
        self.N = int(self._t.shape[0])
        self.K = int(K)
        self.I = int(I)
        self.precision = int(precision)
        self.fs, self.f_w, self.f_lo, self.df = float(fs), float(f_w), float(f_lo), float(df)
        fg = m2_fgrid(self.f_lo, self.df, self.I)
        design = {"gep": 0, "spline": 1}[taper_design]
        op = m2_opts(self.precision, float(tol), int(mem_budget), int(device), int(max_batch), int(path), design,
                     float(sigma), 1 if tune else 0)
        h = _VP()
        self.subband = subband
        if subband is not None:
            sb = m2_subband(*[float(v) for v in subband])
            wp = lp = None
            if tapers is not None:
                wc = np.ascontiguousarray(np.asarray(tapers, dtype=np.complex128))
                if wc.shape != (self.K, self.N):
                    raise ValueError(f"tapers must have shape ({self.K}, {self.N})")
                self._wc_in = wc.view(np.float64)
                wp = _dptr(self._wc_in)
            if lam is not None:
                self._lam_in = np.ascontiguousarray(lam, dtype=np.float64)
                lp = _dptr(self._lam_in)
            st = L.m2nufft_plan_subband(_dptr(self._t), self.N, self.fs, self.f_w, self.K, ctypes.byref(sb),
                                        ctypes.byref(fg), wp, lp, ctypes.byref(op), ctypes.byref(h))
            _check(st, "m2nufft_plan_subband")
        elif tapers is None:
            st = L.m2nufft_plan(_dptr(self._t), self.N, self.fs, self.f_w, self.K, ctypes.byref(fg),
                                ctypes.byref(op), ctypes.byref(h))
            _check(st, "m2nufft_plan")
        else:
            w = np.ascontiguousarray(tapers, dtype=np.float64)
            if w.shape != (self.K, self.N):
                raise ValueError(f"tapers must have shape ({self.K}, {self.N})")
            lp = None
            if lam is not None:
                self._lam_in = np.ascontiguousarray(lam, dtype=np.float64)
                lp = _dptr(self._lam_in)
            st = L.m2nufft_plan_with_tapers(_dptr(self._t), self.N, self.fs, self.f_w, self.K, ctypes.byref(fg),
                                            _dptr(w), lp, ctypes.byref(op), ctypes.byref(h))
            _check(st, "m2nufft_plan_with_tapers")
        self._h = h
        inf = m2_info()
        _check(L.m2nufft_get_info(self._h, ctypes.byref(inf)), "m2nufft_get_info")
        self.info = {f: getattr(inf, f) for f, _ in m2_info._fields_}

    # -- properties -----------------------------------------------------
    @property
    def handle(self):
        return self._h

    @property
    def real_dtype(self):
        import torch
        return torch.float32 if self.precision == 32 else torch.float64

    @property
    def complex_dtype(self):
        import torch
        return torch.complex64 if self.precision == 32 else torch.complex128

    def tapers(self):
        """(w [K, N], lambda [K]); w is complex for a sub-band plan."""
        lam = np.empty(self.K)
        if self.subband is not None:
            wc = np.empty((self.K, self.N), dtype=np.complex128)
            _check(load().m2nufft_get_tapers_complex(self._h, _dptr(wc.view(np.float64)), _dptr(lam)),
                   "m2nufft_get_tapers_complex")
            return wc, lam
        w = np.empty((self.K, self.N))
        _check(load().m2nufft_get_tapers(self._h, _dptr(w), _dptr(lam)), "m2nufft_get_tapers")
        return w, lam

    def leakage(self):
        Lh = np.empty((self.K, self.I))
        Eh = np.empty(self.I)
        _check(load().m2nufft_get_leakage(self._h, _dptr(Lh), _dptr(Eh)), "m2nufft_get_leakage")
        return Lh, Eh

    # -- execution ------------------------------------------------------
    def exec(self, x, J=None, E=None, P=None, Lhat=None, Ehat=None, stream=None, F=None):
        """Enqueue the path for x [B, N] (torch CUDA tensor of the plan's real dtype); with F
        [B, I], also the F-statistic (m2nufft_exec_ftest; L-hat/E-hat then not copied)."""
        if x.dim() != 2 or x.shape[1] != self.N:
            raise ValueError(f"x must have shape [B, {self.N}]")
        if x.dtype != self.real_dtype:
            raise ValueError(f"x must be {self.real_dtype}")
        B = int(x.shape[0])
        for name, a, shape, dt in (("J", J, (B, self.K, self.I), self.complex_dtype),
                                   ("E", E, (B, self.K, self.I), self.real_dtype),
                                   ("P", P, (B, self.I), self.real_dtype),
                                   ("F", F, (B, self.I), self.real_dtype)):
            if a is not None and (tuple(a.shape) != shape or a.dtype != dt):
                raise ValueError(f"{name} must be {dt} with shape {shape}")
        if F is not None:
            if Lhat is not None or Ehat is not None:
                raise ValueError("exec with F does not copy L-hat/E-hat; call leakage() or a second exec")
            st = load().m2nufft_exec_ftest(self._h, _tptr(x), B, _optr(J), _optr(E), _optr(P), _optr(F),
                                           _stream_handle(stream))
            _check(st, "m2nufft_exec_ftest")
            return
        st = load().m2nufft_exec(self._h, _tptr(x), B, _optr(J), _optr(E), _optr(P), _optr(Lhat),
                                 _optr(Ehat), _stream_handle(stream))
        _check(st, "m2nufft_exec")

    def run(self, x, want=("J", "E", "P"), stream=None):
        """Allocate the requested outputs with torch and run; returns a dict."""
        import torch
        B = int(x.shape[0])
        dev = x.device
        out = {}
        if "J" in want:
            out["J"] = torch.empty((B, self.K, self.I), dtype=self.complex_dtype, device=dev)
        if "E" in want:
            out["E"] = torch.empty((B, self.K, self.I), dtype=self.real_dtype, device=dev)
        if "P" in want:
            out["P"] = torch.empty((B, self.I), dtype=self.real_dtype, device=dev)
        if "Lhat" in want:
            out["Lhat"] = torch.empty((self.K, self.I), dtype=torch.float64, device=dev)
        if "Ehat" in want:
            out["Ehat"] = torch.empty((self.I,), dtype=torch.float64, device=dev)
        if "F" in want:
            out["F"] = torch.empty((B, self.I), dtype=self.real_dtype, device=dev)
            self.exec(x, out.get("J"), out.get("E"), out.get("P"), stream=stream, F=out["F"])
            if "Lhat" in out or "Ehat" in out:
                self.exec(x[:0], None, None, None, out.get("Lhat"), out.get("Ehat"), stream)
            return out
        self.exec(x, out.get("J"), out.get("E"), out.get("P"), out.get("Lhat"), out.get("Ehat"), stream)
        return out

    def set_timing(self, enable: bool = True):
        _check(load().m2nufft_set_timing(self._h, 1 if enable else 0), "m2nufft_set_timing")

    def get_timing(self):
        """(ms[4], launches[4]) of spread / column FFT / row FFT / packed epilogue since the last call."""
        ms = np.zeros(4)
        n = np.zeros(4, dtype=np.int64)
        _check(load().m2nufft_get_timing(self._h, _dptr(ms), n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
               "m2nufft_get_timing")
        return ms, n

    def tuning(self):
        """Autotuning report: [(path, sigma, max_batch, ms per exec)] for the candidates tried."""
        L = load()
        n = ctypes.c_int(0)
        _check(L.m2nufft_get_tuning(self._h, ctypes.byref(n), None, None), "m2nufft_get_tuning")
        if n.value == 0:
            return []
        ops = (m2_opts * n.value)()
        ms = np.zeros(n.value)
        _check(L.m2nufft_get_tuning(self._h, ctypes.byref(n), ctypes.cast(ops, _VP), _dptr(ms)),
               "m2nufft_get_tuning")
        return [(int(o.path), float(o.sigma), int(o.max_batch), float(m)) for o, m in zip(ops, ms)]

    def true_suboptimality(self):
        """(E [I], per-band eigenvalues [I, K]) from per-band GEPs (small N only)."""
        E = np.empty(self.I)
        lb = np.empty((self.I, self.K))
        _check(load().m2nufft_true_suboptimality(self._h, _dptr(E), _dptr(lb)), "m2nufft_true_suboptimality")
        return E, lb

    def get_pipe_profile(self):
        """Persistent kernel (path 3): per-stage (spread, columns, rows, epilogue) summed item
        time in ms, summed dependency-wait time in ms and item counts since the last call."""
        busy, wait = np.zeros(4), np.zeros(4)
        n = np.zeros(4, dtype=np.int64)
        _check(load().m2nufft_get_pipe_profile(self._h, _dptr(busy), _dptr(wait),
                                               n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
               "m2nufft_get_pipe_profile")
        return busy, wait, n

    def close(self):
        if getattr(self, "_h", None):
            load().m2nufft_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class BatchCall:
    """m2nufft_exec_batch (m2nufft_exec_batch_ftest when Fs is given) with its argument arrays
    marshalled once: for a batch that is run repeatedly on the same plans and buffers, each call
    then only launches (the library replays its cached graph for the same plans and pointers).
    The tensors must stay alive and in place while the object is used."""

    def __init__(self, plans: Sequence[Plan], xs, Js=None, Es=None, Ps=None, Fs=None):
        n = len(plans)
        arr = lambda vals: (_VP * n)(*vals)
        self._keep = (list(plans), xs, Js, Es, Ps, Fs)
        self.n = n
        self.hp = arr([p.handle.value for p in plans])
        self.hx = arr([_tptr(x) for x in xs])
        self.hJ = arr([_optr(j) for j in Js]) if Js is not None else None
        self.hE = arr([_optr(e) for e in Es]) if Es is not None else None
        self.hP = arr([_optr(q) for q in Ps]) if Ps is not None else None
        self.hF = arr([_optr(f) for f in Fs]) if Fs is not None else None

    def __call__(self, stream=None):
        if self.hF is not None:
            st = load().m2nufft_exec_batch_ftest(self.hp, self.hx, self.n, self.hJ, self.hE, self.hP, self.hF,
                                                 _stream_handle(stream))
            _check(st, "m2nufft_exec_batch_ftest")
            return
        st = load().m2nufft_exec_batch(self.hp, self.hx, self.n, self.hJ, self.hE, self.hP, _stream_handle(stream))
        _check(st, "m2nufft_exec_batch")


def exec_batch(plans: Sequence[Plan], xs, Js=None, Es=None, Ps=None, Fs=None, stream=None):
    """Uneven batch: one signal per entry, each with its own plan; Fs (optional, entries may be
    None) adds Thomson's F-statistic for the signals that give one."""
    BatchCall(plans, xs, Js, Es, Ps, Fs)(stream)


def leakage_static(t, w, lam, fs: float, f_w: float, f_lo: float, df: float, I: int, Lhat, Ehat, stream=None):
    """L-hat [K, I] and E-hat [I] without a plan or any allocation (torch CUDA float64
    tensors for t [N], w [K, N], lam [K], Lhat, Ehat)."""
    K, N = int(w.shape[0]), int(w.shape[1])
    fg = m2_fgrid(float(f_lo), float(df), int(I))
    st = load().m2nufft_leakage_static(_tptr(t), N, float(fs), float(f_w), K, ctypes.byref(fg), _tptr(w),
                                       _tptr(lam), _tptr(Lhat), _tptr(Ehat), _stream_handle(stream))
    _check(st, "m2nufft_leakage_static")


def set_batch_mode(mode: int) -> int:
    """0 = all-packed exec_batch as one launch per stage (default), 1 = one persistent
    pipelined kernel, 2 = the fastest of those forms and CTA shapes, tuned on the first call for a
    batch; returns the previous mode."""
    prev = int(load().m2nufft_set_batch_mode(int(mode)))
    if prev < 0:
        raise ValueError(load().m2nufft_last_error().decode())
    return prev


def batch_tuning():
    """Candidates of the most recently tuned batch (batch mode 2): a list of
    ((mode, spread tiles per CTA, rows per CTA, epilogue tile height), ms per batch)."""
    n = ctypes.c_int(0)
    _check(load().m2nufft_get_batch_tuning(ctypes.byref(n), None, None), "m2nufft_get_batch_tuning")
    cfg = np.zeros((max(n.value, 1), 4), dtype=np.int32)
    ms = np.zeros(max(n.value, 1))
    _check(load().m2nufft_get_batch_tuning(ctypes.byref(n), cfg.ctypes.data_as(ctypes.c_void_p), _dptr(ms)),
           "m2nufft_get_batch_tuning")
    return [(tuple(int(v) for v in cfg[i]), float(ms[i])) for i in range(n.value)]


def batch_pipe_profile():
    """Stage accounting (busy ms, wait ms, items per stage) of the most recently launched
    all-packed exec_batch graph, since the previous call."""
    busy, wait = np.zeros(4), np.zeros(4)
    n = np.zeros(4, dtype=np.int64)
    _check(load().m2nufft_get_pipe_profile(None, _dptr(busy), _dptr(wait),
                                           n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
           "m2nufft_get_pipe_profile")
    return busy, wait, n


def pipe_selftest(timeout_ms: int, stream=None) -> int:
    """Bounded-wait self-test of the persistent kernel; returns the raw status
    (M2_ERR_TIMEOUT is the expected outcome)."""
    return int(load().m2nufft_pipe_selftest(int(timeout_ms), _stream_handle(stream)))


def server_create(plans, mem_budget: int, slots: int, max_batch: int, outputs: int):
    n = len(plans)
    hp = (_VP * n)(*[p.handle.value for p in plans])
    h = _VP()
    _check(load().m2serve_create(hp, n, mem_budget, slots, max_batch, outputs, ctypes.byref(h)), "m2serve_create")
    return h


def server_run(h, patterns, arrivals, xs, ps, plain: bool):
    """Replay a trace; xs / ps are lists of float32 numpy arrays (inputs / P-hat destinations)."""
    n = len(patterns)
    pat = np.ascontiguousarray(patterns, dtype=np.int32)
    arr = np.ascontiguousarray(arrivals, dtype=np.float64)
    hx = (_VP * n)(*[x.ctypes.data for x in xs])
    hpo = (_VP * n)(*[q.ctypes.data for q in ps])
    lat = np.zeros(n)
    st = load().m2serve_run_trace(h, n, pat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dptr(arr), hx, hpo,
                                  _dptr(lat), 1 if plain else 0)
    _check(st, "m2serve_run_trace")
    return lat


def server_stats(h):
    a = ctypes.c_int64()
    b = ctypes.c_int64()
    _check(load().m2serve_stats(h, ctypes.byref(a), ctypes.byref(b)), "m2serve_stats")
    return a.value, b.value


def server_destroy(h):
    load().m2serve_destroy(h)


def version() -> str:
    return load().m2nufft_version().decode()
