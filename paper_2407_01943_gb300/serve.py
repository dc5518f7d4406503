"""Continuous-batching PSD server over cached plans.

Requests (pattern id, signal x) arrive over time.  The server keeps one plan
per sampling pattern resident on the device (tapers, point records, twiddles,
deconvolution factors and workspace are built once, before serving), admits
queued requests whenever a launch slot and room in that slot's share of the
device-memory budget are free, groups the admitted requests by pattern so that
each group is one m2nufft_exec over B signals, and runs slots on separate CUDA
streams so a new batch starts while earlier ones are still on the GPU.  The
loop itself is native (csrc/server.cu, include/m2serve.h); this module wraps
it.  A request's latency is its arrival-to-completion time as seen by the host
(P-hat copied back to host memory).  Per-signal results do not depend on the
batch a request lands in (the exec kernels use fixed summation orders and no
atomics).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Optional

import numpy as np


@dataclass
class Request:
    rid: int
    pattern: int
    x: np.ndarray            # [N] float32 samples, in the pattern's time order
    arrival: float           # seconds after the start of the trace
    admitted: float = -1.0
    done: float = -1.0
    P: Optional[np.ndarray] = None


class PSDServer:
    """Native continuous-batching server (include/m2serve.h) over cached FP32 plans.

    plans: {pattern id: binding.Plan}; mem_budget: bytes of device memory for the plans plus
    the per-slot request arenas; slots: concurrent launch slots (CUDA streams); max_batch: most
    requests per launch; want: device outputs per request ("J", "E"; P-hat always)."""

    def __init__(self, plans: Dict[int, object], mem_budget: int, slots: int = 4, max_batch: int = 16,
                 want=("J", "E", "P"), device: int = 0):
        from . import binding
        self._b = binding
        self.ids = sorted(plans)
        self.index = {pid: k for k, pid in enumerate(self.ids)}
        self.plans = plans
        outputs = (binding.M2_OUT_J if "J" in want else 0) | (binding.M2_OUT_E if "E" in want else 0)
        self._h = binding.server_create([plans[pid] for pid in self.ids], int(mem_budget), int(slots),
                                        int(max_batch), outputs)

    def _run(self, requests: List[Request], plain: bool) -> dict:
        for r in requests:
            r.x = np.ascontiguousarray(r.x, dtype=np.float32)
            r.P = np.empty(self.plans[r.pattern].I, dtype=np.float32)
        lat = self._b.server_run(self._h, [self.index[r.pattern] for r in requests], [r.arrival for r in requests],
                                 [r.x for r in requests], [r.P for r in requests], plain)
        for r, l in zip(requests, lat):
            r.done = r.arrival + float(l)
        stats = summarize(requests, self.plans, max(r.done for r in requests) if requests else 0.0)
        stats["launches"] = self._b.server_stats(self._h)[0]
        return stats

    def serve(self, requests: List[Request]) -> dict:
        """Continuous batching of a trace replayed in real time; returns statistics."""
        return self._run(requests, plain=False)

    def serve_plain(self, requests: List[Request]) -> dict:
        """Plain per-request path on the same server: each request alone (B = 1) on one stream."""
        return self._run(requests, plain=True)

    def close(self):
        if getattr(self, "_h", None):
            self._b.server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def summarize(requests: List[Request], plans: Dict[int, object], wall: float) -> dict:
    lat = np.array([r.done - r.arrival for r in requests])
    units = float(sum(plans[r.pattern].K * plans[r.pattern].N * plans[r.pattern].I for r in requests))
    span = max(r.done for r in requests) - min(r.arrival for r in requests)
    return {
        "requests": len(requests),
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "mean_ms": float(lat.mean() * 1e3),
        "throughput_units_per_s": units / span,
        "requests_per_s": len(requests) / span,
        "wall_s": wall,
    }
