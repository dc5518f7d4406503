"""Continuous-batching PSD server over cached plans.

Requests (pattern id, signal x) arrive over time.  The server keeps one plan
per sampling pattern resident on the device (tapers, point records, twiddles,
deconvolution factors and workspace are built once, before serving), admits
queued requests whenever a launch slot and enough of the device-memory budget
are free, groups the admitted requests by pattern so that each group is one
m2nufft_exec over B signals, and runs slots on separate CUDA streams so a new
batch starts while earlier ones are still on the GPU.  A request's latency is
its arrival-to-completion time as seen by the host (P-hat copied back to host
memory).  The per-signal results do not depend on the batch a request lands in
(the exec kernels use fixed summation orders and no atomics).
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field
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


@dataclass
class _Slot:
    stream: object
    event: object = None
    groups: list = field(default_factory=list)   # (requests, device x, J, E, P, host P)
    bytes: int = 0


class PSDServer:
    """plans: {pattern id: binding.Plan} (FP32).  mem_budget: bytes of device memory the
    request buffers in flight may use (plans are counted once, up front)."""

    def __init__(self, plans: Dict[int, object], mem_budget: int, slots: int = 4, max_batch: int = 16,
                 want=("J", "E", "P"), device: int = 0):
        import torch
        self.torch = torch
        self.plans = plans
        self.dev = torch.device("cuda", device)
        self.want = want
        self.max_batch = max_batch
        self.plan_bytes = sum(p.info["device_bytes"] for p in plans.values())
        self.budget = int(mem_budget) - self.plan_bytes
        if self.budget <= 0:
            raise ValueError("memory budget does not cover the cached plans")
        self.slots = [_Slot(stream=torch.cuda.Stream(device=self.dev)) for _ in range(slots)]
        self.in_use = 0

    def request_bytes(self, pattern: int) -> int:
        p = self.plans[pattern]
        b = p.N * 4 + p.I * 4
        if "J" in self.want:
            b += p.K * p.I * 8
        if "E" in self.want:
            b += p.K * p.I * 4
        return b

    # -- one launch: requests grouped by pattern, one exec per group ------------
    def _launch(self, slot: _Slot, reqs: List[Request], now: float):
        torch = self.torch
        by_pat = collections.OrderedDict()
        for r in reqs:
            by_pat.setdefault(r.pattern, []).append(r)
            r.admitted = now
        slot.groups = []
        slot.bytes = sum(self.request_bytes(r.pattern) for r in reqs)
        with torch.cuda.stream(slot.stream):
            for pat, rs in by_pat.items():
                p = self.plans[pat]
                B = len(rs)
                xh = torch.from_numpy(np.stack([r.x for r in rs])).pin_memory()
                xd = torch.empty((B, p.N), dtype=torch.float32, device=self.dev)
                xd.copy_(xh, non_blocking=True)
                J = torch.empty((B, p.K, p.I), dtype=torch.complex64, device=self.dev) if "J" in self.want else None
                E = torch.empty((B, p.K, p.I), dtype=torch.float32, device=self.dev) if "E" in self.want else None
                P = torch.empty((B, p.I), dtype=torch.float32, device=self.dev)
                p.exec(xd, J, E, P, stream=slot.stream)
                ph = torch.empty((B, p.I), dtype=torch.float32).pin_memory()
                ph.copy_(P, non_blocking=True)
                slot.groups.append((rs, xd, J, E, P, ph, xh))
            slot.event = torch.cuda.Event()
            slot.event.record(slot.stream)

    def _retire(self, slot: _Slot, now: float):
        for rs, _xd, _J, _E, _P, ph, _xh in slot.groups:
            Ph = ph.numpy()
            for k, r in enumerate(rs):
                r.done = now
                r.P = Ph[k].copy()
        self.in_use -= slot.bytes
        slot.groups, slot.event, slot.bytes = [], None, 0

    def serve(self, requests: List[Request]) -> dict:
        """Run a trace (requests sorted by arrival) in real time; returns statistics."""
        for r in requests:
            if self.request_bytes(r.pattern) > self.budget:
                raise ValueError(f"request {r.rid} needs more than the memory budget")
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        queue: collections.deque = collections.deque()
        t0 = time.perf_counter()
        busy = 0
        while pending or queue or busy:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            for s in self.slots:
                if s.event is not None and s.event.query():
                    self._retire(s, time.perf_counter() - t0)
                    busy -= 1
            free = [s for s in self.slots if s.event is None]
            if free and queue:
                # a plan's workspace serves one launch at a time: patterns in flight wait
                busy_pat = {r.pattern for s in self.slots for g in s.groups for r in g[0]}
                take: List[Request] = []
                keep: collections.deque = collections.deque()
                while queue and len(take) < self.max_batch:
                    r = queue.popleft()
                    if r.pattern in busy_pat:
                        keep.append(r)
                        continue
                    need = self.request_bytes(r.pattern)
                    if self.in_use + need > self.budget:
                        keep.append(r)
                        break
                    self.in_use += need
                    take.append(r)
                queue.extendleft(reversed(keep))
                if take:
                    self._launch(free[0], take, time.perf_counter() - t0)
                    busy += 1
                    continue
            if not queue and not busy and pending:
                # idle until the next arrival
                wait = pending[0].arrival - (time.perf_counter() - t0)
                if wait > 2e-4:
                    time.sleep(wait - 1e-4)
        wall = time.perf_counter() - t0
        return summarize(requests, self.plans, wall)


def serve_plain(plans: Dict[int, object], requests: List[Request], want=("J", "E", "P"), device: int = 0) -> dict:
    """Plain per-request path: each request alone (one exec, B = 1) on one stream, in arrival
    order, as soon as it has arrived and the previous one has finished."""
    import torch
    dev = torch.device("cuda", device)
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda r: r.arrival):
        while time.perf_counter() - t0 < r.arrival:
            pass
        p = plans[r.pattern]
        r.admitted = time.perf_counter() - t0
        xh = torch.from_numpy(r.x[None, :]).pin_memory()
        xd = xh.to(dev, non_blocking=True)
        J = torch.empty((1, p.K, p.I), dtype=torch.complex64, device=dev) if "J" in want else None
        E = torch.empty((1, p.K, p.I), dtype=torch.float32, device=dev) if "E" in want else None
        P = torch.empty((1, p.I), dtype=torch.float32, device=dev)
        p.exec(xd, J, E, P, stream=stream)
        r.P = P.cpu().numpy()[0]
        r.done = time.perf_counter() - t0
    wall = time.perf_counter() - t0
    return summarize(requests, plans, wall)


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
