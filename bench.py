#!/usr/bin/env python3
"""Throughput benchmark of the GB300 multitaper NuFFT path.

One step = one exec of the whole per-signal path (spread, four-step FFT,
deconvolve, J, eigenspectra, P-hat; the leakage estimates are plan
constants) over a batch of B synthetic signals that share one sampling
pattern, per GPU.  Default workload: N = 16384 jittered samples
(t_n = n + U(-0.4, 0.4)), AR(4) signals, K = 8 tapers, f_w = 5/N,
I = 2^18 band centres on [-1/2, 1/2), FP32 path with FP64-split coordinates.

Metric: tapered samples x bands per second, sum over signals of K * N * I,
whole job.  Multi-GPU (torchrun): each rank runs its own batch (independent
signals, no data-path collective), weak scaling; the timed region is
bracketed by a barrier and synchronisation and the max over ranks is taken.

--impl reference times the CPU oracle (direct FP64 sum) on a bounded sample
of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "tapered samples x bands per second (sum of K*N*I over signals)"
UNIT = "samples*bands/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="jitter16k",
                    choices=["jitter16k", "periodic16k", "grid1024", "uneven", "serve", "multiband", "subopt"])
    ap.add_argument("--taper-design", default="gep", choices=["gep", "spline"],
                    help="nominal tapers: FP64 GEP, or interpolated DPSS (no GEP)")
    ap.add_argument("--requests", type=int, default=4000, help="requests of the serving trace")
    ap.add_argument("--rate", type=float, default=2000.0, help="Poisson arrival rate of the serving trace (req/s)")
    ap.add_argument("--nsig", type=int, default=2048, help="signals of the uneven batch workload")
    ap.add_argument("--batch", type=int, default=32, help="signals per step per GPU")
    ap.add_argument("--precision", type=int, default=32, choices=[32, 64])
    ap.add_argument("--cpu-seconds", type=float, default=8.0, help="target wall time of the CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--chunk", type=int, default=0, help="signals per internal chunk (0 = the plan's choice)")
    ap.add_argument("--path", type=int, default=0, choices=[0, 1, 2, 3],
                    help="exec path: 0 automatic, 1 generic, 2 packed four-kernel, 3 packed persistent kernel")
    ap.add_argument("--sigma", type=float, default=0.0, help="oversampling factor (0 = the plan's choice)")
    ap.add_argument("--tune", action="store_true",
                    help="autotune the plan (oversampling, chunk, path) before the timed steps")
    ap.add_argument("--outputs", default="JEPL",
                    help="outputs written each step: any of J (eigencoefficients), E (eigenspectra), P (P-hat), "
                         "L (leakage estimates L-hat, E-hat), F (Thomson F-statistic)")
    ap.add_argument("--skip-gep", action="store_true",
                    help="plan from taper-shaped inputs instead of the FP64 GEP (profiling runs; "
                         "the exec kernels and their shapes are identical)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(rank: int) -> int:
    """Each rank draws its own signals (replicas: the units are partitioned, nothing is exchanged)."""
    return 1000 * rank


def job_time_ms(local_ms: float, world: int, device=None) -> float:
    """The job's time: the slowest rank's (max over ranks; one all-reduce of a scalar, outside the
    timed region)."""
    if world <= 1:
        return float(local_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step: float, steps: int, world: int, job_ms: float) -> float:
    """Whole-job aggregate: the units all ranks processed over the slowest rank's time."""
    return world * steps * units_per_rank_step / (job_ms * 1e-3)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.proc:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
            os.unlink(self.path)
        except Exception:
            pass
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def profiled_traffic(workload: str, kernel: str, nb: int):
    """DRAM bytes per launch of `kernel` from the committed ncu capture of this workload
    (profiles/exec_kernels_<workload>_traffic.json), scaled to nb signals per launch; None if there
    is no capture for this kernel/workload, it was taken at another chunk size, or the kernel
    sources changed since it was taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"exec_kernels_{workload}_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for rel, h in d["sources"].items():
            if hashlib.sha256(open(os.path.join(ROOT, rel), "rb").read()).hexdigest()[:16] != h:
                return None
        k = d["kernels"][kernel]
        if int(d["signals_per_launch"]) != nb:
            return None
        return float(k["dram_bytes_read_per_launch"]) + float(k["dram_bytes_write_per_launch"])
    except Exception:
        return None


def algorithmic_bytes(info, kernel: str, nb: int, csz: int, rsz: int, outputs: str = "JEP") -> float:
    """Compulsory bytes one launch of each exec kernel must move (per chunk of nb signals).

    spread : read x (N reals) + point records (cell int32, offset, source int32) + tapers (K x P),
             write the spread grid (K x rows*n2 complex)
    cols   : read the spread grid, write the column-FFT workspace (K x nf complex)
    rows   : write J (K x I complex), eigenspectra (K x I real), P-hat (I real) and read the
             deconvolution factors (I complex); its input is the L2-resident workspace
    """
    N, K, I = info["N"], info["K"], info["I"]
    grid = K * info["rows"] * info["n2"] * csz
    if kernel == "spread":
        per = N * rsz + grid
        shared = N * (8 + rsz) + K * N * (rsz if info["real_taper"] else csz)
        return nb * per + shared
    if kernel == "cols":
        return nb * (grid + K * info["nf"] * csz)
    if kernel == "rows":
        if info["path"] == 2:  # packed path: row FFTs only (L2-resident input and output)
            return nb * 2 * ((K + 1) // 2) * info["nf"] * csz
        per = I * rsz + (K * I * csz if "J" in outputs else 0) + (K * I * rsz if "E" in outputs else 0)
        return nb * per + I * csz
    if kernel == "epi":
        per = I * rsz + (K * I * csz if "J" in outputs else 0) + (K * I * rsz if "E" in outputs else 0)
        per += I * rsz if "F" in outputs else 0
        return nb * per + I * csz
    if kernel == "pipe":
        # the whole path in one launch over nb signals: read x, write J, |J|^2, P-hat; the plan's
        # point records, tapers and deconvolution factors once; the intermediates (spread grids,
        # column-FFT and row-FFT workspaces) are consumed from L2 and are not compulsory traffic
        per = N * rsz + I * rsz + (K * I * csz if "J" in outputs else 0) + (K * I * rsz if "E" in outputs else 0)
        shared = N * (8 + rsz) + K * N * rsz + I * csz
        return nb * per + shared
    raise KeyError(kernel)


def cpu_oracle_rate(wl, target_s: float, seed: int = 0):
    """Time the oracle's direct FP64 sum on a band subset of one signal."""
    from oracle import _native
    from oracle import estimator as oest
    from synth import taper_like  # taper-shaped rows; the direct sum costs the same for any taper
    w = taper_like(wl.K, wl.N, seed)
    rng = np.random.default_rng(seed)
    probe = np.sort(rng.choice(wl.I, size=256, replace=False)).astype(np.int64)
    t0 = time.perf_counter()
    oest.eigencoefficients(wl.t, wl.x[0], w, wl.f_lo, wl.df, wl.I, probe)
    dt = time.perf_counter() - t0
    nb = int(min(wl.I, max(256, 256 * target_s / max(dt, 1e-6))))
    idx = np.sort(rng.choice(wl.I, size=nb, replace=False)).astype(np.int64)
    t0 = time.perf_counter()
    oest.eigencoefficients(wl.t, wl.x[0], w, wl.f_lo, wl.df, wl.I, idx)
    dt = time.perf_counter() - t0
    units = wl.K * wl.N * nb
    return units / dt, nb, dt, _native.num_threads()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import synth
    wl = synth.workload(args.workload, batch=1, seed=0)
    from oracle import _native
    from oracle import estimator as oest
    from synth import taper_like
    w = taper_like(wl.K, wl.N, 0)
    # bounded sample per step so that warmup + steps stay within a few minutes
    rate, nb, dt, cores = cpu_oracle_rate(wl, min(args.cpu_seconds, 4.0))
    per_step_s = max(0.5, min(6.0, 150.0 / max(1, args.steps + args.warmup)))
    nb_step = int(min(wl.I, max(64, rate * per_step_s / (wl.K * wl.N))))
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(wl.I, size=nb_step, replace=False)).astype(np.int64)
    for _ in range(args.warmup):
        oest.eigencoefficients(wl.t, wl.x[0], w, wl.f_lo, wl.df, wl.I, idx[: max(64, nb_step // 8)])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oest.eigencoefficients(wl.t, wl.x[0], w, wl.f_lo, wl.df, wl.I, idx)
    total = time.perf_counter() - t0
    units = args.steps * wl.K * wl.N * nb_step
    value = units / total
    sample = (f"{args.workload}: one signal, {nb_step} of {wl.I} band centres per step "
              f"(direct FP64 sum, {cores} threads)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "bands_per_step": nb_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_uneven(args):
    """Uneven batch (2048 signals by default): nsig signals with their own sampling patterns (grid length
    log-uniform in [1024, 16384], Markov gaps, K in {4,6,8}, I = 4G) through m2nufft_exec_batch
    (one cached CUDA graph per call) against the plain per-signal path (one m2nufft_exec per
    signal on one stream).  Plans use taper-shaped inputs instead of 2048 dense GEPs; the exec
    kernels and their shapes are the same."""
    import torch

    import paper_2407_01943_gb300 as pkg
    import synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    ws = synth.batched_uneven(args.nsig, seed=rank)
    t_plan = time.perf_counter()
    plans, xs, Js, Es, Ps = [], [], [], [], []
    units = 0
    for s_, wl in enumerate(ws):
        p = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32, device=local, max_batch=1,
                     tapers=synth.taper_like(wl.K, wl.N, s_), lam=np.linspace(0.999, 0.99, wl.K))
        plans.append(p)
        xs.append(torch.from_numpy(wl.x[0].astype(np.float32)).to(dev))
        Js.append(torch.empty((wl.K, wl.I), dtype=torch.complex64, device=dev))
        Es.append(torch.empty((wl.K, wl.I), dtype=torch.float32, device=dev))
        Ps.append(torch.empty((wl.I,), dtype=torch.float32, device=dev))
        units += wl.K * wl.N * wl.I
    t_plan = time.perf_counter() - t_plan
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def flush_l2():
        flush.fill_(1)
        flush.view(torch.int32).max()

    def timed(fn):
        for _ in range(args.warmup):
            flush_l2()
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for s_ in range(args.steps):
            flush_l2()
            evs[s_][0].record(stream)
            fn()
            evs[s_][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / args.steps

    all_packed = all(p.info["path"] >= 2 for p in plans)

    def coset_len(n1):
        f = 1
        while f < 32 and n1 % (2 * f) == 0:
            f *= 2
        return f
    kp_classes = {0 if (p.info["K"] + 1) // 2 <= 2 else (1 if (p.info["K"] + 1) // 2 <= 4 else 2) for p in plans}
    hb_launches = len(kp_classes) + len({coset_len(p.info["n1"]) for p in plans}) + 2
    t0 = time.perf_counter()
    pkg.exec_batch(plans, xs, Js, Es, Ps, stream=stream)  # first call: build + capture + instantiate
    torch.cuda.synchronize()
    t_capture = time.perf_counter() - t0
    ms_batch = timed(lambda: pkg.exec_batch(plans, xs, Js, Es, Ps, stream=stream))
    # the same batch as one persistent pipelined kernel (batch mode 1), for comparison
    stage_split, ms_pipe = None, None
    if all_packed:
        prev = pkg.binding.set_batch_mode(1)
        pkg.exec_batch(plans, xs, Js, Es, Ps, stream=stream)
        torch.cuda.synchronize()
        pkg.binding.batch_pipe_profile()  # reset the stage accounting
        ms_pipe = timed(lambda: pkg.exec_batch(plans, xs, Js, Es, Ps, stream=stream))
        pkg.binding.set_batch_mode(prev)
        busy, waitms, nitems = pkg.binding.batch_pipe_profile()
        tot = max(float(busy.sum()), 1e-12)
        stage_split = {n: {"items": int(nitems[i]), "busy_ms_sum": float(busy[i]), "share": float(busy[i] / tot),
                           "avg_item_us": float(1e3 * busy[i] / max(nitems[i], 1)), "wait_ms_sum": float(waitms[i])}
                       for i, n in enumerate(["spread", "cols", "rows", "epi"])}

    def plain():
        for p, x, J, E, P in zip(plans, xs, Js, Es, Ps):
            p.exec(x[None, :], J[None], E[None], P[None], stream=stream)

    wall0 = time.perf_counter()
    ms_plain = timed(plain)
    wall_plain = time.perf_counter() - wall0
    line = {
        "metric": METRIC, "value": units / (ms_batch * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_batch, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"uneven batch: {args.nsig} signals, grid length log-uniform in [1024, 16384], "
                               f"Markov gaps 15%, K in {{4,6,8}}, I = 4G; m2nufft_exec_batch (one CUDA graph: "
                               f"one launch per stage over all signals)",
                   "signals": args.nsig, "units_per_step": units,
                   "l2": "flushed between timed steps (512 MiB write + read-back)"},
        "plain_per_signal": {"value": units / (ms_plain * 1e-3), "ms_per_step": ms_plain,
                             "host_wall_s": wall_plain},
        "batch_over_plain": ms_plain / ms_batch,
        "persistent_kernel": None if ms_pipe is None else {
            "value": units / (ms_pipe * 1e-3), "ms_per_step": ms_pipe, "gpu_launches": 1, "stages": stage_split},
        "gpu_launches": hb_launches if all_packed else 4 * args.nsig,
        "plain_gpu_launches_per_step": sum(1 if p.info["path"] == 3 else (4 if p.info["path"] == 2 else 3)
                                           for p in plans),
        "plan_seconds": t_plan, "capture_seconds": t_capture,
    }
    print(json.dumps(line), flush=True)
    for p in plans:
        p.close()
    return 0


def run_multiband(args):
    """Multiband partition (Sec. 3): Q = 4 sub-bands [0, 1/8), [1/8, 1/4), [1/4, 3/8), [3/8, 1/2] of a
    jittered pattern (N = 4096, +-0.4), nominal centres at the sub-band middles, f_w = 5/N, K = 6,
    2^14 band centres per sub-band on [f_min + f_w, f_max - f_w); one complex Hermitian GEP per
    sub-band on the GPU; B signals (AR(4)) per step run as one m2nufft_exec_batch over the B x Q
    (signal, sub-band) pairs, against per-pair m2nufft_exec."""
    import torch

    import paper_2407_01943_gb300 as pkg
    import synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()
    N, K, Iq, Q, B = 4096, 6, 1 << 14, 4, min(args.batch, 8)
    fw = 5.0 / N
    t = synth.jittered(N, 0.4, 77 + rank_seed(rank))
    idx = np.arange(N)
    poles = [0.95 * np.exp(1j * a) for a in (0.1 * np.pi, -0.1 * np.pi, 0.3 * np.pi, -0.3 * np.pi)]
    X = np.stack([synth.ar_process(idx, poles, 5000 + rank_seed(rank) + b) for b in range(B)])
    edges = [0.0, 0.125, 0.25, 0.375, 0.5]
    t0 = time.perf_counter()
    plans = []
    for q in range(Q):
        a, b = edges[q], edges[q + 1]
        f_c0 = 0.5 * (a + b)
        lo, hi = a + fw, b - fw
        plans.append(pkg.Plan(t, 1.0, fw, K, lo, (hi - lo) / Iq, Iq, precision=32, device=local,
                              subband=(f_c0, a, b)))
    t_plan = time.perf_counter() - t0
    xs = [torch.from_numpy(X[b].astype(np.float32)).to(dev) for b in range(B)]
    Ps = [torch.empty((Iq,), dtype=torch.float32, device=dev) for _ in range(B * Q)]
    Js = [torch.empty((K, Iq), dtype=torch.complex64, device=dev) for _ in range(B * Q)]
    bp = [plans[q] for b in range(B) for q in range(Q)]
    bx = [xs[b] for b in range(B) for q in range(Q)]
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def flush_l2():
        flush.fill_(1)
        flush.view(torch.int32).max()

    def timed(fn):
        for _ in range(args.warmup):
            flush_l2()
            fn()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for s_ in range(args.steps):
            flush_l2()
            evs[s_][0].record(stream)
            fn()
            evs[s_][1].record(stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in evs) / args.steps

    ms_batch = timed(lambda: pkg.exec_batch(bp, bx, Js, None, Ps, stream=stream))

    def plain():
        for p, x, J, P in zip(bp, bx, Js, Ps):
            p.exec(x[None, :], J[None], None, P[None], stream=stream)
    ms_plain = timed(plain)
    units = B * Q * K * N * Iq
    line = {
        "metric": METRIC, "value": units / (ms_batch * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_batch, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"multiband: Q = {Q} sub-bands of [0, 1/2], N = {N} jittered, K = {K}, f_w = 5/N, "
                               f"{Iq} band centres per sub-band, B = {B} signals; complex tapers (generic path)",
                   "units_per_step": units, "l2": "flushed between timed steps (512 MiB write + read-back)"},
        "plain_per_pair": {"value": units / (ms_plain * 1e-3), "ms_per_step": ms_plain},
        "batch_over_plain": ms_plain / ms_batch,
        "plan_seconds": t_plan, "gep_seconds_per_subband": [p.info["gep_seconds"] for p in plans],
        "gpu_launches": 3 * B * Q,
    }
    print(json.dumps(line), flush=True)
    for p in plans:
        p.close()
    return 0


def run_subopt(args):
    """Suboptimality at the paper's scale (Sec. 4: N = 50 samples): the estimate E-hat (App. B) that
    every plan carries, against the true E_i from per-band GEPs (Eq. subopt_measure), on the paper's
    arithmetic-sampling scheme E1 stand-in (jittered N = 50) and a 1.2 Hz rate mismatch grid."""
    import torch

    import paper_2407_01943_gb300 as pkg
    import synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pkg.build()
    out = {}
    for name, t in (("jittered N=50", synth.jittered(50, 0.4, 3)), ("rate 1.2, N=50", np.arange(50) / 1.2)):
        K, fw, I = 3, 2.5 / 50, 1024
        t0 = time.perf_counter()
        plan = pkg.Plan(t, 1.0, fw, K, -0.45, 0.9 / I, I, precision=64, device=local)
        t_plan = time.perf_counter() - t0
        t0 = time.perf_counter()
        E, _ = plan.true_suboptimality()
        t_true = time.perf_counter() - t0
        _, Eh = plan.leakage()
        out[name] = {"plan_seconds": t_plan, "true_E_seconds": t_true, "bands": I,
                     "max_true_E": float(E.max()), "max_E_hat": float(Eh.max()),
                     "max_abs_diff": float(np.abs(E - Eh).max()),
                     "corr": float(np.corrcoef(E, Eh)[0, 1]) if E.std() > 0 and Eh.std() > 0 else None}
        plan.close()
    print(json.dumps({"workload": "subopt", "results": out}), flush=True)
    return 0


def run_serve(args):
    """Serving: Poisson arrivals of PSD requests over 64 fixed sampling patterns
    (grid length uniform in [2048, 16384], jittered or Bernoulli-missing 10-30%, K = 8, I = 4G),
    plans cached before the trace, 40 GB device-memory budget; continuous batching (4 slots,
    up to 16 requests per launch) against the plain per-request path.  The 64 plans take their
    tapers from interpolated DPSS (Table 1 step 3 a-c: no GEP), built before the trace."""
    import torch

    import paper_2407_01943_gb300 as pkg
    import synth
    from paper_2407_01943_gb300 import serve
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pkg.build()
    pats = synth.serving_patterns(64, seed=rank)
    t_plan = time.perf_counter()
    plans = {i: pkg.Plan(pt["t"], 1.0, pt["f_w"], pt["K"], pt["f_lo"], pt["df"], pt["I"], precision=32,
                         device=local, max_batch=16, taper_design="spline")
             for i, pt in enumerate(pats)}
    t_plan = time.perf_counter() - t_plan

    def trace(n, rate, seed):
        arr = synth.poisson_arrivals(rate, n, seed) if rate > 0 else np.zeros(n)
        rng = np.random.default_rng(seed + 1)
        out = []
        for k, a in enumerate(arr):
            pid = int(rng.integers(0, len(pats)))
            out.append(serve.Request(k, pid, rng.standard_normal(pats[pid]["t"].shape[0]).astype(np.float32),
                                     float(a)))
        return out

    budget = 40 << 30
    srv = serve.PSDServer(plans, mem_budget=budget, slots=4, max_batch=16, device=local)
    srv.serve(trace(200, 0, 99))                               # warm-up (allocator, pinned pools)
    loaded = srv.serve(trace(args.requests, args.rate, 1))
    plain = srv.serve_plain(trace(args.requests, args.rate, 1))
    sat = srv.serve(trace(args.requests, 0, 2))               # all requests at t = 0
    sat_plain = srv.serve_plain(trace(args.requests, 0, 2))
    line = {
        "metric": METRIC, "value": sat["throughput_units_per_s"], "unit": UNIT, "n_gpus": world, "steps": 1,
        "warmup": 1, "ms_per_step": sat["wall_s"] * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"serving: 64 cached patterns, G uniform in [2048, 16384], K = 8, I = 4G; "
                               f"{args.requests} requests; continuous batching, 4 slots, <= 16 per launch, "
                               f"40 GB budget", "rate_req_per_s": args.rate},
        "served_at_rate": loaded, "plain_at_rate": plain,
        "served_saturated": sat, "plain_saturated": sat_plain,
        "plan_seconds": t_plan,
    }
    print(json.dumps(line), flush=True)
    srv.close()
    for p in plans.values():
        p.close()
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2407_01943_gb300 as pkg
    import synth

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.build()

    B = args.batch
    wl = synth.workload(args.workload, batch=B, seed=rank_seed(rank))
    rdt = torch.float32 if args.precision == 32 else torch.float64
    cdt = torch.complex64 if args.precision == 32 else torch.complex128
    csz, rsz = (8, 4) if args.precision == 32 else (16, 8)

    t_plan = time.perf_counter()
    if args.skip_gep:
        # taper-shaped rows and placeholder eigenvalues: the exec kernels and their shapes are the same
        plan = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=args.precision, device=local,
                        tapers=synth.taper_like(wl.K, wl.N, 0), lam=np.linspace(0.999, 0.99, wl.K),
                        max_batch=args.chunk, path=args.path, sigma=args.sigma, tune=args.tune)
    else:
        plan = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=args.precision, device=local,
                        max_batch=args.chunk, path=args.path, taper_design=args.taper_design, sigma=args.sigma,
                        tune=args.tune)
    t_plan = time.perf_counter() - t_plan
    info = plan.info

    x = torch.from_numpy(wl.x.astype(np.float32 if args.precision == 32 else np.float64)).to(dev)
    J = torch.empty((B, wl.K, wl.I), dtype=cdt, device=dev) if "J" in args.outputs else None
    E = torch.empty((B, wl.K, wl.I), dtype=rdt, device=dev) if "E" in args.outputs else None
    P = torch.empty((B, wl.I), dtype=rdt, device=dev)
    # leakage estimates (plan constants, App. B) are handed out with every exec
    Lh = torch.empty((wl.K, wl.I), dtype=torch.float64, device=dev) if "L" in args.outputs else None
    Eh = torch.empty((wl.I,), dtype=torch.float64, device=dev) if "L" in args.outputs else None
    # Thomson F-statistic per band (Sec. 3, Eq. f_stat), optional output
    Fb = torch.empty((B, wl.I), dtype=rdt, device=dev) if "F" in args.outputs else None

    def step(xin, Pout=None):
        Pout = P if Pout is None else Pout
        if Fb is None:
            plan.exec(xin, J, E, Pout, Lh, Eh, stream=stream)
        else:
            plan.exec(xin, J, E, Pout, stream=stream, F=Fb)
            if Lh is not None:
                plan.exec(xin[:0], None, None, None, Lh, Eh, stream=stream)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    def flush_l2():
        # write a buffer 4x the L2, then read it back so no dirty lines are left to drain
        # into the timed step
        flush.fill_(1)
        flush.view(torch.int32).max()
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        flush_l2()
        step(x)
    torch.cuda.synchronize()

    # ---- timed region: K device-timed steps, L2 flushed between them ----
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    # per-kernel events serialise a packed exec's chunks (no overlap between chunks while
    # instrumented), so with more than one chunk the kernel breakdown comes from a separate pass
    chunks = -(-B // info["chunk"])
    separate_kernel_pass = info["path"] == 2 and chunks >= 2
    plan.get_timing()
    plan.set_timing(not separate_kernel_pass)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for s in range(args.steps):
        flush_l2()
        evs[s][0].record(stream)
        step(x)
        evs[s][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    if separate_kernel_pass:
        plan.set_timing(True)
        for _ in range(min(args.steps, 5)):
            flush_l2()
            step(x)
        torch.cuda.synchronize()
    plan.set_timing(False)
    kms, klaunch = plan.get_timing()
    stage_split = None
    if info["path"] == 3:
        busy, waitms, nitems = plan.get_pipe_profile()
        tot = max(float(busy.sum()), 1e-12)
        stage_split = {n: {"items": int(nitems[i]), "busy_ms_sum": float(busy[i]), "share": float(busy[i] / tot),
                           "avg_item_us": float(1e3 * busy[i] / max(nitems[i], 1)), "wait_ms_sum": float(waitms[i])}
                       for i, n in enumerate(["spread", "cols", "rows", "epi"])}
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = job_time_ms(float(sum(step_ms)), world, dev)
    units_per_signal = wl.K * wl.N * wl.I
    value = job_throughput(B * units_per_signal, args.steps, world, total_ms)
    pipelined = info["path"] == 3
    per_step = chunks * (4 if info["path"] == 2 else 3)
    kp = (wl.K + 1) // 2
    # execs of several chunks spread all their signals in one launch (grids up to 256 MiB)
    hoisted = info["path"] == 2 and chunks > 1 and B * kp * info["rows"] * 1024 * 8 <= (256 << 20)
    if hoisted:
        per_step = 1 + 3 * chunks  # one spread launch for all signals, then three kernels per chunk
    launches = args.steps * (1 if pipelined else per_step)
    per_launch = B if pipelined else min(B, info["chunk"])

    # ---- per-kernel roofline from the live event timing ----
    names = ["pipe", "", "", ""] if pipelined else ["spread", "cols", "rows", "epi"]
    hbm_peak, peak_kind = measured_peaks()
    kern = {}
    for i, n in enumerate(names):
        if klaunch[i] == 0:
            continue
        avg_ms = kms[i] / klaunch[i]
        byts = algorithmic_bytes(info, n, B if (hoisted and n == "spread") else per_launch, csz, rsz, args.outputs)
        kern[n] = {"launches": int(klaunch[i]), "total_ms": float(kms[i]), "avg_us": 1e3 * avg_ms,
                   "alg_bytes_per_launch": byts, "gbs": byts / (avg_ms * 1e-3) / 1e9,
                   "frac_of_hbm_peak": byts / (avg_ms * 1e-3) / 1e9 / hbm_peak,
                   # where the algorithmic bytes live: the FFT intermediates stay in L2, so their
                   # fraction is an L2 rate measured against the HBM peak, not HBM efficiency
                   "alg_bytes_in": {"spread": "HBM (samples, point records, tapers) and L2 (grids)",
                                    "cols": "L2", "rows": "L2", "epi": "HBM", "pipe": "HBM"}.get(n, "HBM"),
                   "share": float(kms[i] / max(sum(kms), 1e-12))}
    dom = max(kern, key=lambda n: kern[n]["total_ms"]) if kern else None
    roofline = None
    if dom:
        achieved = kern[dom]["gbs"]
        roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                    "alg_bytes_per_launch": kern[dom]["alg_bytes_per_launch"],
                    "traffic": profiled_traffic(args.workload, dom, per_launch)}

    # ---- end to end through the public API with host buffers ----
    # Every step copies its x from pinned host memory and reads its P-hat back to pinned host
    # memory.  Steps are double-buffered the way a streaming caller would run them: step s+1's
    # input is copied in on one copy stream and step s's P-hat read back on another while step s
    # computes (the execs themselves stay ordered on one stream, as a plan requires).
    e2e = None
    if not args.no_e2e:
        xh = torch.from_numpy(wl.x.astype(np.float32 if args.precision == 32 else np.float64)).pin_memory()
        ph = [torch.empty((B, wl.I), dtype=rdt).pin_memory() for _ in range(2)]
        xd = [torch.empty_like(x) for _ in range(2)]
        Pd = [P, torch.empty_like(P)]
        cstream = torch.cuda.Stream(device=dev)  # device -> host
        hstream = torch.cuda.Stream(device=dev)  # host -> device
        out_bytes = B * wl.I * rsz + (B * wl.K * wl.I * csz if J is not None else 0) + \
            (B * wl.K * wl.I * rsz if E is not None else 0)
        d2h_done = [torch.cuda.Event() for _ in range(2)]
        h2d_done = [torch.cuda.Event() for _ in range(2)]
        step_done = [torch.cuda.Event() for _ in range(2)]

        def e2e_steps(n):
            go = torch.cuda.Event()  # the first input's copy starts when the compute stream gets here
            go.record(stream)
            hstream.wait_event(go)
            with torch.cuda.stream(hstream):
                xd[0].copy_(xh, non_blocking=True)
                h2d_done[0].record(hstream)
            for s_ in range(n):
                b = s_ % 2
                stream.wait_event(h2d_done[b])  # this step's x is in
                stream.wait_event(d2h_done[b])  # P-hat buffer b was read back two steps ago
                step(xd[b], Pd[b])
                step_done[b].record(stream)
                cstream.wait_event(step_done[b])
                with torch.cuda.stream(cstream):
                    ph[b].copy_(Pd[b], non_blocking=True)
                    d2h_done[b].record(cstream)
                if s_ + 1 < n:
                    nb_ = (s_ + 1) % 2
                    if s_ >= 1:
                        hstream.wait_event(step_done[nb_])  # step s-1 is done with x buffer nb_
                    with torch.cuda.stream(hstream):
                        xd[nb_].copy_(xh, non_blocking=True)
                        h2d_done[nb_].record(hstream)
            stream.wait_stream(cstream)

        for ev in d2h_done:
            ev.record(stream)
        e2e_steps(2)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_steps(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = job_time_ms(float(e0.elapsed_time(e1)), world, dev)
        e2e = {"value": job_throughput(B * units_per_signal, args.steps, world, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(xh.numel() * xh.element_size()),
               "d2h_bytes_per_step": int(ph[0].numel() * ph[0].element_size()),
               "ms_per_step": e2e_ms / args.steps,
               "overlap": "double-buffered: step s+1's x copy-in and step s's P-hat read-back overlap the execs of step s",
               "l2": f"not flushed between steps: each step writes {out_bytes / 1e9:.2f} GB of outputs "
                     f"({out_bytes / 129e6:.1f}x the 129 MB L2)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, nb, dt, cores = cpu_oracle_rate(wl, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.workload}: one signal, {nb} of {wl.I} band centres, direct FP64 sum, "
                         f"{dt:.1f} s wall"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == 32 else "f64",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: N={wl.N} samples ({'jittered' if 'jitter' in args.workload else 'grid'}), "
                                   f"K={wl.K}, f_w={wl.f_w:.3g}, I={wl.I}, B={B} signals per GPU per step",
                       "signals_per_gpu_per_step": B, "N": wl.N, "K": wl.K, "I": wl.I, "nf": info["nf"],
                       "outputs": args.outputs,
                       "kernel_width": info["width"], "chunk": info["chunk"], "exec_path": info["path"],
                       "autotune": ([{"path": r[0], "sigma": r[1], "max_batch": r[2], "ms": r[3]}
                                     for r in plan.tuning()] if args.tune else None),
                       "kernel_timing": ("separate instrumented pass (one spread launch for all signals, then the "
                                         "chunks one after the other); the timed steps overlap consecutive "
                                         "chunks on two streams"
                                         if separate_kernel_pass else "instrumented timed steps"),
                       "l2": "flushed between timed steps (512 MiB write + read-back)", "parallelism": f"replicas x{world}"},
            "gpu_launches": launches,
            "roofline": roofline,
            "kernels": kern,
            "pipe_stages": stage_split,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk,
            "plan_seconds": t_plan,
            "gep_seconds": info["gep_seconds"],
            "taper_design": "taper-shaped inputs" if args.skip_gep else args.taper_design,
            "wall_seconds_timed": wall,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "uneven":
        return run_uneven(args)
    if args.workload == "multiband":
        return run_multiband(args)
    if args.workload == "subopt":
        return run_subopt(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
