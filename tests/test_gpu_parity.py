"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

J_k(A_i) and P-hat are compared element by element at every compared band
(Eq. eigencoefficients / Eq. power_spectrum_estimator): the NuFFT's
per-output bound |dJ_k| <= tol * sum_n |w_k x| and the bounds it implies for
|J_k|^2 and P-hat (tests/_util.py), beside the relative l2 over the array;
tol = 1e-5 for the FP32 path and 1e-10 for the FP64 path.  The full-size
cases compare sampled bands plus the packed path's special positions (both
ends of the band grid, the first and last in-band FFT columns at every row,
row 0's partner columns).  Where the oracle's dense GEP
is cheap, the tapers come from the oracle and are handed to the GPU plan
(m2nufft_plan_with_tapers), so J is compared with identical tapers; the
GPU's own GEP is checked separately (eigenvalues, subspace, residuals) and
through P-hat, which depends only on the span of the tapers.
"""
import numpy as np
import pytest

import synth
from oracle import estimator as oest
from oracle import gpss as ogpss
from oracle import leakage as oleak
from tests._util import TOL, assert_elementwise, packed_edge_bands, rel_l2, sample_bands, seeded_tapers, source_l1

torch = pytest.importorskip("torch")
pkg = pytest.importorskip("paper_2407_01943_gb300")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    d = torch.device("cuda:0")
    torch.cuda.set_device(d)
    return d


def run_plan(plan, x, dev, want=("J", "E", "P")):
    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32 if plan.precision == 32 else np.float64)).to(dev)
    out = plan.run(xt, want=want)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def oracle_all(t, X, w, f_lo, df, I, idx=None):
    Js, Ps = [], []
    for b in range(X.shape[0]):
        J, E, P = oest.m2nufft(t, X[b], w, f_lo, df, I, idx)
        Js.append(J)
        Ps.append(P)
    return np.stack(Js), np.stack(Ps)


_ORACLE_CACHE = {}


def oracle_cached(key, t, X, w, f_lo, df, I, idx):
    """oracle_all for a full-size workload, computed once per module for the same inputs (key names
    the workload, its signals and tapers; idx is part of the key)."""
    k = (key, I, idx.tobytes())
    if k not in _ORACLE_CACHE:
        _ORACLE_CACHE[k] = oracle_all(t, X, w, f_lo, df, I, idx)
    return _ORACLE_CACHE[k]


def full_size_bands(I, n1, n, seed):
    """Sampled bands plus the packed path's special positions for its n1 (test infrastructure)."""
    return np.union1d(sample_bands(I, n, seed), packed_edge_bands(I, n1))


def check(out, Jr, Pr, w, X, prec, idx=None, with_E=True):
    """Relative l2 over the compared array and the element-wise bound at every compared band for J,
    P-hat and (when present) the eigenspectra; returns the worst ratio to the bound per output."""
    sel = (lambda a: a) if idx is None else (lambda a: a[..., idx])
    Jg, Pg = sel(out["J"]), sel(out["P"])
    Eg = sel(out["E"]) if with_E and "E" in out else None
    assert rel_l2(Jg, Jr) <= TOL[prec]
    assert rel_l2(Pg, Pr) <= TOL[prec]
    if Eg is not None:
        assert rel_l2(Eg, np.abs(Jr) ** 2) <= TOL[prec]
    return assert_elementwise(Jg, Jr, source_l1(w, X), TOL[prec], Pg, Pr, Eg)


# ---------------------------------------------------------------------------
# full-array parity at oracle-friendly sizes
# ---------------------------------------------------------------------------
PATHS = [(64, 1), (32, 1), (32, 2), (32, 3)]  # (precision, exec path): generic FP64 / generic FP32 /
# packed FP32 as four kernels / packed FP32 as one persistent pipelined kernel


@pytest.mark.parametrize("prec,path", PATHS)
def test_grid1024_full_parity(dev, prec, path):
    """N=1024 grid with 20% Bernoulli missing, 3 tones + noise, K=6, I=1024."""
    wl = synth.workload("grid1024", batch=3)
    w, lam = ogpss.nominal_tapers(wl.t, wl.fs, wl.f_w, wl.K)
    plan = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=prec, tapers=w, lam=lam,
                    path=path)
    assert plan.info["path"] == path
    out = run_plan(plan, wl.x, dev)
    Jr, Pr = oracle_all(wl.t, wl.x, w, wl.f_lo, wl.df, wl.I)
    check(out, Jr, Pr, w, wl.x, prec)
    assert plan.info["wrap"] == 1  # span ~ period: wrap-around spreading


@pytest.mark.parametrize("prec,path", PATHS)
def test_jittered_medium_full_parity(dev, prec, path):
    """Jittered N=2048 (+-0.4), AR(4)-like tones, K=8, I=2^14: zero-padded
    grid (support 1/8 of the period) spanning many tiles and FFT rows."""
    t = synth.jittered(2048, 0.4, 21)
    X = np.stack([synth.tones(t, (0.1, 0.31), (2.0, 1.0), 1.0, 30 + b) for b in range(2)])
    K, fw, I = 8, 5.0 / 2048, 1 << 14
    w, lam = ogpss.nominal_tapers(t, 1.0, fw, K)
    plan = pkg.Plan(t, 1.0, fw, K, -0.5, 1.0 / I, I, precision=prec, tapers=w, lam=lam, path=path)
    out = run_plan(plan, X, dev)
    Jr, Pr = oracle_all(t, X, w, -0.5, 1.0 / I, I)
    assert plan.info["wrap"] == 0 and plan.info["rows"] < plan.info["n1"]
    check(out, Jr, Pr, w, X, prec)


@pytest.mark.parametrize("prec", [64, 32])
def test_general_band_grid_complex_taper(dev, prec):
    """Band grid not centred on 0 (f_lo = 0.013, df = 0.37/1000, I = 1000, odd
    offsets): the modulated taper is complex; large time offset 1e5."""
    t = 1.0e5 + synth.jittered(700, 0.3, 4)
    x = synth.tones(t, (0.05, 0.2), (1.0, 1.0), 0.5, 5)[None, :]
    K, fw = 4, 4.0 / 700
    w, lam = ogpss.nominal_tapers(t, 1.0, fw, K)
    f_lo, df, I = 0.013, 0.37 / 1000, 1000
    plan = pkg.Plan(t, 1.0, fw, K, f_lo, df, I, precision=prec, tapers=w, lam=lam)
    assert plan.info["real_taper"] == 0
    out = run_plan(plan, x, dev)
    Jr, Pr = oracle_all(t, x, w, f_lo, df, I)
    check(out, Jr, Pr, w, x, prec)


@pytest.mark.parametrize("I", [1, 2, 7, 63, 65, 1023])
def test_small_and_odd_band_counts(dev, I):
    """Degenerate and ragged grids: I = 1, 2, odd, just below/above a power of two."""
    t = synth.jittered(90, 0.4, 8)
    x = synth.white(t, 1.0, 9)[None, :]
    w = seeded_tapers(3, 90, 1)
    plan = pkg.Plan(t, 1.0, 0.03, 3, -0.45, 0.9 / max(I, 1), I, precision=64, tapers=w)
    out = run_plan(plan, x, dev)
    Jr, Pr = oracle_all(t, x, w, -0.45, 0.9 / max(I, 1), I)
    check(out, Jr, Pr, w, x, 64)


def test_single_sample_single_taper(dev):
    """N = 1, K = 1: J(f) = w x exp(-i 2 pi f t) exactly."""
    t = np.array([3.25])
    plan = pkg.Plan(t, 1.0, 0.1, 1, -0.5, 1.0 / 64, 64, precision=64, tapers=np.array([[0.7]]))
    out = run_plan(plan, np.array([[2.0]]), dev)
    f = -0.5 + np.arange(64) / 64
    np.testing.assert_allclose(out["J"][0, 0], 1.4 * np.exp(-2j * np.pi * f * 3.25), rtol=1e-11, atol=1e-12)


def test_many_chunks_and_empty_batch(dev):
    """B larger than the internal chunk (max_batch=2, B=5) gives the same
    result per signal; B = 0 is a no-op."""
    t = synth.jittered(300, 0.4, 3)
    X = np.stack([synth.white(t, 1.0, 40 + b) for b in range(5)])
    w = seeded_tapers(4, 300, 2)
    plan = pkg.Plan(t, 1.0, 0.02, 4, -0.5, 1 / 512, 512, precision=64, tapers=w, max_batch=2)
    assert plan.info["chunk"] == 2
    out = run_plan(plan, X, dev)
    Jr, Pr = oracle_all(t, X, w, -0.5, 1 / 512, 512)
    check(out, Jr, Pr, w, X, 64)
    xe = torch.zeros((0, 300), dtype=torch.float64, device=dev)
    plan.run(xe)
    torch.cuda.synchronize()


@pytest.mark.parametrize("path", [1, 2, 3])
def test_batch_equals_alone_bitwise(dev, path):
    """Deterministic kernels: a signal gives bit-identical J and P-hat alone
    and inside a batch (no atomics, fixed summation order)."""
    t = synth.jittered(1500, 0.4, 13)
    X = np.stack([synth.white(t, 1.0, 60 + b) for b in range(4)])
    w = seeded_tapers(6, 1500, 3)
    plan = pkg.Plan(t, 1.0, 0.004, 6, -0.5, 1 / 8192, 8192, precision=32, tapers=w, path=path)
    allb = run_plan(plan, X, dev)
    one = run_plan(plan, X[2:3], dev)
    assert np.array_equal(allb["J"][2], one["J"][0])
    assert np.array_equal(allb["P"][2], one["P"][0])


@pytest.mark.parametrize("K,I,N", [(1, 1024, 400), (5, 1024, 700), (3, 2048, 900), (7, 4096, 1500),
                                   (2, 3000, 1000), (9, 20000, 4000), (4, 1024, 8000), (6, 2048, 20000)])
def test_packed_path_edge_cases(dev, K, I, N):
    """Packed FP32 path: odd K (last pair half empty), K = 1, the smallest row
    counts n1 = 2, 4, 8 (self-paired rows 0 and n1/2), wrap-around (span
    longer than the period), I not a power of two, and many more samples than
    bands (N = 8 I, 10 I: the support wraps many times, ~30 spreading-matrix
    entries per cell, tiles whose samples span the whole signal and are read
    from global memory instead of staged); against the oracle and against the
    generic FP32 path."""
    t = synth.jittered(N, 0.4, K + N)
    X = np.stack([synth.white(t, 1.0, 70 + b) for b in range(3)])
    w = seeded_tapers(K, N, K)
    p2 = pkg.Plan(t, 1.0, 2.0 / N, K, -0.5, 1.0 / I, I, precision=32, tapers=w, path=2, max_batch=2)
    p1 = pkg.Plan(t, 1.0, 2.0 / N, K, -0.5, 1.0 / I, I, precision=32, tapers=w, path=1)
    o2 = run_plan(p2, X, dev)
    o1 = run_plan(p1, X, dev)
    # the persistent kernel runs the same stage code: bit-identical to the four kernels, with a
    # two-slot ring (stages of a signal back to back) and with the default seven-slot ring
    for mb in (2, 0):
        p3 = pkg.Plan(t, 1.0, 2.0 / N, K, -0.5, 1.0 / I, I, precision=32, tapers=w, path=3, max_batch=mb)
        o3 = run_plan(p3, X, dev)
        for k in ("J", "E", "P"):
            assert np.array_equal(o3[k], o2[k]), (mb, k)
    Jr, Pr = oracle_all(t, X, w, -0.5, 1.0 / I, I)
    check(o2, Jr, Pr, w, X, 32)
    check(o1, Jr, Pr, w, X, 32)
    assert rel_l2(o2["P"], o1["P"]) <= TOL[32]


def test_packed_path_rejects_complex_taper(dev):
    t = synth.jittered(300, 0.4, 1)
    with pytest.raises(pkg.M2Error) as e:
        pkg.Plan(t, 1.0, 0.01, 2, 0.01, 1 / 1024, 1024, precision=32, tapers=seeded_tapers(2, 300, 0), path=2)
    assert e.value.status == 1
    with pytest.raises(pkg.M2Error):
        pkg.Plan(t, 1.0, 0.01, 2, -0.5, 1 / 1024, 1024, precision=64, tapers=seeded_tapers(2, 300, 0), path=2)


# ---------------------------------------------------------------------------
# the GPU GEP (cuSOLVER FP64) against LAPACK
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["grid", "jitter"])
def test_gep_matches_lapack(dev, kind):
    if kind == "grid":
        wl = synth.workload("grid1024")
        t, fw, K, x = wl.t, wl.f_w, wl.K, wl.x
    else:
        t = synth.jittered(1200, 0.4, 17)
        fw, K = 5.0 / 1200, 8
        x = synth.tones(t, (0.2,), (1.0,), 1.0, 3)[None, :]
    plan = pkg.Plan(t, 1.0, fw, K, -0.5, 1 / 2048, 2048, precision=64)
    wg, lg = plan.tapers()
    wo, lo = ogpss.nominal_tapers(t, 1.0, fw, K)
    np.testing.assert_allclose(lg, lo, atol=1e-12)
    RB = ogpss.gpss_matrix_b(t, 0.5)
    RA = ogpss.gpss_matrix_a(t, fw)
    np.testing.assert_allclose(wg @ RB @ wg.T, 2 * fw * np.eye(K), atol=1e-11)
    res = RA @ wg.T - (RB @ wg.T) * lg[None, :]
    assert np.linalg.norm(res) / (np.linalg.norm(RA) * np.linalg.norm(wg)) < 1e-12
    # same K-dimensional subspace (projector), independent of rotations inside it
    Pg = wg.T @ wg @ RB / (2 * fw)
    Po = wo.T @ wo @ RB / (2 * fw)
    assert np.max(np.abs(Pg - Po)) < 1e-8
    # P-hat depends only on the span: GPU-GEP plan vs oracle tapers
    out = run_plan(plan, x, dev, want=("P",))
    _, Pr = oracle_all(t, x, wo, -0.5, 1 / 2048, 2048)
    assert rel_l2(out["P"], Pr) <= 1e-9


def test_gep_errors_are_reported(dev):
    t = np.array([0.0, 1.0, 1.0, 2.0, 3.0])
    with pytest.raises(pkg.M2Error) as e:
        pkg.Plan(t, 1.0, 0.1, 2, -0.5, 0.1, 10, precision=64)
    assert e.value.status == 4  # M2_ERR_GEP (repeated time => R(B) singular)
    # repeated times are fine with given tapers
    pkg.Plan(t, 1.0, 0.1, 2, -0.5, 0.1, 10, precision=64, tapers=np.ones((2, 5)) * 0.1).close()
    for bad in [dict(K=6), dict(f_w=0.5), dict(f_w=0.0)]:
        kw = dict(K=2, f_w=0.1)
        kw.update(bad)
        with pytest.raises(pkg.M2Error) as e:
            pkg.Plan(np.arange(5.0), 1.0, kw["f_w"], kw["K"], -0.5, 0.1, 10)
        assert e.value.status == 1
    with pytest.raises(pkg.M2Error):
        pkg.Plan(np.array([0.0, np.nan, 2.0]), 1.0, 0.1, 1, -0.5, 0.1, 10)
    with pytest.raises(pkg.M2Error) as e:
        pkg.Plan(np.arange(64.0), 1.0, 0.05, 2, -0.5, 1 / 64, 64, mem_budget=1000)
    assert e.value.status == 3  # M2_ERR_BUDGET


# ---------------------------------------------------------------------------
# leakage estimate (App. B)
# ---------------------------------------------------------------------------
def test_leakage_integer_grid_is_zero(dev):
    wl = synth.workload("grid1024")
    plan = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=64)
    L, E = plan.leakage()
    assert np.max(L) < 1e-12 and np.max(E) < 1e-12
    out = run_plan(plan, wl.x, dev, want=("Lhat", "Ehat"))
    np.testing.assert_array_equal(out["Lhat"], L)


def test_leakage_rate_mismatch_matches_oracle(dev):
    """t_n = 5n/6 with 10 of 60 dropped (Sec. 4 missing-data scheme):
    identical tapers, every band."""
    t = synth.scaled_missing(60, 10, 5.0 / 6.0, 0)
    fw, K, I = 0.05, 4, 200
    w, lam = ogpss.nominal_tapers(t, 1.0, fw, K)
    plan = pkg.Plan(t, 1.0, fw, K, -0.5, 1 / I, I, precision=64, tapers=w, lam=lam)
    L, E = plan.leakage()
    Lr, Er = oleak.leakage_at(t, w, lam, 1.0, fw, -0.5 + np.arange(I) / I)
    np.testing.assert_allclose(L, Lr, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(E, Er, rtol=1e-9, atol=1e-13)


# ---------------------------------------------------------------------------
# full-size workloads (sampled outputs)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("path", [1, 2, 3])
def test_jitter16k_full_size_fp32(dev, path):
    """N = 16384 jittered, K = 8, I = 2^18 (the benchmark workload): FP32
    path with FP64-split coordinates against the direct FP64 sum on sampled
    band centres; seeded tapers (any real taper is a valid input)."""
    wl = synth.workload("jitter16k", batch=2)
    w = seeded_tapers(wl.K, wl.N, 7)
    plan = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32, tapers=w, path=path)
    out = run_plan(plan, wl.x, dev)
    idx = full_size_bands(wl.I, 384, 384, 1)  # 384 = n1 of the packed path at this size
    Jr, Pr = oracle_cached("jitter16k/b2/w7", wl.t, wl.x, w, wl.f_lo, wl.df, wl.I, idx)
    check(out, Jr, Pr, w, wl.x, 32, idx)
    # P-hat is the taper average of the eigenspectra everywhere
    np.testing.assert_allclose(out["P"], out["E"].mean(axis=1), rtol=2e-6, atol=1e-30)


def test_jitter16k_gep_on_gpu(dev):
    """The full-size GEP (N = 16384, FP64 cuSOLVER): eigenvalues in (0,1)
    descending, R(B)-orthonormal tapers and small residuals on sampled rows."""
    wl = synth.workload("jitter16k")
    plan = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32)
    w, lam = plan.tapers()
    assert np.all((lam > 0) & (lam < 1)) and np.all(np.diff(lam) <= 0)
    rows = np.random.default_rng(0).choice(wl.N, 48, replace=False)
    RBr = ogpss.gpss_rows(wl.t, rows, 0.5)
    RAr = ogpss.gpss_rows(wl.t, rows, wl.f_w)
    res = RAr @ w.T - (RBr @ w.T) * lam[None, :]
    scale = np.abs(RBr @ w.T).max()
    assert np.max(np.abs(res)) < 1e-9 * scale
    # R(B)-orthonormality at full size, R(B) w^T formed block by block
    RBw = np.zeros((wl.N, wl.K))
    for r0 in range(0, wl.N, 1024):
        blk = np.arange(r0, min(r0 + 1024, wl.N))
        RBw[blk] = ogpss.gpss_rows(wl.t, blk, 0.5) @ w.T
    np.testing.assert_allclose(w @ RBw, 2 * wl.f_w * np.eye(wl.K), atol=1e-10)


@pytest.mark.parametrize("path", [1, 2, 3])
def test_periodic16k_full_size_fp32(dev, path):
    """N = 16384 grid, blocks of 8 drop 2 (12288 kept), K = 10, I = 2^20."""
    wl = synth.workload("periodic16k")
    w = seeded_tapers(wl.K, wl.N, 9)
    plan = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32, tapers=w, path=path)
    out = run_plan(plan, wl.x, dev)
    idx = full_size_bands(wl.I, 1536, 256, 2)  # 1536 = n1 of the packed path at this size
    Jr, Pr = oracle_cached("periodic16k/b1/w9", wl.t, wl.x, w, wl.f_lo, wl.df, wl.I, idx)
    check(out, Jr, Pr, w, wl.x, 32, idx)


def test_jitter16k_fp64_path(dev):
    wl = synth.workload("jitter16k")
    w = seeded_tapers(wl.K, wl.N, 5)
    plan = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=64, tapers=w)
    out = run_plan(plan, wl.x, dev, want=("J", "P"))
    idx = full_size_bands(wl.I, 384, 128, 3)
    Jr, Pr = oracle_all(wl.t, wl.x, w, wl.f_lo, wl.df, wl.I, idx)
    check(out, Jr, Pr, w, wl.x, 64, idx)


def test_exec_batch_uneven_matches_single(dev, batch_mode):
    """m2nufft_exec_batch over signals with different plans equals
    per-signal exec bit for bit."""
    ws = synth.batched_uneven(4, seed=3, n_min=256, n_max=1500)
    plans, xs, Js, Ps = [], [], [], []
    for s, wl in enumerate(ws):
        p = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32,
                     tapers=seeded_tapers(wl.K, wl.N, s))
        plans.append(p)
        xs.append(torch.from_numpy(wl.x[0].astype(np.float32)).to(dev))
        Js.append(torch.empty((wl.K, wl.I), dtype=torch.complex64, device=dev))
        Ps.append(torch.empty((wl.I,), dtype=torch.float32, device=dev))
    pkg.exec_batch(plans, xs, Js, None, Ps)
    torch.cuda.synchronize()
    for p, x, J, P in zip(plans, xs, Js, Ps):
        single = p.run(x[None, :], want=("J", "P"))
        torch.cuda.synchronize()
        assert torch.equal(single["J"][0], J) and torch.equal(single["P"][0], P)


def test_leakage_windowed_matches_oracle_medium(dev):
    """General sampling above the direct-sum size (N = 2048 jittered, I = 2^14):
    D_k(f) by the windowed band-limited quadrature of |W_k|^2 (App. B,
    Eq. lambda_hat_ki), against the oracle's dense pair sum on sampled bands."""
    t = synth.jittered(2048, 0.4, 41)
    fw, K, I = 5.0 / 2048, 8, 1 << 14
    w, lam = ogpss.nominal_tapers(t, 1.0, fw, K)
    plan = pkg.Plan(t, 1.0, fw, K, -0.5, 1.0 / I, I, precision=64, tapers=w, lam=lam)
    L, E = plan.leakage()
    idx = sample_bands(I, 40, 5)
    Lr, Er = oleak.leakage_at(t, w, lam, 1.0, fw, -0.5 + idx / I)
    assert np.max(np.abs(L[:, idx] - Lr)) <= 1e-10 * max(np.max(np.abs(Lr)), 1e-3)
    assert np.max(np.abs(E[idx] - Er)) <= 1e-10 * max(np.max(np.abs(Er)), 1e-3)
    # the nominal band centre f = 0 has D = 2 f_w exactly (normalisation), so L = 0 there
    assert np.max(np.abs(L[:, I // 2])) < 1e-9


def test_leakage_windowed_full_size(dev):
    """N = 16384 jittered, I = 2^18 (the benchmark workload): L-hat and E-hat
    exist and match the oracle's pair sum on sampled bands (taper-shaped
    inputs and fixed eigenvalues, so no GPU result feeds the oracle)."""
    wl = synth.workload("jitter16k")
    w = seeded_tapers(wl.K, wl.N, 11)
    # scale each row so w^T R(B) w is near 2 f_w (keeps D near the paper's regime)
    w = w * np.sqrt(2 * wl.f_w / np.sum(w ** 2, axis=1))[:, None]
    lam = np.linspace(0.999, 0.95, wl.K)
    plan = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32, tapers=w, lam=lam)
    L, E = plan.leakage()
    idx = sample_bands(wl.I, 4, 9)[:6]
    Lr, Er = oleak.leakage_at(wl.t, w, lam, 1.0, wl.f_w, wl.f_lo + idx * wl.df)
    assert np.max(np.abs(L[:, idx] - Lr)) <= 1e-9 * max(np.max(np.abs(Lr)), 1e-3)
    out = run_plan(plan, wl.x, dev, want=("Lhat", "Ehat"))
    np.testing.assert_array_equal(out["Ehat"], E)


def test_exec_batch_graph_replay_and_repeated_plans(dev):
    """The cached batch graph: repeated plans in one batch (they share a
    stream), replay on a second call, and a new graph after a plan is
    destroyed; every result equals the per-signal exec bit for bit."""
    ws = synth.batched_uneven(3, seed=7, n_min=300, n_max=1200)
    plans = [pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32,
                      tapers=seeded_tapers(wl.K, wl.N, i), max_batch=1) for i, wl in enumerate(ws)]
    order = [0, 1, 0, 2, 1, 0]
    rng = np.random.default_rng(1)
    xs = [torch.from_numpy(rng.standard_normal(ws[i].N).astype(np.float32)).to(dev) for i in order]
    Js = [torch.empty((ws[i].K, ws[i].I), dtype=torch.complex64, device=dev) for i in order]
    Ps = [torch.empty((ws[i].I,), dtype=torch.float32, device=dev) for i in order]
    bp = [plans[i] for i in order]
    for _ in range(2):  # capture, then replay
        for J in Js:
            J.zero_()
        pkg.exec_batch(bp, xs, Js, None, Ps)
        torch.cuda.synchronize()
        for i, x, J, P in zip(order, xs, Js, Ps):
            single = plans[i].run(x[None, :], want=("J", "P"))
            torch.cuda.synchronize()
            assert torch.equal(single["J"][0], J) and torch.equal(single["P"][0], P)
    plans[2].close()
    keep = [k for k, i in enumerate(order) if i != 2]
    pkg.exec_batch([bp[k] for k in keep], [xs[k] for k in keep], [Js[k] for k in keep], None,
                   [Ps[k] for k in keep])
    torch.cuda.synchronize()


# ---------------------------------------------------------------------------
# persistent pipelined kernel (path 3)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("B", [1, 3, 9, 20])
def test_pipe_matches_four_kernels_full_size(dev, B):
    """N = 16384 jittered, K = 8, I = 2^18: the persistent kernel over B signals
    (one launch; B = 9 and 20 wrap the seven-slot workspace ring) equals the
    four-kernel path bit for bit in J, |J|^2 and P-hat."""
    wl = synth.workload("jitter16k", batch=B, seed=B)
    w = seeded_tapers(wl.K, wl.N, 17)
    p2 = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32, tapers=w, path=2)
    p3 = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32, tapers=w, path=3)
    assert p3.info["path"] == 3 and p2.info["path"] == 2
    o2 = run_plan(p2, wl.x, dev)
    o3 = run_plan(p3, wl.x, dev)
    for k in ("J", "E", "P"):
        assert np.array_equal(o3[k], o2[k]), k
    # and twice in a row on the same plan (counters reset per launch)
    o3b = run_plan(p3, wl.x, dev, want=("P",))
    assert np.array_equal(o3b["P"], o2["P"])


def test_default_path_selection(dev):
    """Automatic choice: packed four-kernel path for qualifying FP32 plans, the persistent
    kernel on request, the generic path for FP64; the packed chunk is 4 to 16 signals by the
    workspace rule (4 for this size) and exactly max_batch when given (at most 64)."""
    wl = synth.workload("jitter16k")
    w = seeded_tapers(wl.K, wl.N, 1)
    args = (wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I)
    p2 = pkg.Plan(*args, precision=32, tapers=w)
    assert p2.info["path"] == 2 and p2.info["chunk"] == 4
    assert pkg.Plan(*args, precision=32, tapers=w, max_batch=24).info["chunk"] == 24
    assert pkg.Plan(*args, precision=32, tapers=w, max_batch=500).info["chunk"] == 64
    assert pkg.Plan(*args, precision=32, tapers=w, path=3).info["path"] == 3
    assert pkg.Plan(*args, precision=64, tapers=w).info["path"] == 1
    small = synth.workload("grid1024")
    ws = seeded_tapers(small.K, small.N, 1)
    assert pkg.Plan(small.t, small.fs, small.f_w, small.K, small.f_lo, small.df, small.I, precision=32,
                    tapers=ws).info["chunk"] == 16


def test_pipe_bounded_wait_reports_timeout(dev):
    """A work item whose dependency never completes: the wait gives up after the
    limit, the kernel returns M2_ERR_TIMEOUT through its status word, and the
    context stays usable (a following exec is correct)."""
    import time
    t0 = time.perf_counter()
    st = pkg.binding.pipe_selftest(50)
    dt = time.perf_counter() - t0
    assert st == 6, pkg.binding.load().m2nufft_last_error().decode()
    assert dt >= 0.05
    t = synth.jittered(900, 0.4, 5)
    X = np.stack([synth.white(t, 1.0, 80 + b) for b in range(2)])
    w = seeded_tapers(4, 900, 2)
    plan = pkg.Plan(t, 1.0, 2.0 / 900, 4, -0.5, 1.0 / 2048, 2048, precision=32, tapers=w, path=3)
    out = run_plan(plan, X, dev)
    Jr, Pr = oracle_all(t, X, w, -0.5, 1.0 / 2048, 2048)
    check(out, Jr, Pr, w, X, 32)


@pytest.fixture(params=[0, 1], ids=["stage_batched", "persistent"])
def batch_mode(request):
    prev = pkg.binding.set_batch_mode(request.param)
    yield request.param
    pkg.binding.set_batch_mode(prev)


def test_exec_batch_pipe_heterogeneous_matches_oracle(dev, batch_mode):
    """All-packed uneven batch (one launch per stage, or one persistent launch):
    plans of different N, K (odd K included), I and n1 (coset FFT lengths
    F = 2..32), more signals than ring slots; equals the four-kernel
    per-signal exec bit for bit and the oracle within the FP32 tolerance."""
    ws = synth.batched_uneven(11, seed=12, n_min=300, n_max=8000)
    Ks = [1, 3, 5, 8, 6, 4, 7, 2, 8, 5, 3]
    plans2, plans3, xs, Js, Es, Ps, ws2 = [], [], [], [], [], [], []
    for s, (wl, K) in enumerate(zip(ws, Ks)):
        w = seeded_tapers(K, wl.N, 40 + s)
        args = (wl.t, wl.fs, (K / 2 + 1) / wl.N, K, wl.f_lo, wl.df, wl.I)
        plans2.append(pkg.Plan(*args, precision=32, tapers=w, path=2))
        plans3.append(pkg.Plan(*args, precision=32, tapers=w, path=3))
        xs.append(torch.from_numpy(wl.x[0].astype(np.float32)).to(dev))
        Js.append(torch.empty((K, wl.I), dtype=torch.complex64, device=dev))
        Es.append(torch.empty((K, wl.I), dtype=torch.float32, device=dev))
        Ps.append(torch.empty((wl.I,), dtype=torch.float32, device=dev))
        ws2.append((wl, w))
    assert len({p.info["n1"] for p in plans3}) >= 3
    for rep in range(2):  # build + launch, then graph replay
        for J in Js:
            J.zero_()
        pkg.exec_batch(plans3, xs, Js, Es, Ps)
        torch.cuda.synchronize()
        for p, x, J, E, P in zip(plans2, xs, Js, Es, Ps):
            single = p.run(x[None, :], want=("J", "E", "P"))
            torch.cuda.synchronize()
            assert torch.equal(single["J"][0], J) and torch.equal(single["E"][0], E)
            assert torch.equal(single["P"][0], P)
    for (wl, w), J, E, P in zip(ws2, Js, Es, Ps):
        Jr, _, Pr = oest.m2nufft(wl.t, wl.x[0], w, wl.f_lo, wl.df, wl.I)
        o = {"J": J.cpu().numpy()[None], "E": E.cpu().numpy()[None], "P": P.cpu().numpy()[None]}
        check(o, Jr[None], Pr[None], w, wl.x, 32)


def test_exec_batch_mixed_generic_and_pipelined(dev):
    """A batch with a generic-path plan among pipelined plans is captured per
    signal; the pipelined plans' launches are prepared outside the capture."""
    ws = synth.batched_uneven(3, seed=21, n_min=300, n_max=1200)
    paths = [3, 1, 3]
    plans = [pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32,
                      tapers=seeded_tapers(wl.K, wl.N, i), path=pth) for i, (wl, pth) in enumerate(zip(ws, paths))]
    xs = [torch.from_numpy(wl.x[0].astype(np.float32)).to(dev) for wl in ws]
    Ps = [torch.empty((wl.I,), dtype=torch.float32, device=dev) for wl in ws]
    pkg.exec_batch(plans, xs, None, None, Ps)
    torch.cuda.synchronize()
    for p, x, P in zip(plans, xs, Ps):
        single = p.run(x[None, :], want=("P",))
        torch.cuda.synchronize()
        assert torch.equal(single["P"][0], P)


# ---------------------------------------------------------------------------
# Thomson F-statistic (Sec. 3, Eq. f_stat)
# ---------------------------------------------------------------------------
def _f_bound(Jg, Jr, Fr, K, prec):
    """Per-band bound on |F_gpu - F_ref| / F_ref propagated from the eigencoefficient error at
    that band: with eps = ||J_gpu - J_ref|| / ||J_ref|| over the K tapers, the projections of J on
    W and on its complement move by at most eps ||J||, so the relative error of F is at most
    2 eps (sqrt(1 + (K-1)/F) + sqrt(1 + F/(K-1))) to first order; 3x that, plus the rounding of
    the statistic's own arithmetic (eps floor)."""
    eps = np.linalg.norm(Jg - Jr, axis=0) / np.linalg.norm(Jr, axis=0)
    eps = eps + (4e-7 * np.sqrt(K) if prec == 32 else 1e-14)
    return 3 * eps * (np.sqrt(1 + (K - 1) / Fr) + np.sqrt(1 + Fr / (K - 1)))


@pytest.mark.parametrize("prec,path", PATHS)
def test_ftest_parity(dev, prec, path):
    """F at every band against the oracle's F from its FP64 eigencoefficients (same tapers), within
    the bound propagated from the eigencoefficient error; the injected lines are detected."""
    from oracle import ftest as oft
    scipy_stats = pytest.importorskip("scipy.stats")
    N, K, I = 3000, 6, 8192
    fw = 4.0 / N
    t = synth.jittered(N, 0.4, 31)
    X = np.stack([synth.tones(t, np.array([0.1 + 0.01 * b, -0.3]), np.array([1.5, 0.8]), 1.0, 90 + b)
                  for b in range(2)])
    w, lam = ogpss.nominal_tapers(t, 1.0, fw, K)
    plan = pkg.Plan(t, 1.0, fw, K, -0.5, 1.0 / I, I, precision=prec, tapers=w, lam=lam, path=path)
    out = run_plan(plan, X, dev, want=("J", "P", "F"))
    Jr, Pr = oracle_all(t, X, w, -0.5, 1.0 / I, I)
    crit = scipy_stats.f(2, 2 * K - 2).ppf(1 - 1.0 / N)
    for b in range(X.shape[0]):
        Fr = oft.f_statistic(Jr[b], w)
        bound = _f_bound(out["J"][b], Jr[b], Fr, K, prec)
        rel = np.abs(out["F"][b] - Fr) / Fr
        assert np.all(rel <= bound), (np.max(rel / bound), int(np.argmax(rel / bound)))
        line = int(round((0.1 + 0.01 * b + 0.5) * I))
        assert out["F"][b][line] > crit
    check(out, Jr, Pr, w, X, prec)


def test_ftest_generic_without_J(dev):
    """Generic path, F requested without J: the internal J buffer gives the same F."""
    N, K, I = 1200, 5, 4096
    t = synth.jittered(N, 0.4, 8)
    X = np.stack([synth.white(t, 1.0, 60 + b) for b in range(3)])
    w = seeded_tapers(K, N, 3)
    plan = pkg.Plan(t, 1.0, 3.0 / N, K, -0.5, 1.0 / I, I, precision=64, tapers=w, path=1, max_batch=2)
    a = run_plan(plan, X, dev, want=("J", "F"))
    b = run_plan(plan, X, dev, want=("P", "F"))
    assert np.array_equal(a["F"], b["F"])


def test_ftest_full_size_sampled(dev):
    """jitter16k (N = 16384, K = 8, I = 2^18), FP32 packed path: F on sampled bands against the
    oracle's F from its FP64 eigencoefficients at those bands."""
    from oracle import ftest as oft
    wl = synth.workload("jitter16k", batch=1)
    w = seeded_tapers(wl.K, wl.N, 7)
    plan = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32, tapers=w)
    out = run_plan(plan, wl.x, dev, want=("J", "F"))
    idx = sample_bands(wl.I, 256, 4)
    Jr, _ = oracle_all(wl.t, wl.x, w, wl.f_lo, wl.df, wl.I, idx)
    Fr = oft.f_statistic(Jr[0], w)
    bound = _f_bound(out["J"][0][:, idx], Jr[0], Fr, wl.K, 32)
    assert np.all(np.abs(out["F"][0][idx] - Fr) / Fr <= bound)


def test_ftest_rejects_single_taper(dev):
    t = synth.jittered(300, 0.4, 1)
    plan = pkg.Plan(t, 1.0, 0.01, 1, -0.5, 1 / 1024, 1024, precision=32, tapers=seeded_tapers(1, 300, 0))
    x = torch.zeros((1, 300), dtype=torch.float32, device=dev)
    F = torch.empty((1, 1024), dtype=torch.float32, device=dev)
    with pytest.raises(pkg.M2Error) as e:
        plan.exec(x, F=F)
    assert e.value.status == 1


@pytest.mark.parametrize("mode", [0, 1, 2], ids=["stage_batched", "persistent", "tuned"])
def test_exec_batch_ftest_matches_single(dev, mode):
    """m2nufft_exec_batch_ftest over an all-packed uneven batch (different N, K, I; one signal
    without F): F, J and P-hat equal per-signal m2nufft_exec_ftest bit for bit in every batch
    mode (mode 1 runs stage-batched, the persistent kernel forms no F); the batch without F
    outputs on the same plans still equals plain exec."""
    ws = synth.batched_uneven(5, seed=44, n_min=300, n_max=6000)
    Ks = [4, 3, 8, 2, 5]
    plans, xs, Js, Ps, Fs = [], [], [], [], []
    for s, (wl, K) in enumerate(zip(ws, Ks)):
        plans.append(pkg.Plan(wl.t, wl.fs, wl.f_w, K, wl.f_lo, wl.df, wl.I, precision=32,
                              tapers=seeded_tapers(K, wl.N, 70 + s)))
        xs.append(torch.from_numpy(wl.x[0].astype(np.float32)).to(dev))
        Js.append(torch.empty((K, wl.I), dtype=torch.complex64, device=dev))
        Ps.append(torch.empty((wl.I,), dtype=torch.float32, device=dev))
        Fs.append(None if s == 2 else torch.empty((wl.I,), dtype=torch.float32, device=dev))
    prev = pkg.binding.set_batch_mode(mode)
    try:
        pkg.exec_batch(plans, xs, Js, None, Ps, Fs=Fs)
        torch.cuda.synchronize()
        for p, x, J, P, F in zip(plans, xs, Js, Ps, Fs):
            Jr = torch.empty((1,) + tuple(J.shape), dtype=J.dtype, device=dev)
            Pr = torch.empty((1,) + tuple(P.shape), dtype=P.dtype, device=dev)
            if F is None:
                p.exec(x[None, :], J=Jr, P=Pr)
            else:
                Fr = torch.empty((1,) + tuple(F.shape), dtype=F.dtype, device=dev)
                p.exec(x[None, :], J=Jr, P=Pr, F=Fr)
            torch.cuda.synchronize()
            assert torch.equal(Jr[0], J) and torch.equal(Pr[0], P)
            if F is not None:
                assert torch.equal(Fr[0], F)
        # same plans and buffers without F: another graph, plain exec's bits
        P2 = [torch.empty_like(P) for P in Ps]
        pkg.exec_batch(plans, xs, None, None, P2)
        torch.cuda.synchronize()
        for P, Q in zip(Ps, P2):
            assert torch.equal(P, Q)
    finally:
        pkg.binding.set_batch_mode(prev)


def test_exec_batch_ftest_generic_and_rejections(dev):
    """A batch with a generic-path plan is captured per signal with each signal's F (bitwise equal
    to exec_ftest); a signal with F on a one-taper plan or a sub-band plan is rejected, and the
    one-taper plan without an F output is accepted."""
    ws = synth.batched_uneven(3, seed=45, n_min=300, n_max=1500)
    paths = [2, 1, 3]
    plans = [pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32,
                      tapers=seeded_tapers(wl.K, wl.N, 80 + i), path=pth) for i, (wl, pth) in enumerate(zip(ws, paths))]
    xs = [torch.from_numpy(wl.x[0].astype(np.float32)).to(dev) for wl in ws]
    Fs = [torch.empty((wl.I,), dtype=torch.float32, device=dev) for wl in ws]
    pkg.exec_batch(plans, xs, None, None, None, Fs=Fs)
    torch.cuda.synchronize()
    for p, x, F in zip(plans, xs, Fs):
        Fr = torch.empty((1,) + tuple(F.shape), dtype=F.dtype, device=dev)
        p.exec(x[None, :], F=Fr)
        torch.cuda.synchronize()
        assert torch.equal(Fr[0], F)
    t = synth.jittered(300, 0.4, 1)
    one = pkg.Plan(t, 1.0, 0.01, 1, -0.5, 1 / 1024, 1024, precision=32, tapers=seeded_tapers(1, 300, 0))
    x1 = torch.zeros((300,), dtype=torch.float32, device=dev)
    F1 = torch.empty((1024,), dtype=torch.float32, device=dev)
    with pytest.raises(pkg.M2Error) as e:
        pkg.exec_batch([plans[0], one], [xs[0], x1], None, None, None, Fs=[Fs[0], F1])
    assert e.value.status == 1
    P1 = torch.empty((1024,), dtype=torch.float32, device=dev)
    pkg.exec_batch([plans[0], one], [xs[0], x1], None, None, [None, P1], Fs=[Fs[0], None])
    torch.cuda.synchronize()
    fw, f_c0, f_min, f_max = 4.0 / 300, 0.3, 0.2, 0.4
    w, lam = ogpss.subband_tapers(t, fw, 3, f_c0, f_min, f_max)
    sb = pkg.Plan(t, 1.0, fw, 3, 0.25, 0.1 / 512, 512, precision=32, tapers=w, lam=lam, subband=(f_c0, f_min, f_max))
    Fsb = torch.empty((512,), dtype=torch.float32, device=dev)
    with pytest.raises(pkg.M2Error) as e:
        pkg.exec_batch([sb], [x1], None, None, None, Fs=[Fsb])
    assert e.value.status == 1


# ---------------------------------------------------------------------------
# interpolated-DPSS tapers (Table 1 step 3 a-c), no GEP
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["jitter", "bernoulli"])
def test_spline_tapers_match_oracle(dev, kind):
    """Plan-time tapers from DPSS + not-a-knot spline + R(B) normalisation against the oracle's
    (independent tridiagonal solver, scipy spline, dense quadratic forms); then J and P-hat with
    them against the oracle's direct sum."""
    from oracle import spline_tapers as ost
    N, K, I = 1500, 6, 4096
    fw = 4.0 / N
    t = synth.jittered(N, 0.4, 17) if kind == "jitter" else synth.grid_bernoulli(1800, 0.17, 17)
    N = t.size
    wr, lr = ost.spline_tapers(t, 1.0, fw, K)
    plan = pkg.Plan(t, 1.0, fw, K, -0.5, 1.0 / I, I, precision=64, taper_design="spline")
    w, lam = plan.tapers()
    np.testing.assert_allclose(w, wr, rtol=0, atol=1e-10 * np.abs(wr).max())
    np.testing.assert_allclose(lam, lr, rtol=1e-10)
    X = np.stack([synth.white(t, 1.0, 33 + b) for b in range(2)])
    out = run_plan(plan, X, dev, want=("J", "P"))
    Jr, Pr = oracle_all(t, X, w, -0.5, 1.0 / I, I)
    check(out, Jr, Pr, w, X, 64)


def test_spline_tapers_full_size(dev):
    """N = 16384 jittered, K = 8: the interpolated tapers are R(B)-normalised (checked block by
    block against the oracle's R(B) rows), their concentrations lie in (0, 1) and do not exceed
    the first GEP eigenvalue bound 1, and planning takes well under the GEP's time."""
    import time
    wl = synth.workload("jitter16k")
    t0 = time.perf_counter()
    plan = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32, taper_design="spline")
    dt = time.perf_counter() - t0
    w, lam = plan.tapers()
    assert np.all((lam > 0) & (lam < 1))
    RBw = np.zeros((wl.N, wl.K))
    for r0 in range(0, wl.N, 1024):
        blk = np.arange(r0, min(r0 + 1024, wl.N))
        RBw[blk] = ogpss.gpss_rows(wl.t, blk, 0.5) @ w.T
    np.testing.assert_allclose(np.einsum("kn,nk->k", w, RBw), 2 * wl.f_w, rtol=1e-10)
    assert plan.info["gep_seconds"] < 5.0 and dt < 30.0


# ---------------------------------------------------------------------------
# multiband: sub-band plans (Sec. 2.3, Sec. 3, Eq. gpss_matrix_b_q, f_c0 != 0)
# ---------------------------------------------------------------------------
def _subband_oracle(t, X, w, f_c0, f_lo, df, I):
    Js, Ps = [], []
    for b in range(X.shape[0]):
        J, _, P = oest.m2nufft(t, X[b], w, f_lo - f_c0, df, I)
        Js.append(J)
        Ps.append(P)
    return np.stack(Js), np.stack(Ps)


@pytest.mark.parametrize("prec", [64, 32])
def test_subband_parity(dev, prec):
    """Sub-band [0.1, 0.3] with nominal centre 0.2 on a jittered pattern: complex tapers from the
    oracle's Hermitian GEP; J and P-hat at absolute band centres inside the sub-band against the
    direct sum with Delta f_i = f_ci - f_c0."""
    N, K, I = 1200, 4, 2048
    fw, f_c0, f_min, f_max = 4.0 / N, 0.2, 0.1, 0.3
    t = synth.jittered(N, 0.4, 23)
    w, lam = ogpss.subband_tapers(t, fw, K, f_c0, f_min, f_max)
    f_lo, df = 0.105, 0.19 / I
    X = np.stack([synth.tones(t, np.array([0.17, 0.26]), np.array([1.0, 0.5]), 1.0, 70 + b) for b in range(2)])
    plan = pkg.Plan(t, 1.0, fw, K, f_lo, df, I, precision=prec, tapers=w, lam=lam, subband=(f_c0, f_min, f_max))
    assert plan.info["path"] == 1 and plan.info["real_taper"] == 0
    out = run_plan(plan, X, dev, want=("J", "P"))
    Jr, Pr = _subband_oracle(t, X, w, f_c0, f_lo, df, I)
    check(out, Jr, Pr, w, X, prec)
    wg, lg = plan.tapers()
    np.testing.assert_array_equal(wg, w)


def test_subband_gep_matches_oracle(dev):
    """The GPU's range-restricted Hermitian GEP against the oracle's: eigenvalues, the K-dimensional
    taper subspace (R(B^q) inner products of the two bases are 2 f_w times a unitary matrix), the
    normalisation and the phase rule."""
    N, K = 900, 5
    fw, f_c0, f_min, f_max = 4.0 / N, 0.31, 0.22, 0.45
    t = synth.grid_bernoulli(1100, 0.18, 4)
    N = t.size
    w, lam = ogpss.subband_tapers(t, fw, K, f_c0, f_min, f_max)
    plan = pkg.Plan(t, 1.0, fw, K, 0.25, 0.1 / 512, 512, precision=64, subband=(f_c0, f_min, f_max))
    wg, lg = plan.tapers()
    np.testing.assert_allclose(lg, lam, atol=1e-10)
    RB = ogpss.gpss_matrix_b_sub(t, f_min, f_max)
    G = np.conj(wg) @ RB @ w.T / (2 * fw)
    sv = np.linalg.svd(G, compute_uv=False)
    np.testing.assert_allclose(sv, 1.0, atol=1e-8)
    np.testing.assert_allclose(np.real(np.einsum("kn,nm,km->k", np.conj(wg), RB, wg)), 2 * fw, rtol=1e-10)
    dem = np.exp(-2j * np.pi * f_c0 * t)
    tc = t - t.mean()
    for k in range(K):
        s = np.sum(wg[k] * dem * (tc if k % 2 else 1.0))
        assert s.real > 0 and abs(s.imag) < 1e-9 * abs(s)


@pytest.mark.parametrize("prec", [64, 32])
def test_subband_leakage_matches_oracle(dev, prec):
    """Leakage estimates of a sub-band plan (App. B with R(B^q), shifts f_ci - f_c0) against the
    oracle's dense form at every band, from the plan's own tapers and eigenvalues; exec hands them
    out like those of a full-band plan."""
    fw, f_c0, f_min, f_max = 4.0 / 400, 0.31, 0.22, 0.45
    t = synth.grid_bernoulli(500, 0.2, 7)
    K, I = 4, 256
    plan = pkg.Plan(t, 1.0, fw, K, 0.25, 0.12 / I, I, precision=prec, subband=(f_c0, f_min, f_max))
    wg, lg = plan.tapers()
    L, E = plan.leakage()
    Lo, Eo = oleak.leakage_subband_at(t, wg, lg, fw, f_min, f_max, 0.25 - f_c0 + 0.12 / I * np.arange(I))
    np.testing.assert_allclose(L, Lo, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(E, Eo, rtol=1e-9, atol=1e-13)
    x = torch.from_numpy(synth.white(t, 1.0, 3)[None, :].astype(np.float64 if prec == 64 else np.float32)).to(dev)
    out = plan.run(x, want=("P", "Lhat", "Ehat"))
    torch.cuda.synchronize()
    assert np.array_equal(out["Lhat"].cpu().numpy(), L) and np.array_equal(out["Ehat"].cpu().numpy(), E)


def test_multiband_partition_batch(dev):
    """Q = 3 sub-bands partitioning [0, 1/2] run as one exec_batch on the same signal: each equals
    its own exec bit for bit and the oracle within the FP64 tolerance."""
    N, K = 700, 3
    fw = 3.0 / N
    t = synth.jittered(N, 0.4, 29)
    x = synth.white(t, 1.0, 5)
    bands = [(0.06, 0.0, 0.12), (0.2, 0.12, 0.3), (0.4, 0.3, 0.5)]
    I = 512
    plans, Ps, ws = [], [], []
    for f_c0, a, b in bands:
        w, lam = ogpss.subband_tapers(t, fw, K, f_c0, a, b)
        lo = max(a, f_c0 - 0.05)
        plans.append(pkg.Plan(t, 1.0, fw, K, lo, 0.1 / I, I, precision=64, tapers=w, lam=lam,
                              subband=(f_c0, a, b)))
        ws.append((w, f_c0, lo))
        Ps.append(torch.empty((I,), dtype=torch.float64, device=dev))
    xs = [torch.from_numpy(x).to(dev) for _ in bands]
    pkg.exec_batch(plans, xs, None, None, Ps)
    torch.cuda.synchronize()
    for p, P, (w, f_c0, lo) in zip(plans, Ps, ws):
        single = p.run(xs[0][None, :], want=("P",))
        torch.cuda.synchronize()
        assert torch.equal(single["P"][0], P)
        Jr, Pr = _subband_oracle(t, x[None, :], w, f_c0, lo, 0.1 / I, I)
        assert rel_l2(P.cpu().numpy(), Pr[0]) <= TOL[64]
        l1 = source_l1(w, x)
        assert_elementwise(None, Jr, l1, TOL[64], P.cpu().numpy()[None], Pr)


def test_subband_rejects_band_outside(dev):
    t = synth.jittered(300, 0.4, 1)
    with pytest.raises(pkg.M2Error) as e:
        pkg.Plan(t, 1.0, 0.02, 2, 0.1, 1e-4, 64, precision=64, subband=(0.11, 0.1, 0.3))
    assert e.value.status == 1


# ---------------------------------------------------------------------------
# true suboptimality from per-band GEPs (Sec. 3, Eq. subopt_measure)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["jitter", "integer"])
def test_true_suboptimality_matches_oracle(dev, kind):
    """E_i from the GPU's per-band Hermitian GEPs against the oracle's (LAPACK per band); on an
    integer grid E = 0; the plan's own L-hat for the leading taper is consistent with the per-band
    optimum (lambda_hat_0^i <= lambda_0^i, Courant-Fischer)."""
    from oracle import true_subopt as ots
    t = synth.jittered(40, 0.4, 5) if kind == "jitter" else synth.grid_bernoulli(52, 0.2, 3)
    N, K, fw, I = t.size, 3, 3.0 / 40, 96
    w, lam0 = ogpss.nominal_tapers(t, 1.0, fw, K)
    f_lo, df = -0.42, 0.84 / I  # analysis bands inside |f| <= 1/2
    plan = pkg.Plan(t, 1.0, fw, K, f_lo, df, I, precision=64, tapers=w, lam=lam0)
    E, lb = plan.true_suboptimality()
    freqs = f_lo + df * np.arange(I)
    lbr = ots.band_eigenvalues(t, 1.0, fw, K, freqs)
    np.testing.assert_allclose(lb, lbr, atol=1e-10)
    np.testing.assert_allclose(E, ots.true_suboptimality(lam0, lbr), atol=1e-10)
    if kind == "integer":
        assert np.max(np.abs(E)) < 1e-10
    else:
        L, Eh = plan.leakage()
        lam_hat0 = lam0[0] * 2 * fw / oleak.leakage_denominator(t, w, 1.0, freqs)[0]
        np.testing.assert_allclose(np.abs(lam0[0] - lam_hat0), L[0], atol=1e-9)
        assert np.all(lb[:, 0] >= lam_hat0 - 1e-10)


# ---------------------------------------------------------------------------
# oversampling option and plan-time autotuning
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec,path,sigma", [(32, 2, 2.0), (32, 3, 2.0), (32, 2, 3.0), (64, 1, 3.0)])
def test_sigma_option_parity(dev, prec, path, sigma):
    """A requested oversampling factor sigma: nf >= sigma I, the packed path takes the narrower
    width of the sigma >= 2 rule, and the result still meets the parity bar."""
    wl = synth.workload("jitter16k", batch=2)
    w = seeded_tapers(wl.K, wl.N, 5)
    args = (wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I)
    base = pkg.Plan(*args, precision=prec, tapers=w, path=path)
    plan = pkg.Plan(*args, precision=prec, tapers=w, path=path, sigma=sigma)
    assert plan.info["path"] == path
    assert plan.info["nf"] >= sigma * wl.I
    if path >= 2:
        assert plan.info["width"] < base.info["width"]
    out = run_plan(plan, wl.x, dev)
    idx = full_size_bands(wl.I, plan.info["n1"] if path >= 2 else 384, 256, 2)
    Jr, Pr = oracle_cached(f"jitter16k/b2/w5/n1={plan.info['n1']}", wl.t, wl.x, w, wl.f_lo, wl.df, wl.I, idx)
    check(out, Jr, Pr, w, wl.x, prec, idx)


@pytest.mark.parametrize("path", [2, 3])
def test_sigma_125_parity(dev, path):
    """Oversampling 1.25 on the packed path: nf = 5 * 2^a (n1 = 320 for I = 2^18, ten cosets of 32),
    the wider kernel of the sigma < 1.5 rule, results within the parity bar at the full-size
    special positions, and the stage-batched executor bit-identical to the plan's own exec."""
    wl = synth.workload("jitter16k", batch=2)
    w = seeded_tapers(wl.K, wl.N, 5)
    args = (wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I)
    base = pkg.Plan(*args, precision=32, tapers=w, path=path)
    plan = pkg.Plan(*args, precision=32, tapers=w, path=path, sigma=1.25)
    assert plan.info["path"] == path
    assert plan.info["nf"] == 5 * 65536 and plan.info["n1"] == 320
    assert plan.info["width"] > base.info["width"]
    out = run_plan(plan, wl.x, dev)
    idx = full_size_bands(wl.I, plan.info["n1"], 256, 2)
    Jr, Pr = oracle_cached(f"jitter16k/b2/w5/n1={plan.info['n1']}", wl.t, wl.x, w, wl.f_lo, wl.df, wl.I, idx)
    check(out, Jr, Pr, w, wl.x, 32, idx)
    Ps = [torch.empty((wl.I,), dtype=torch.float32, device=dev) for _ in range(2)]
    xs = [torch.from_numpy(wl.x[b].astype(np.float32)).to(dev) for b in range(2)]
    pkg.exec_batch([plan, plan], xs, None, None, Ps)
    torch.cuda.synchronize()
    assert all(np.array_equal(Ps[b].cpu().numpy(), out["P"][b]) for b in range(2))


def test_sigma_option_rejects_out_of_range(dev):
    wl = synth.workload("jitter16k")
    w = seeded_tapers(wl.K, wl.N, 5)
    for s in (1.2, 9.0, -1.0):
        with pytest.raises(pkg.M2Error):
            pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32, tapers=w, sigma=s)


def test_autotuned_plan(dev):
    """tune = True: the report lists the packed configurations (default, sigma 2, chunks of 4, 8
    and 16 signals other than the default, persistent), the plan kept is the fastest of them, its output meets the parity bar, and the
    eigenvalues handed in survive the rebuild (the leakage estimate is the untuned plan's)."""
    wl = synth.workload("jitter16k", batch=3)
    w = seeded_tapers(wl.K, wl.N, 8)
    lam = np.linspace(0.999, 0.95, wl.K)
    args = (wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I)
    ref = pkg.Plan(*args, precision=32, tapers=w, lam=lam)
    plan = pkg.Plan(*args, precision=32, tapers=w, lam=lam, tune=True)
    rep = plan.tuning()
    ch = ref.info["chunk"]
    chunks = [c for c in (4, 8, 16) if c != ch]
    assert [r[0] for r in rep] == [2, 2] + [2] * len(chunks) + [3]
    assert rep[1][1] == 2.0 and [r[2] for r in rep[2:-1]] == chunks
    ms = [r[3] for r in rep]
    assert all(0 < m < 1e3 for m in ms)
    best = int(np.argmin(ms))
    assert plan.info["path"] == rep[best][0]
    if best == 1:
        assert plan.info["nf"] >= 2 * wl.I
    if 2 <= best < len(rep) - 1:
        assert plan.info["chunk"] == rep[best][2]
    assert ref.tuning() == []
    out = run_plan(plan, wl.x, dev)
    idx = full_size_bands(wl.I, plan.info["n1"], 256, 3)
    Jr, Pr = oracle_all(wl.t, wl.x, w, wl.f_lo, wl.df, wl.I, idx)
    check(out, Jr, Pr, w, wl.x, 32, idx)
    for a, b in zip(plan.leakage(), ref.leakage()):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=0)


def test_autotune_leaves_generic_plans_untuned(dev):
    wl = synth.workload("jitter16k")
    w = seeded_tapers(wl.K, wl.N, 8)
    plan = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=64, tapers=w, tune=True)
    assert plan.info["path"] == 1 and plan.tuning() == []


def test_multichunk_spread_buffer_reuse_bitwise(dev):
    """Execs of several chunks spread all their signals in one launch into a buffer the plan keeps
    and grows: B = 9, then 20, then 5 on one plan give, signal by signal, the same bits as execs
    of one signal (spread per chunk, one signal per CTA)."""
    wl = synth.workload("jitter16k", batch=20)
    w = seeded_tapers(wl.K, wl.N, 13)
    plan = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32, tapers=w, path=2)
    assert plan.info["chunk"] < 9
    xt = torch.from_numpy(wl.x.astype(np.float32)).to(dev)
    alone = [plan.run(xt[b:b + 1], want=("J", "P")) for b in range(20)]
    for B in (9, 20, 5):
        out = plan.run(xt[:B], want=("J", "P"))
        torch.cuda.synchronize()
        for b in range(B):
            assert torch.equal(out["J"][b], alone[b]["J"][0]), (B, b)
            assert torch.equal(out["P"][b], alone[b]["P"][0]), (B, b)


# ---------------------------------------------------------------------------
# the uneven batch at its full size: 2048 signals in one exec_batch, 64 of them against the oracle
# ---------------------------------------------------------------------------
def _uneven_subset(ws, n, seed):
    """A seeded subset of the batch that holds its shortest and longest signals and every K class."""
    rng = np.random.default_rng(seed)
    Ns = np.array([wl.N for wl in ws])
    pick = {int(np.argmin(Ns)), int(np.argmax(Ns))}
    for K in sorted({wl.K for wl in ws}):
        pick.add(int(next(s for s, wl in enumerate(ws) if wl.K == K)))
    rest = [s for s in rng.permutation(len(ws)) if s not in pick]
    return sorted(pick | set(int(s) for s in rest[: n - len(pick)]))


@pytest.mark.parametrize("mode", [0, 1, 2], ids=["stage_batched", "persistent", "tuned"])
def test_uneven_2048_batch_against_oracle(dev, mode):
    """The uneven-batch workload at its size: 2048 signals (grid length log-uniform in
    [1024, 16384], Markov gaps, K in {4, 6, 8}, I = 4G) planned with taper-shaped inputs and run as
    one m2nufft_exec_batch; 64 of them (the shortest and longest, every K) against the oracle on
    sampled bands plus each plan's packed special positions, and the persistent form (batch mode 1)
    equal to the stage-batched one bit for bit on the subset."""
    ws = synth.batched_uneven(2048, seed=0)
    sub = _uneven_subset(ws, 64, 5)
    plans, xs, Js, Es, Ps, tap = [], [], [], [], [], []
    for s, wl in enumerate(ws):
        w = seeded_tapers(wl.K, wl.N, s)
        plans.append(pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32, tapers=w,
                              max_batch=1))
        xs.append(torch.from_numpy(wl.x[0].astype(np.float32)).to(dev))
        Js.append(torch.empty((wl.K, wl.I), dtype=torch.complex64, device=dev))
        Es.append(torch.empty((wl.K, wl.I), dtype=torch.float32, device=dev))
        Ps.append(torch.empty((wl.I,), dtype=torch.float32, device=dev))
        tap.append(w if s in sub else None)
    assert all(p.info["path"] == 2 for p in plans)
    prev = pkg.binding.set_batch_mode(0)
    try:
        pkg.exec_batch(plans, xs, Js, Es, Ps)
        torch.cuda.synchronize()
        got = {s: {"J": Js[s].cpu().numpy()[None], "E": Es[s].cpu().numpy()[None], "P": Ps[s].cpu().numpy()[None]}
               for s in sub}
        if mode in (1, 2):
            pkg.binding.set_batch_mode(mode)
            for J in Js:
                J.zero_()
            pkg.exec_batch(plans, xs, Js, Es, Ps)
            torch.cuda.synchronize()
            for s in sub:
                assert np.array_equal(Js[s].cpu().numpy()[None], got[s]["J"]), s
                assert np.array_equal(Ps[s].cpu().numpy()[None], got[s]["P"]), s
        if mode == 2:
            rep = pkg.binding.batch_tuning()
            assert len(rep) == 13 and all(ms > 0 for _, ms in rep)
            assert {c[0] for c, _ in rep} == {0, 1}
    finally:
        pkg.binding.set_batch_mode(prev)
    worst = {}
    for s in sub:
        wl = ws[s]
        idx = np.union1d(sample_bands(wl.I, 64, s), packed_edge_bands(wl.I, plans[s].info["n1"]))
        Jr, _, Pr = oest.m2nufft(wl.t, wl.x[0], tap[s], wl.f_lo, wl.df, wl.I, idx)
        r = check(got[s], Jr[None], Pr[None], tap[s], wl.x, 32, idx)
        for k, v in r.items():
            worst[k] = max(worst.get(k, 0.0), v)
    assert set(worst) == {"J", "P", "E"}
    for p in plans:
        p.close()


def test_exec_batch_tuned_mode_bitwise_and_report(dev):
    """Batch mode 2: the first call times every stage-batched CTA shape and the persistent kernel
    and keeps the fastest; the report lists the 13 candidates, and the tuned batch (first call and
    replay) equals per-signal exec bit for bit."""
    ws = synth.batched_uneven(9, seed=31, n_min=300, n_max=6000)
    plans, xs, Js, Es, Ps = [], [], [], [], []
    for s_, wl in enumerate(ws):
        plans.append(pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32,
                              tapers=seeded_tapers(wl.K, wl.N, 60 + s_)))
        xs.append(torch.from_numpy(wl.x[0].astype(np.float32)).to(dev))
        Js.append(torch.empty((wl.K, wl.I), dtype=torch.complex64, device=dev))
        Es.append(torch.empty((wl.K, wl.I), dtype=torch.float32, device=dev))
        Ps.append(torch.empty((wl.I,), dtype=torch.float32, device=dev))
    prev = pkg.binding.set_batch_mode(2)
    try:
        for rep in range(2):  # tune + keep the fastest, then replay the cached graph
            for J in Js:
                J.zero_()
            pkg.exec_batch(plans, xs, Js, Es, Ps)
            torch.cuda.synchronize()
            for p, x, J, E, P in zip(plans, xs, Js, Es, Ps):
                single = p.run(x[None, :], want=("J", "E", "P"))
                torch.cuda.synchronize()
                assert torch.equal(single["J"][0], J) and torch.equal(single["E"][0], E)
                assert torch.equal(single["P"][0], P)
        table = pkg.binding.batch_tuning()
        assert len(table) == 13
        cfgs = {c for c, _ in table}
        assert (0, 2, 8, 32) in cfgs and (1, 2, 8, 32) in cfgs
        assert {c[1] for c in cfgs if c[0] == 0} == {1, 2, 4}
        assert all(0 < ms < 1e3 for _, ms in table)
    finally:
        pkg.binding.set_batch_mode(prev)
    with pytest.raises(ValueError):
        pkg.binding.set_batch_mode(3)


@pytest.mark.parametrize("path", [2, 3])
def test_permuted_sample_order_bitwise(dev, path):
    """Samples given in a shuffled order (times, tapers and x permuted alike): the plan spreads the
    points in time order whatever the caller's order, so J, |J|^2 and P-hat are bit-identical to the
    sorted input -- on the four-kernel path (whose spread copies a tile's contiguous run of samples
    when there is one and otherwise gathers them), the persistent kernel and the stage-batched
    executor -- and meet the oracle."""
    N, K, I = 3000, 6, 8192
    t = synth.jittered(N, 0.4, 44)
    X = np.stack([synth.white(t, 1.0, 50 + b) for b in range(3)])
    w = seeded_tapers(K, N, 12)
    perm = np.random.default_rng(3).permutation(N)
    args = (1.0, 3.0 / N, K, -0.5, 1.0 / I, I)
    ps = pkg.Plan(t, *args, precision=32, tapers=w, path=path)
    pp = pkg.Plan(t[perm], *args, precision=32, tapers=w[:, perm], path=path)
    a = run_plan(ps, X, dev)
    b = run_plan(pp, X[:, perm], dev)
    for k in ("J", "E", "P"):
        assert np.array_equal(a[k], b[k]), k
    Ps = [torch.empty((I,), dtype=torch.float32, device=dev) for _ in range(2)]
    xs = [torch.from_numpy(X[0].astype(np.float32)).to(dev), torch.from_numpy(X[0, perm].astype(np.float32)).to(dev)]
    pkg.exec_batch([ps, pp], xs, None, None, Ps)
    torch.cuda.synchronize()
    assert np.array_equal(Ps[0].cpu().numpy(), a["P"][0]) and np.array_equal(Ps[1].cpu().numpy(), a["P"][0])
    Jr, Pr = oracle_all(t, X, w, -0.5, 1.0 / I, I)
    check(b, Jr, Pr, w, X, 32)


def test_outputs_in_pinned_host_memory_bitwise(dev):
    """Output buffers in page-locked host memory: the kernels write J, |J|^2, P-hat (and L-hat / E-hat
    are copied) straight into host memory, bit-identical to device outputs -- for a multi-chunk exec
    on the four-kernel path and for the stage-batched executor."""
    wl = synth.workload("grid1024", batch=12)
    w, lam = ogpss.nominal_tapers(wl.t, wl.fs, wl.f_w, wl.K)
    plan = pkg.Plan(wl.t, wl.fs, wl.f_w, wl.K, wl.f_lo, wl.df, wl.I, precision=32, tapers=w, lam=lam, max_batch=4)
    assert plan.info["path"] == 2
    x = torch.from_numpy(wl.x.astype(np.float32)).to(dev)
    B, K, I = x.shape[0], wl.K, wl.I
    ref = plan.run(x, want=("J", "E", "P", "Lhat", "Ehat"))
    Jh = torch.empty((B, K, I), dtype=torch.complex64).pin_memory()
    Eh = torch.empty((B, K, I), dtype=torch.float32).pin_memory()
    Ph = torch.empty((B, I), dtype=torch.float32).pin_memory()
    Lh = torch.empty((K, I), dtype=torch.float64).pin_memory()
    Ah = torch.empty((I,), dtype=torch.float64).pin_memory()
    plan.exec(x, Jh, Eh, Ph, Lh, Ah)
    torch.cuda.synchronize()
    for got, want in ((Jh, ref["J"]), (Eh, ref["E"]), (Ph, ref["P"]), (Lh, ref["Lhat"]), (Ah, ref["Ehat"])):
        assert torch.equal(got, want.cpu())
    Pb = [torch.empty((I,), dtype=torch.float32).pin_memory() for _ in range(3)]
    pkg.exec_batch([plan] * 3, [x[b] for b in range(3)], None, None, Pb)
    torch.cuda.synchronize()
    assert all(torch.equal(Pb[b], ref["P"][b].cpu()) for b in range(3))
    with pytest.raises(ValueError):
        plan.exec(x, None, None, torch.empty((B, I), dtype=torch.float32))  # pageable host memory
    plan.close()
