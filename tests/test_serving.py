"""Continuous-batching server: every request completes, and each result is
the same alone (one exec with B = 1) and in the mix (batched with other
requests and patterns, several slots in flight)."""
import numpy as np
import pytest

import synth
from oracle import estimator as oest
from tests._util import TOL, assert_elementwise, packed_edge_bands, rel_l2, sample_bands, source_l1

torch = pytest.importorskip("torch")
pkg = pytest.importorskip("paper_2407_01943_gb300")
from paper_2407_01943_gb300 import serve  # noqa: E402

pytestmark = pytest.mark.gpu


def _patterns(n=6, path=0):
    pats = synth.serving_patterns(n, seed=5, n_min=300, n_max=1500)
    plans = {}
    for i, pt in enumerate(pats):
        plans[i] = pkg.Plan(pt["t"], 1.0, pt["f_w"], 4, pt["f_lo"], pt["df"], pt["I"], precision=32,
                            tapers=synth.taper_like(4, pt["t"].shape[0], i), max_batch=8, path=path)
    return pats, plans


@pytest.mark.parametrize("path", [0, 1], ids=["cross_pattern", "per_pattern"])
def test_server_results_equal_alone(path):
    """path 0: packed plans, so each launch runs all its requests (any patterns) through the
    stage-batched kernels; path 1: generic plans, grouped by pattern into m2nufft_exec calls."""
    torch.cuda.set_device(0)
    pats, plans = _patterns(path=path)
    arr = synth.poisson_arrivals(20000.0, 80, seed=3)   # bursty: batches of several requests form
    rng = np.random.default_rng(4)
    reqs = []
    for k, a in enumerate(arr):
        pid = int(rng.integers(0, len(pats)))
        N = pats[pid]["t"].shape[0]
        reqs.append(serve.Request(k, pid, rng.standard_normal(N).astype(np.float32), float(a)))
    srv = serve.PSDServer(plans, mem_budget=2 << 30, slots=3, max_batch=6)
    stats = srv.serve(reqs)
    assert stats["launches"] < 80  # requests were batched
    assert stats["requests"] == 80 and stats["p99_ms"] > 0
    for r in reqs:
        assert r.done >= r.arrival and r.P is not None
        p = plans[r.pattern]
        x = torch.from_numpy(r.x[None, :]).cuda()
        alone = p.run(x, want=("P",))["P"].cpu().numpy()[0]
        assert np.array_equal(alone, r.P)
        assert rel_l2(r.P, alone) <= TOL[32]
    # served P-hat against the oracle (Eq. power_spectrum_estimator with the plan's tapers) on a
    # sample of requests, at sampled bands plus the packed path's special positions
    for r in reqs[::10]:
        p = plans[r.pattern]
        pt = pats[r.pattern]
        w = synth.taper_like(4, pt["t"].shape[0], r.pattern)  # the tapers the plan was made with
        idx = np.union1d(sample_bands(p.I, 64, r.rid), packed_edge_bands(p.I, p.info["n1"]))
        Jr, _, Pr = oest.m2nufft(pt["t"], r.x.astype(np.float64), w, pt["f_lo"], pt["df"], p.I, idx)
        assert rel_l2(r.P[idx], Pr) <= TOL[32]
        assert_elementwise(None, Jr[None], source_l1(w, r.x.astype(np.float64)), TOL[32], r.P[idx][None], Pr[None])
    # the plain path on the same server gives the same results too
    plain_reqs = [serve.Request(r.rid, r.pattern, r.x, r.arrival) for r in reqs]
    srv.serve_plain(plain_reqs)
    for a, b in zip(reqs, plain_reqs):
        assert np.array_equal(a.P, b.P)
    srv.close()
    for p in plans.values():
        p.close()


def test_server_respects_memory_budget():
    torch.cuda.set_device(0)
    pats, plans = _patterns(2)
    srv = serve.PSDServer(plans, mem_budget=sum(p.info["device_bytes"] for p in plans.values())
                          + 3 * srv_bytes(plans), slots=2, max_batch=8)
    rng = np.random.default_rng(0)
    reqs = [serve.Request(k, k % 2, rng.standard_normal(pats[k % 2]["t"].shape[0]).astype(np.float32), 0.0)
            for k in range(10)]
    stats = srv.serve(reqs)
    assert stats["requests"] == 10
    srv.close()
    with pytest.raises(pkg.M2Error) as e:  # not even one request per slot fits
        serve.PSDServer(plans, mem_budget=sum(p.info["device_bytes"] for p in plans.values()) + 1000, slots=2)
    assert e.value.status == 3
    for p in plans.values():
        p.close()


def srv_bytes(plans):
    """Upper bound of one request's device bytes: samples, outputs, and for the cross-pattern
    launches of packed plans its workspace (spread grids, column and row transforms) and work maps."""
    return max(p.N * 4 + p.I * 4 + p.K * p.I * 12
               + ((p.K + 1) // 2) * (p.info["rows"] * 1024 + 2 * p.info["nf"]) * 8 + (1 << 20)
               for p in plans.values())
