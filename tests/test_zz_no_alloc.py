"""The allocation-free leakage entry point (m2nufft_leakage_static), for
callers that may not call cudaMalloc, gives the same L-hat / E-hat as the
plan's own computation (m2nufft_plan_with_tapers + m2nufft_get_leakage).

Two calls in a row with different problems share the library's static
scratch; each must match.  This file is collected last on purpose."""
import numpy as np
import pytest

import synth
from oracle import gpss as ogpss
from oracle import leakage as oleak
from tests._util import TOL

torch = pytest.importorskip("torch")
pkg = pytest.importorskip("paper_2407_01943_gb300")
from paper_2407_01943_gb300 import binding  # noqa: E402

pytestmark = pytest.mark.gpu


def _case(t, fw, K, I, f_lo=-0.5):
    w, lam = ogpss.nominal_tapers(t, 1.0, fw, K)
    plan = pkg.Plan(t, 1.0, fw, K, f_lo, 1.0 / I, I, precision=64, tapers=w, lam=lam)
    L_ref, E_ref = plan.leakage()
    plan.close()
    return w, lam, L_ref, E_ref


def test_leakage_static_matches_plan_two_calls():
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    cases = [
        (synth.jittered(300, 0.4, 31), 4.0 / 300, 4, 512),
        (synth.scaled_missing(60, 10, 5.0 / 6.0, 0), 0.05, 3, 200),
    ]
    for t, fw, K, I in cases:
        w, lam, L_ref, E_ref = _case(t, fw, K, I)
        td = torch.from_numpy(t).to(dev)
        wd = torch.from_numpy(np.ascontiguousarray(w)).to(dev)
        ld = torch.from_numpy(lam).to(dev)
        Lh = torch.empty((K, I), dtype=torch.float64, device=dev)
        Eh = torch.empty((I,), dtype=torch.float64, device=dev)
        binding.leakage_static(td, wd, ld, 1.0, fw, -0.5, 1.0 / I, I, Lh, Eh)
        torch.cuda.synchronize()
        L = Lh.cpu().numpy()
        E = Eh.cpu().numpy()
        scale = max(np.max(np.abs(L_ref)), 1e-300)
        assert np.max(np.abs(L - L_ref)) <= TOL[64] * scale
        assert np.max(np.abs(E - E_ref)) <= TOL[64] * scale
        # and against the oracle's dense pair sum, at every band
        Lo, Eo = oleak.leakage_at(t, w, lam, 1.0, fw, -0.5 + np.arange(I) / I)
        np.testing.assert_allclose(L, Lo, rtol=1e-9, atol=1e-13)
        np.testing.assert_allclose(E, Eo, rtol=1e-9, atol=1e-13)


def test_leakage_static_rejects_oversized():
    dev = torch.device("cuda:0")
    t = torch.arange(100, dtype=torch.float64, device=dev)
    w = torch.ones((16, 100), dtype=torch.float64, device=dev)
    lam = torch.ones((16,), dtype=torch.float64, device=dev)
    I = 1 << 20  # K * I above the 32 MiB scratch
    Lh = torch.empty((1,), dtype=torch.float64, device=dev)
    with pytest.raises(pkg.M2Error) as e:
        binding.leakage_static(t, w, lam, 1.0, 0.05, -0.5, 1.0 / I, I, Lh, Lh)
    assert e.value.status == 1
