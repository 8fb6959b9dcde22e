"""The heavy-quark measure correction (App. A.2) on the GPU, with the
thresholded synthetic table: FP64 events bit-identical to the oracle's, the
mixed-precision wavefront identical to the persistent kernel, and the
mixed-precision histograms against the oracle's (chi^2/ndf)."""
import os

import numpy as np
import pytest

from tests.gpu_common import compare, gaps, identical, run_gpu, run_oracle
from tests.hist_common import GOLDEN, chi2_per_hist, chi2_summary, load_golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    return gaps()


@pytest.fixture(scope="module")
def hq_pdf():
    from paper_2511_19633_gb300 import inputs
    return inputs.synthetic_pdf_grid(thresholds=True)


@pytest.mark.parametrize("process,schedule", [(2, 0), (2, 1), (1, 0)])
def test_fp64_heavy_quark_parity(G, oracle_mod, hq_pdf, process, schedule):
    n, first = 6007, 2024
    g = run_gpu(G, process, 13600.0, first, n, hq_pdf, schedule=schedule, blocks_per_sm=2 if schedule else 0)
    o = run_oracle(oracle_mod, process, 13600.0, first, n, hq_pdf)
    assert np.all(g["status"] == 1)
    # events with an incoming heavy quark are present, and some convert
    assert np.isin(np.abs(o["flav"][:, :2]), [4, 5]).sum() > 0
    assert identical(g, o) == []
    assert compare(g, o) == []
    c = o["counters"].astype(np.int64).sum(0)
    st = g["stats"]
    assert (st["steps"], st["trials"], st["isr_trials"], st["vetoes"], st["accepts"]) == tuple(c[:5])
    assert st["violations"] == 0


def _mixed(G, pdf, n, schedule, first=0, trial_mode=None):
    import torch
    cfg = G.make_config(2, 13600.0, pdf_grid=pdf, nmax=128, seed=1, precision=G.GAPS_MIXED, schedule=schedule,
                        trial_mode=trial_mode)
    ctx = G.gaps_init(cfg)
    try:
        cap = min(n, 1 << 20)
        buf = G.EventBuffers.allocate(cap, 128)
        ev = buf.view()
        hw = torch.zeros((G.GAPS_NHIST, G.GAPS_HIST_BINS), dtype=torch.float64, device="cuda")
        hw2 = torch.zeros_like(hw)
        hists = G.GapsHists(hw.data_ptr(), hw2.data_ptr())
        last = None
        for f0 in range(0, n, cap):
            m = min(cap, n - f0)
            G.gaps_generate_hard(ctx, first + f0, m, ev)
            G.gaps_shower(ctx, first + f0, m, ev)
            G.gaps_observables(ctx, first + f0, m, ev, None, hists)
            if f0 == 0:
                torch.cuda.synchronize()
                last = buf.to_host(min(m, 20000))
        torch.cuda.synchronize()
        st = G.gaps_get_stats(ctx)
    finally:
        G.gaps_destroy(ctx)
    return hw.cpu().numpy(), hw2.cpu().numpy(), st, last


def test_mixed_wave_equals_persistent_with_thresholds(G, hq_pdf):
    n = 20000
    a = _mixed(G, hq_pdf, n, G.GAPS_SCHED_PERSISTENT)
    b = _mixed(G, hq_pdf, n, G.GAPS_SCHED_WAVE)
    for k in ("p", "flav", "col", "acol", "npart", "status", "n_emit", "weight"):
        assert np.array_equal(a[3][k], b[3][k]), k
    for k in ("events", "steps", "trials", "vetoes", "accepts", "violations"):
        assert a[2][k] == b[2][k], k
    assert a[2]["violations"] == 0 and np.all(a[3]["status"] == 1)


def test_mixed_histograms_with_thresholds_match_oracle(G, hq_pdf):
    path = os.path.join(GOLDEN, "oracle_hists_pp_nlo_hq.json")
    if not os.path.exists(path):
        pytest.fail("reference histograms missing: run tests/golden/make_oracle_hists.py --only pp_nlo_hq")
    gold = load_golden("pp_nlo_hq")
    n = gold["events"]
    w, w2, st, _ = _mixed(G, hq_pdf, n, G.GAPS_SCHED_WAVE, first=5 << 40)
    assert st["events"] == n and st["violations"] == 0
    per = chi2_per_hist(w, w2, n, gold["sumw"], gold["sumw2"], gold["events"])
    red, _, _ = chi2_summary(per)
    # one sample of 2e6 events against 2e6 oracle events, about 200 degrees of
    # freedom: a correct generator exceeds 1.3 with probability ~1e-4
    assert red < 1.3, (red, per)
