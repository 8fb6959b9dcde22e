"""Mixed batch (50 % NLO pp -> Z at 13.6 TeV with t_c = 1 GeV^2, 25 % e+e- at
91.2 GeV with t_c = 0.5 GeV^2, 25 % e+e- at 500 GeV with t_c = 4 GeV^2) in one
launch: FP64 events bit-identical to the oracle's mixed batch, and the
mixed-precision persistent shower's histograms per row against the oracle's
one-process histograms of that row (chi^2/ndf < 1.2)."""
import numpy as np
import pytest

from tests.gpu_common import compare, gaps, identical, run_gpu
from tests.hist_common import chi2_per_hist, chi2_summary, load_golden

pytestmark = pytest.mark.gpu

MIX = [(2, 13600.0, 1.0, 0.5), (0, 91.2, 0.5, 0.25), (0, 500.0, 4.0, 0.25)]
GOLDEN_OF_ROW = ["pp_nlo", "ee91_tc0.5", "ee500_tc4"]


@pytest.fixture(scope="module")
def G():
    return gaps()


def _oracle_rows(O):
    return [O.Settings(process=p, sqrt_s=rs, t_cut=tc, nmax=128, seed=1) for p, rs, tc, _ in MIX]


@pytest.mark.parametrize("schedule", [0, 1])
def test_fp64_mixed_batch_is_bit_identical(G, oracle_mod, pdf, schedule):
    first, n = 12345, 3001
    g = run_gpu(G, 0, 91.2, first, n, pdf, schedule=schedule, blocks_per_sm=2 if schedule else 0, mix=MIX)
    o = oracle_mod.run_mix(_oracle_rows(oracle_mod), [r[3] for r in MIX], first, n, pdf, threads=8)
    assert set(np.unique(o["row"])) == {0, 1, 2}
    bad = identical(g, o)
    assert not bad, bad[:10]
    # observables go through libm on both sides: 1e-9 relative
    assert compare(g, o) == []


def test_mixed_precision_rows_follow_fp64(G, pdf, oracle_mod):
    """The GPU assigns the oracle's rows: event structure per row matches the
    one-process mixed-precision runs of that row."""
    first, n = 500, 4001
    g = run_gpu(G, 0, 91.2, first, n, pdf, precision=1, schedule=1, mix=MIX)
    rows = oracle_mod.mix_rows(1, [r[3] for r in MIX], first, n)
    for r, (proc, rs, tc, _) in enumerate(MIX):
        one = run_gpu(G, proc, rs, first, n, pdf, precision=1, schedule=1, t_cut=tc)
        sel = rows == r
        for k in ("p", "flav", "npart", "weight", "obs"):
            assert np.array_equal(g[k][sel], one[k][sel]), (r, k)


def test_mixed_batch_histograms_match_oracle_rows(G, pdf, oracle_mod):
    import os
    import torch
    from tests.hist_common import GOLDEN
    for name in GOLDEN_OF_ROW:
        if not os.path.exists(os.path.join(GOLDEN, "oracle_hists_%s.json" % name)):
            pytest.fail("reference histograms missing: run tests/golden/make_oracle_hists.py --only " + name)
    n, chunk = 10_000_000, 1 << 22
    cfg = G.make_config(0, 91.2, pdf_grid=pdf, nmax=128, seed=1, precision=1, schedule=1, mix=MIX)
    ctx = G.gaps_init(cfg)
    try:
        buf = G.EventBuffers.allocate(chunk, 128)
        ev = buf.view()
        hw = torch.zeros((len(MIX), G.GAPS_NHIST, G.GAPS_HIST_BINS), dtype=torch.float64, device="cuda")
        hw2 = torch.zeros_like(hw)
        hists = G.GapsHists(hw.data_ptr(), hw2.data_ptr())
        for first in range(0, n, chunk):
            m = min(chunk, n - first)
            G.gaps_generate_hard(ctx, first, m, ev)
            G.gaps_shower(ctx, first, m, ev)
            G.gaps_observables(ctx, first, m, ev, None, hists)
        torch.cuda.synchronize()
        binning = [G.gaps_hist_binning(ctx, h) for h in range(len(MIX) * G.GAPS_NHIST)]
        stats = G.gaps_get_stats(ctx)
    finally:
        G.gaps_destroy(ctx)
    assert stats["events"] == n and stats["violations"] == 0
    rows = oracle_mod.mix_rows(1, [r[3] for r in MIX], 0, n)
    w, w2 = hw.cpu().numpy(), hw2.cpu().numpy()
    for r, name in enumerate(GOLDEN_OF_ROW):
        gold = load_golden(name)
        for (lo, hi, nb, oi, lg), b in zip(gold["binning"], binning[r * G.GAPS_NHIST:(r + 1) * G.GAPS_NHIST]):
            assert (b["lo"], b["hi"], b["nbins"], b["obs"], int(b["log10"])) == pytest.approx((lo, hi, nb, oi, lg))
        n_r = int((rows == r).sum())
        red, chi2, ndf = chi2_summary(chi2_per_hist(w[r], w2[r], n_r, gold["sumw"], gold["sumw2"], gold["events"]))
        assert red < 1.2, (name, red)


def test_fp64_mixed_batch_with_dilepton_row_is_bit_identical(G, oracle_mod, pdf):
    """A batch mixing on-shell Z, Z/gamma* -> e+ e- and e+e- rows: FP64 events
    bit-identical to the oracle's mixed batch."""
    mix = [(2, 13600.0, 1.0, 0.4), (3, 13600.0, 1.0, 0.4), (0, 91.2, 1.0, 0.2)]
    first, n = 777, 3001
    g = run_gpu(G, 0, 91.2, first, n, pdf, mix=mix)
    rows = [oracle_mod.Settings(process=p, sqrt_s=rs, t_cut=tc, nmax=128, seed=1) for p, rs, tc, _ in mix]
    o = oracle_mod.run_mix(rows, [r[3] for r in mix], first, n, pdf, threads=8)
    assert set(np.unique(o["row"])) == {0, 1, 2}
    assert np.any(o["flav"][:, 2] == 11)
    bad = identical(g, o)
    assert not bad, bad[:10]
    assert compare(g, o) == []
