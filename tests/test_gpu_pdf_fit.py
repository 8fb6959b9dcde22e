"""The paper's percentile-fitted PDF-ratio overestimate (App. A.2, eqs. pdfmax
and pdfmax_ud) as a comparison mode of the mixed-precision shower.

The collection pass logs the PDF ratios the certified shower evaluates; every
logged ratio must lie under the oracle's certified bound of its transition.
The fit installed, the shower draws fewer trials, counts the acceptance
weights above one it meets (the fit is not a strict bound), and taking the
fit out again gives back the certified shower's events bit for bit."""
import numpy as np
import pytest

from tests.gpu_common import gaps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    return gaps()


def _ctx(G, pdf, schedule):
    cfg = G.make_config(2, 13600.0, pdf_grid=pdf, nmax=128, seed=1, precision=G.GAPS_MIXED, schedule=schedule)
    return G.gaps_init(cfg)


def _shower(G, ctx, buf, first, n):
    import torch
    ev = buf.view()
    G.gaps_reset_stats(ctx)
    G.gaps_generate_hard(ctx, first, n, ev)
    G.gaps_shower(ctx, first, n, ev)
    torch.cuda.synchronize()
    return buf.to_host(n), G.gaps_get_stats(ctx)


@pytest.fixture(scope="module")
def collected(G, pdf):
    import torch
    n = 1 << 17
    ctx = _ctx(G, pdf, G.GAPS_SCHED_PERSISTENT)
    try:
        buf = G.EventBuffers.allocate(n, 128)
        cap = 1 << 23
        samples = torch.full((cap, 4), -1.0, dtype=torch.float32, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        ev = buf.view()
        G.gaps_generate_hard(ctx, 1 << 36, n, ev)
        G.gaps_collect_pdf_ratios(ctx, 1 << 36, n, ev, samples, count, keep_fraction=0.25)
        torch.cuda.synchronize()
        m = int(count.item())
        st = G.gaps_get_stats(ctx)
    finally:
        G.gaps_destroy(ctx)
    assert 0 < m <= cap
    return samples[:m].cpu().numpy(), st


def test_collected_ratios_lie_under_the_certified_bound(oracle_mod, pdf, collected):
    s, st = collected
    assert st["violations"] == 0
    num, den = s[:, 0].astype(int), s[:, 1].astype(int)
    assert np.all((num >= 0) & (num <= 11) & (den >= 0) & (den <= 11))
    assert np.all(np.isfinite(s[:, 3])) and np.all(s[:, 3] >= 0.0)
    assert np.all((s[:, 2] > 0.0) & (s[:, 2] < 1.0))
    # a quarter of the winners' ratio evaluations (initial-state and
    # final-initial winners, about half of the cycles) are kept
    assert 0.05 * st["steps"] < s.shape[0] < 0.25 * st["steps"]
    rng = np.random.default_rng(0)
    for i in rng.choice(s.shape[0], 3000, replace=False):
        B = oracle_mod.pdf_bound(pdf, int(s[i, 0]), int(s[i, 1]), float(s[i, 2]))
        assert s[i, 3] <= B * (1 + 1e-4), (s[i], B)


def _three_runs(G, pdf, fit, schedule, n=1 << 18, first=3 << 36):
    """Certified bounds, the given fit, certified again, on the same events."""
    ctx = _ctx(G, pdf, schedule)
    try:
        buf = G.EventBuffers.allocate(n, 128)
        a, sa = _shower(G, ctx, buf, first, n)
        G.gaps_set_pdf_ratio_fit(ctx, fit)
        b, sb = _shower(G, ctx, buf, first, n)
        G.gaps_set_pdf_ratio_fit(ctx, None)
        c, sc = _shower(G, ctx, buf, first, n)
    finally:
        G.gaps_destroy(ctx)
    assert np.all(a["status"] == 1) and np.all(b["status"] == 1) and sa["violations"] == 0
    # taking the fit out gives back the certified shower bit for bit (the
    # buffer is reused: slots past an event's parton count hold stale data)
    for k in ("npart", "status", "n_emit", "weight"):
        assert np.array_equal(a[k], c[k]), k
    used = np.arange(a["flav"].shape[1])[None, :] < a["npart"][:, None]
    for k in ("p", "flav", "col", "acol"):
        assert np.array_equal(a[k][used], c[k][used]), k
    assert (sa["trials"], sa["accepts"]) == (sc["trials"], sc["accepts"])
    return sa, sb


@pytest.mark.parametrize("schedule", [1, 3])
def test_percentile_fit_counts_its_violations(G, pdf, collected, schedule):
    """The paper's fit from the collected ratios: a different trial count and
    few acceptance weights above one, each counted (at most the share of
    ratios above the 99th percentile)."""
    s, _ = collected
    fit = G.gaps_fit_pdf_ratios(s)
    assert np.count_nonzero(fit[:, :, 1]) >= 10
    assert np.all(fit[:, :, 0] <= fit[:, :, 1])
    sa, sb = _three_runs(G, pdf, fit, schedule)
    assert sb["trials"] != sa["trials"]
    assert sb["violations"] <= 0.01 * sb["steps"], sb
    print("trials per event: certified %.1f, fitted %.1f; violations %d" % (
        sa["trials"] / sa["events"], sb["trials"] / sb["events"], sb["violations"]))


def test_constant_fit_above_the_certified_bound_is_exact(G, oracle_mod, pdf):
    """A 'fit' that is flat at the largest certified bound of each transition
    (over a dense eta grid, times 1.05) bounds every ratio: no violation, and
    more trials than the eta-dependent certified bound."""
    etas = np.exp(np.linspace(np.log(1.1e-6), np.log(0.999), 1500))
    fit = np.zeros((12, 12, 2), dtype=np.float32)
    pairs = [(f, f) for f in range(11)] + [(0, f) for f in range(1, 11)] + [(f, 0) for f in range(1, 11)]
    for num, den in pairs:
        m = max(oracle_mod.pdf_bound(pdf, num, den, float(e)) for e in etas)
        fit[num, den] = 1.05 * m
    sa, sb = _three_runs(G, pdf, fit, 1, n=1 << 17)
    assert sb["violations"] == 0
    assert sb["trials"] > sa["trials"]
