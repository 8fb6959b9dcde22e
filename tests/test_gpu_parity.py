"""Parity of the CUDA library (through its C ABI) with the FP64 oracle, event
by event, for every process, launch schedule and the edge cases."""
import numpy as np
import pytest

from tests.gpu_common import PROCESS, compare, gaps, identical, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

# sizes the oracle finishes in seconds; not multiples of any block size
SIZES = {"ee91": 20011, "ee500": 6007, "pp_lo": 8009, "pp_nlo": 6007, "pp_ll": 8009}


@pytest.fixture(scope="module")
def G():
    return gaps()


def _max_mismatch(n):
    # per-event parity target: >= 99.99 % of events identical (near-ties of
    # libm rounding between the two evaluations are the only allowed cause)
    return int(1e-4 * n) + 1


@pytest.mark.parametrize("name", list(SIZES))
def test_fp64_per_event_parity(G, oracle_mod, pdf, name):
    proc, sqrt_s = PROCESS[name]
    n, first = SIZES[name], 1000
    g = run_gpu(G, proc, sqrt_s, first, n, pdf)
    o = run_oracle(oracle_mod, proc, sqrt_s, first, n, pdf)
    bad = compare(g, o)
    assert len(bad) <= _max_mismatch(n), ("mismatching events", bad[:20])
    assert np.all(g["status"] == 1)
    # both sides evaluate the same exactly rounded operations (their own
    # elementary functions, no FMA contraction): records are bit-identical
    not_exact = identical(g, o)
    assert not_exact == [], ("events not bit-identical", not_exact[:20])
    # counters: trials / vetoes / emissions summed over events agree
    if not bad:
        c = o["counters"].astype(np.int64).sum(0)
        st = g["stats"]
        assert st["events"] == n
        assert (st["steps"], st["trials"], st["isr_trials"], st["vetoes"], st["accepts"]) == tuple(c[:5])
        assert st["violations"] == 0


@pytest.mark.parametrize("schedule,block,bps", [(1, 128, 4), (1, 64, 8), (0, 32, 0), (0, 256, 0)])
def test_schedules_and_block_sizes_give_identical_events(G, pdf, schedule, block, bps):
    proc, sqrt_s = PROCESS["pp_nlo"]
    n = 3001
    ref = run_gpu(G, proc, sqrt_s, 7, n, pdf)
    g = run_gpu(G, proc, sqrt_s, 7, n, pdf, schedule=schedule, block_size=block, blocks_per_sm=bps)
    for k in ("p", "flav", "col", "acol", "npart", "weight", "obs", "n_emit"):
        assert np.array_equal(g[k], ref[k]), k


def test_chunking_does_not_change_events(G, pdf):
    proc, sqrt_s = PROCESS["pp_lo"]
    whole = run_gpu(G, proc, sqrt_s, 500, 1000, pdf)
    part = run_gpu(G, proc, sqrt_s, 700, 300, pdf)
    assert np.array_equal(whole["p"][200:500], part["p"])
    other = run_gpu(G, proc, sqrt_s, 500, 1000, pdf, seed=2)
    assert not np.array_equal(whole["p"], other["p"])


def test_capacity_errors_match_oracle(G, oracle_mod, pdf):
    proc, sqrt_s = PROCESS["pp_nlo"]
    n = 2003
    g = run_gpu(G, proc, sqrt_s, 0, n, pdf, nmax=6)
    o = run_oracle(oracle_mod, proc, sqrt_s, 0, n, pdf, nmax=6)
    assert np.array_equal(g["status"], o["status"])
    assert (g["status"] == -2).sum() > 100
    assert g["stats"]["err_capacity"] == (g["status"] == -2).sum()
    bad = compare(g, o)
    assert len(bad) <= _max_mismatch(n)


@pytest.mark.parametrize("n", [0, 1, 31, 33])
def test_tiny_and_empty_batches(G, oracle_mod, pdf, n):
    proc, sqrt_s = PROCESS["pp_nlo"]
    g = run_gpu(G, proc, sqrt_s, 123456789, n, pdf)
    assert g["stats"]["events"] == n
    if n:
        o = run_oracle(oracle_mod, proc, sqrt_s, 123456789, n, pdf, threads=1)
        assert compare(g, o) == []


def test_high_cutoff_and_large_event_ids(G, oracle_mod, pdf):
    proc, sqrt_s = PROCESS["ee500"]
    first = (1 << 40) + 17
    g = run_gpu(G, proc, sqrt_s, first, 2000, pdf, t_cut=4.0)
    o = run_oracle(oracle_mod, proc, sqrt_s, first, 2000, pdf, t_cut=4.0)
    assert len(compare(g, o)) <= _max_mismatch(2000)


@pytest.mark.parametrize("proc,sqrt_s,n,above,count", [(0, 1.0e5, 1003, 96, 50), (2, 13600.0, 3001, 48, 10)])
def test_high_multiplicity_events(G, oracle_mod, pdf, proc, sqrt_s, n, above, count):
    """The lowest cutoff (0.5 GeV^2) and, for e+e-, a 100 TeV collision:
    events up to the 128-slot capacity, so that the observables' clusterings
    run over every word of their pseudo-jet masks and the thrust over the
    candidate axes of up to 128 partons (some e+e- events end with the
    capacity error), event by event against the oracle."""
    g = run_gpu(G, proc, sqrt_s, 1000, n, pdf, t_cut=0.5)
    o = run_oracle(oracle_mod, proc, sqrt_s, 1000, n, pdf, t_cut=0.5)
    start = 2 if proc else 0
    coloured = np.array([np.sum(~np.isin(o["flav"][e, start:int(o["npart"][e])], (23, 11, -11)))
                         for e in range(n)])
    assert (coloured > above).sum() > count
    if proc == 0:
        assert (o["status"] == -2).sum() > 0
    assert np.array_equal(g["status"], o["status"])
    assert len(compare(g, o)) <= _max_mismatch(n)


@pytest.mark.parametrize("name", ["pp_lo", "pp_ll", "pp_nlo"])
def test_full_size_lo_sampled_against_oracle(G, oracle_mod, pdf, name):
    """pp -> Z and pp -> Z/gamma* -> e+ e- at LO and NLO-matched pp -> Z,
    full 1e6-event batches in the persistent FP64 launch: 2000 events spread
    over the batch are recomputed by the oracle one by one."""
    proc, sqrt_s = PROCESS[name]
    n = 1_000_000
    g = run_gpu(G, proc, sqrt_s, 0, n, pdf, schedule=1, block_size=128, blocks_per_sm=4, obs=True)
    assert g["stats"]["events"] == n and g["stats"]["violations"] == 0
    assert np.all(g["status"] == 1)
    rng = np.random.default_rng(4)
    idx = np.sort(rng.choice(n, 2000, replace=False))
    bad = []
    for e in idx:
        o = run_oracle(oracle_mod, proc, sqrt_s, int(e), 1, pdf, threads=1)
        sub = {k: v[e:e + 1] for k, v in g.items() if k != "stats"}
        if compare(sub, o):
            bad.append(int(e))
    assert len(bad) <= 1, bad


def test_invalid_events_view_is_rejected(G, pdf):
    import torch
    cfg = G.make_config(1, 13600.0, pdf_grid=pdf)
    ctx = G.gaps_init(cfg)
    try:
        buf = G.EventBuffers.allocate(16, 128)
        ev = buf.view()
        with pytest.raises(G.GapsError):
            G.gaps_shower(ctx, 0, 17, ev)          # n > capacity
        bad = G.EventBuffers.allocate(16, 64).view()
        with pytest.raises(G.GapsError):
            G.gaps_generate_hard(ctx, 0, 16, bad)  # nmax differs from the context
        torch.cuda.synchronize()
    finally:
        G.gaps_destroy(ctx)
