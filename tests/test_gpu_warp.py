"""Warp-per-event schedule (GAPS_SCHED_WARP): every event identical to the
lane-per-event persistent kernel's without trial caching (same trials, draws,
winner, veto and emission arithmetic), for every process, the mixed batch,
capacity errors and the learned proposal."""
import numpy as np
import pytest

from tests.gpu_common import PROCESS, gaps, run_gpu

pytestmark = pytest.mark.gpu

MIX = [(2, 13600.0, 1.0, 0.5), (0, 91.2, 0.5, 0.25), (0, 500.0, 4.0, 0.25)]


@pytest.fixture(scope="module")
def G():
    return gaps()


def _same(a, b, keys=("p", "flav", "col", "acol", "npart", "status", "n_emit", "weight", "obs")):
    for k in keys:
        assert np.array_equal(a[k], b[k]), k
    for k in ("events", "steps", "trials", "isr_trials", "vetoes", "accepts", "violations"):
        assert a["stats"][k] == b["stats"][k], k


@pytest.mark.parametrize("name", ["ee91", "ee500", "pp_lo", "pp_nlo"])
@pytest.mark.parametrize("block,bps", [(128, 2), (64, 4), (256, 1)])
def test_warp_schedule_equals_lane_schedule(G, pdf, name, block, bps):
    proc, sqrt_s = PROCESS[name]
    n = 6007
    a = run_gpu(G, proc, sqrt_s, 1234, n, pdf, precision=1, schedule=1, trial_mode=G.GAPS_TRIALS_REDRAW)
    b = run_gpu(G, proc, sqrt_s, 1234, n, pdf, precision=1, schedule=2, block_size=block, blocks_per_sm=bps)
    _same(a, b)


def test_warp_schedule_mixed_batch(G, pdf):
    a = run_gpu(G, 0, 91.2, 99, 5003, pdf, precision=1, schedule=1, mix=MIX, trial_mode=G.GAPS_TRIALS_REDRAW)
    b = run_gpu(G, 0, 91.2, 99, 5003, pdf, precision=1, schedule=2, mix=MIX)
    _same(a, b)


def test_warp_schedule_capacity_errors(G, pdf):
    proc, sqrt_s = PROCESS["pp_nlo"]
    a = run_gpu(G, proc, sqrt_s, 0, 3001, pdf, nmax=6, precision=1, schedule=1, trial_mode=G.GAPS_TRIALS_REDRAW)
    b = run_gpu(G, proc, sqrt_s, 0, 3001, pdf, nmax=6, precision=1, schedule=2)
    assert (b["status"] == -2).sum() > 100
    _same(a, b)
    assert a["stats"]["err_capacity"] == b["stats"]["err_capacity"]


def test_warp_schedule_rejects_fp64(G, pdf):
    with pytest.raises(G.GapsError):
        G.gaps_init(G.make_config(0, 91.2, schedule=2, precision=0))


def test_warp_schedule_learned(G, pdf):
    """Same network and margins: identical events and counters (violations
    included) in both schedules."""
    import torch
    from paper_2511_19633_gb300 import learned
    proc, sqrt_s = PROCESS["pp_nlo"]
    cfg = G.make_config(proc, sqrt_s, pdf_grid=pdf, nmax=128, precision=1, schedule=1, trial_mode=G.GAPS_TRIALS_REDRAW)
    ctx = G.gaps_init(cfg)
    try:
        res = learned.train_and_install(ctx, first_event=7 << 40, n_events=1 << 18, capacity=1 << 18,
                                        steps=4000, holdout_events=1 << 17)
    finally:
        G.gaps_destroy(ctx)
    out = []
    for sched in (1, 2):
        cfg = G.make_config(proc, sqrt_s, pdf_grid=pdf, nmax=128, precision=1, schedule=sched,
                            trial_mode=G.GAPS_TRIALS_REDRAW)
        ctx = G.gaps_init(cfg)
        try:
            G.gaps_set_learned_proposal(ctx, res["params"], res["log_margins"])
            buf = G.EventBuffers.allocate(20000, 128)
            ev = buf.view()
            G.gaps_generate_hard(ctx, 5, 20000, ev)
            G.gaps_shower(ctx, 5, 20000, ev)
            torch.cuda.synchronize()
            h = buf.to_host(20000)
            h["stats"] = G.gaps_get_stats(ctx)
            out.append(h)
        finally:
            G.gaps_destroy(ctx)
    assert out[0]["stats"]["mlp_tiles"] == out[1]["stats"]["mlp_tiles"] > 0
    _same(out[0], out[1], keys=("p", "flav", "col", "acol", "npart", "status", "n_emit", "weight"))
