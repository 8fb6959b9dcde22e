"""The wavefront schedule (GAPS_SCHED_WAVE): end tables, veto cycles and
emissions as separate kernels over lists of live events, the trials of the
rebuilt ends drawn one end per lane, then the persistent kernel for the
events still live. Every event takes the same steps with the same random
numbers as in the persistent schedule, so the records are compared bit for
bit (the persistent schedule itself is checked against the oracle's
histograms in test_gpu_mixed.py and test_gpu_learned.py)."""
import numpy as np
import pytest

from tests.gpu_common import gaps

pytestmark = pytest.mark.gpu

MIX = [(2, 13600.0, 1.0, 0.5), (0, 91.2, 0.5, 0.25), (0, 500.0, 4.0, 0.25)]
COUNTERS = ("events", "steps", "trials", "isr_trials", "vetoes", "accepts", "violations", "err_capacity",
            "err_iter_cap", "err_numeric", "rebuilds", "mlp_tiles")


@pytest.fixture(scope="module")
def G():
    return gaps()


def _run(G, pdf, process, sqrt_s, first, n, schedule, learned=None, cap=None, **kw):
    import torch
    uses_pdf = process != 0 or any(r[0] for r in kw.get("mix") or [])
    cfg = G.make_config(process, sqrt_s, pdf_grid=pdf if uses_pdf else None, nmax=kw.pop("nmax", 128), seed=1,
                        precision=G.GAPS_MIXED, schedule=schedule, **kw)
    ctx = G.gaps_init(cfg)
    try:
        if learned is not None:
            G.gaps_set_learned_proposal(ctx, *learned)
        buf = G.EventBuffers.allocate(max(cap or n, 1), cfg.nmax_partons)
        ev = buf.view()
        G.gaps_generate_hard(ctx, first, n, ev)
        G.gaps_shower(ctx, first, n, ev)
        torch.cuda.synchronize()
        out = buf.to_host(n)
        out["stats"] = G.gaps_get_stats(ctx)
    finally:
        G.gaps_destroy(ctx)
    return out


def _same(a, b):
    for k in ("p", "flav", "col", "acol", "npart", "status", "n_emit", "weight", "t", "eta"):
        assert np.array_equal(a[k], b[k]), k
    for k in COUNTERS:
        assert a["stats"][k] == b["stats"][k], k


@pytest.mark.parametrize("name,process,sqrt_s", [("pp_nlo", 2, 13600.0), ("pp_lo", 1, 13600.0),
                                                 ("pp_ll", 3, 13600.0), ("ee91", 0, 91.2)])
def test_wave_equals_persistent(G, pdf, name, process, sqrt_s):
    n = 20000
    a = _run(G, pdf, process, sqrt_s, 777, n, G.GAPS_SCHED_PERSISTENT)
    b = _run(G, pdf, process, sqrt_s, 777, n, G.GAPS_SCHED_WAVE)
    assert np.all(b["status"] == 1)
    _same(a, b)


@pytest.mark.parametrize("passes", [0, 1, 3, 64])
def test_pass_count_does_not_change_events(G, pdf, passes):
    """0 passes: everything in the persistent kernel; 64: almost every event
    finishes inside the wavefront passes."""
    n = 6000
    a = _run(G, pdf, 2, 13600.0, 31, n, G.GAPS_SCHED_PERSISTENT)
    b = _run(G, pdf, 2, 13600.0, 31, n, G.GAPS_SCHED_WAVE, wave_passes=passes)
    _same(a, b)


@pytest.mark.parametrize("mode", [0, 2])
def test_wave_redraw_and_select_trials(G, pdf, mode):
    n = 6000
    a = _run(G, pdf, 2, 13600.0, 99, n, G.GAPS_SCHED_PERSISTENT, trial_mode=mode)
    b = _run(G, pdf, 2, 13600.0, 99, n, G.GAPS_SCHED_WAVE, trial_mode=mode)
    _same(a, b)


def test_wave_mixed_batch(G, pdf):
    n = 12000
    a = _run(G, pdf, 0, 91.2, 4242, n, G.GAPS_SCHED_PERSISTENT, mix=MIX)
    b = _run(G, pdf, 0, 91.2, 4242, n, G.GAPS_SCHED_WAVE, mix=MIX)
    _same(a, b)


def test_wave_learned_proposal_and_violation_fallback(G, pdf):
    """An untrained network with zero margins proposes heights below the true
    ratio in many bins: the violations and their plain-bound fallback happen
    in the same events and cycles in both schedules."""
    from paper_2511_19633_gb300 import learned
    params = learned.init_params(5)
    margins = np.zeros((G.GAPS_ISR_CLASSES, G.GAPS_ISR_ETA_BINS, G.GAPS_ISR_BINS), dtype=np.float32)
    n = 8000
    a = _run(G, pdf, 2, 13600.0, 5151, n, G.GAPS_SCHED_PERSISTENT, learned=(params, margins))
    b = _run(G, pdf, 2, 13600.0, 5151, n, G.GAPS_SCHED_WAVE, learned=(params, margins))
    assert a["stats"]["violations"] > 0 and a["stats"]["mlp_tiles"] > 0
    _same(a, b)


def test_wave_capacity_errors_and_ragged_chunk(G, pdf):
    """nmax = 8: many events end with GAPS_ERR_CAPACITY; the chunk is smaller
    than the buffer (ragged), and a single event and an empty call work."""
    n = 3001
    a = _run(G, pdf, 2, 13600.0, 1, n, G.GAPS_SCHED_PERSISTENT, nmax=8, cap=4096)
    b = _run(G, pdf, 2, 13600.0, 1, n, G.GAPS_SCHED_WAVE, nmax=8, cap=4096)
    assert np.any(b["status"] == G.GAPS_ERR_CAPACITY)
    _same(a, b)
    one_a = _run(G, pdf, 2, 13600.0, 17, 1, G.GAPS_SCHED_PERSISTENT)
    one_b = _run(G, pdf, 2, 13600.0, 17, 1, G.GAPS_SCHED_WAVE)
    _same(one_a, one_b)
    zero = _run(G, pdf, 2, 13600.0, 17, 0, G.GAPS_SCHED_WAVE, cap=16)
    assert zero["stats"]["events"] == 0


def test_wave_cycle_cap(G, pdf):
    n = 2000
    b = _run(G, pdf, 2, 13600.0, 0, n, G.GAPS_SCHED_WAVE, max_cycles=3)
    a = _run(G, pdf, 2, 13600.0, 0, n, G.GAPS_SCHED_PERSISTENT, max_cycles=3)
    assert np.mean(b["status"] == G.GAPS_ERR_ITER_CAP) > 0.9
    _same(a, b)


def test_wave_needs_mixed_precision(G, pdf):
    cfg = G.make_config(2, 13600.0, pdf_grid=pdf, precision=G.GAPS_FP64, schedule=G.GAPS_SCHED_WAVE)
    with pytest.raises(G.GapsError):
        G.gaps_init(cfg)
