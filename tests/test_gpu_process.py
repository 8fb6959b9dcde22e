"""gaps_process: the whole path over several chunks as one CUDA graph gives
the same records, observables and histograms as the per-call entry points,
also when the graph is reused for another event range."""
import numpy as np
import pytest

from tests.gpu_common import PROCESS, gaps

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    return gaps()


def _per_call(G, ctx, first, n, chunk, ev, obs, hists):
    import torch
    out = np.zeros((G.GAPS_NOBS, n))
    for f0 in range(0, n, chunk):
        m = min(chunk, n - f0)
        G.gaps_generate_hard(ctx, first + f0, m, ev)
        G.gaps_shower(ctx, first + f0, m, ev)
        G.gaps_observables(ctx, first + f0, m, ev, obs, hists)
        torch.cuda.synchronize()
        out[:, f0:f0 + m] = obs[:, :m].cpu().numpy()
    return out


@pytest.mark.parametrize("precision,schedule", [(0, 1), (1, 1), (1, 3)])
def test_graph_equals_per_call(G, pdf, precision, schedule):
    """(1, 3): the wavefront schedule, whose graph runs every other chunk in a
    second slot on a second stream."""
    import torch
    proc, sqrt_s = PROCESS["pp_nlo"]
    n, chunk = 25_000, 8192  # four chunks, the last one ragged
    cfg = G.make_config(proc, sqrt_s, pdf_grid=pdf, nmax=128, precision=precision, schedule=schedule,
                        blocks_per_sm=2)
    ctx_a, ctx_b = G.gaps_init(cfg), G.gaps_init(cfg)
    try:
        buf = G.EventBuffers.allocate(chunk, 128)
        ev = buf.view()
        obs = torch.zeros((G.GAPS_NOBS, chunk), dtype=torch.float64, device="cuda")
        ha = [torch.zeros((G.GAPS_NHIST, G.GAPS_HIST_BINS), dtype=torch.float64, device="cuda") for _ in range(2)]
        hb = [torch.zeros_like(ha[0]) for _ in range(2)]
        for first in (0, 777_777):  # the second range reuses the graph
            for h in ha + hb:
                h.zero_()
            ref = _per_call(G, ctx_a, first, n, chunk, ev, obs, G.GapsHists(ha[0].data_ptr(), ha[1].data_ptr()))
            host = torch.empty((G.GAPS_NOBS, n), dtype=torch.float64).pin_memory()
            G.gaps_process(ctx_b, first, n, ev, obs, host, G.GapsHists(hb[0].data_ptr(), hb[1].data_ptr()))
            torch.cuda.synchronize()
            assert np.array_equal(host.numpy(), ref)
            assert torch.equal(ha[0], hb[0]) or np.allclose(ha[0].cpu(), hb[0].cpu(), rtol=1e-12)
            assert np.allclose(ha[1].cpu(), hb[1].cpu(), rtol=1e-12)
            ms = G.gaps_process_shower_ms(ctx_b)
            assert len(ms) == 4 and all(t > 0 for t in ms)
        sa, sb = G.gaps_get_stats(ctx_a), G.gaps_get_stats(ctx_b)
        assert sa["events"] == sb["events"] == 2 * n and sa["steps"] == sb["steps"]
    finally:
        G.gaps_destroy(ctx_a)
        G.gaps_destroy(ctx_b)


def test_graph_rejects_bad_arguments(G, pdf):
    import torch
    cfg = G.make_config(0, 91.2, nmax=16)
    ctx = G.gaps_init(cfg)
    try:
        buf = G.EventBuffers.allocate(64, 16)
        ev = buf.view()
        host = torch.empty((G.GAPS_NOBS, 64), dtype=torch.float64).pin_memory()
        with pytest.raises(G.GapsError):
            G.gaps_process(ctx, 0, 64, ev, None, host, None)  # host copy needs device staging
        G.gaps_process(ctx, 0, 0, ev)  # nothing to do
    finally:
        G.gaps_destroy(ctx)
