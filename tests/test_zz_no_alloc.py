"""The allocation-free shower entry point, for callers that cannot allocate
device memory themselves. It must give the same events as the mixed-precision
gaps_shower on two calls in a row. Collected last on purpose."""
import numpy as np
import pytest

from tests.gpu_common import PROCESS, gaps

pytestmark = pytest.mark.gpu

NMAX = 32


@pytest.fixture(scope="module")
def G():
    return gaps()


def _records(G, buf, n):
    h = buf.to_host(n)
    return {k: h[k] for k in ("p", "flav", "col", "acol", "npart", "status", "n_emit", "weight", "eta")}


@pytest.mark.parametrize("name", ["pp_nlo", "ee91"])
def test_static_entry_point_matches_gaps_shower(G, pdf, name):
    import torch
    proc, sqrt_s = PROCESS[name]
    n = 20011
    cfg = G.make_config(proc, sqrt_s, pdf_grid=pdf if proc else None, nmax=NMAX, seed=1,
                        precision=G.GAPS_MIXED, schedule=G.GAPS_SCHED_PERSISTENT)
    ctx = G.gaps_init(cfg)
    try:
        for first in (0, 5_000_000):  # two calls in a row
            a = G.EventBuffers.allocate(n, NMAX)
            b = G.EventBuffers.allocate(n, NMAX)
            G.gaps_generate_hard(ctx, first, n, a.view())
            G.gaps_generate_hard(ctx, first, n, b.view())
            G.gaps_reset_stats(ctx)
            G.gaps_shower(ctx, first, n, a.view())
            ref_stats = G.gaps_get_stats(ctx)
            st = G.gaps_shower_static(cfg, first, n, b.view())
            torch.cuda.synchronize()
            ra, rb = _records(G, a, n), _records(G, b, n)
            for k in ra:
                assert np.array_equal(ra[k], rb[k]), (first, k)
            for k in ("events", "steps", "trials", "accepts", "vetoes", "err_capacity"):
                assert st[k] == ref_stats[k], (first, k)
            assert st["events"] == n
    finally:
        G.gaps_destroy(ctx)


def test_static_entry_point_rejects_large_records(G, pdf):
    cfg = G.make_config(2, 13600.0, pdf_grid=pdf, nmax=64, precision=G.GAPS_MIXED)
    buf = G.EventBuffers.allocate(16, 64)
    with pytest.raises(G.GapsError) as e:
        G.gaps_shower_static(cfg, 0, 16, buf.view())
    assert e.value.code == G.GAPS_ERR_INVALID_ARG
