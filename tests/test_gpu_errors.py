"""Device-side error paths: an event that reaches the veto-cycle cap ends
with GAPS_ERR_ITER_CAP (per event and in the counters), the launch returns,
and the context stays usable."""
import numpy as np
import pytest

from tests.gpu_common import gaps, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,schedule", [(0, 0), (0, 1), (1, 1)])
def test_cycle_cap_ends_events_with_iter_cap(pdf, precision, schedule):
    G = gaps()
    n = 3000
    cap = 3
    g = run_gpu(G, 2, 13600.0, 0, n, pdf, precision=precision, schedule=schedule, obs=False,
                max_cycles=cap)
    st = g["stats"]
    capped = g["status"] == G.GAPS_ERR_ITER_CAP
    # with three cycles almost every NLO event is still evolving
    assert capped.mean() > 0.9
    assert np.all((g["status"] == 1) | capped)
    assert st["err_iter_cap"] == int(capped.sum()) and st["events"] == n
    assert st["steps"] <= cap * n
    # the same events without the cap all finish
    h = run_gpu(G, 2, 13600.0, 0, n, pdf, precision=precision, schedule=schedule, obs=False)
    assert np.all(h["status"] == 1) and h["stats"]["err_iter_cap"] == 0
