"""Launch-shape autotuner for the mixed-precision shower.

Sweeps, on a sample of the workload, threads per block x resident blocks per
SM x refill (compaction) period x emission batch for the persistent schedule,
or block shape x wavefront passes x veto cycles per pass for the wavefront
schedule, timing gaps_shower with CUDA events, and returns the fastest shape
with the whole table. The sample
must give every lane of the widest grid several events (2^21 events for up to
155 648 lanes), or the tail of the launch decides. The paper
tunes a single block size for all its kernels by hand (Section 3.2); here the
persistent kernel's shape is tuned per workload.
"""
from __future__ import annotations

import itertools

import torch

from . import gaps as G

DEFAULT_GRID = {
    "block_size": (128, 256),
    "blocks_per_sm": (2, 4, 8),
    "refill_period": (1, 4),
    "emit_batch": (8, 16),
}
WAVE_GRID = {
    "block_size": (256,),
    "blocks_per_sm": (3, 4),
    "wave_veto_blocks_per_sm": (2, 3, 4),
    "wave_passes": (16, 24, 32),
    "wave_cycles": (64,),
    "refill_period": (1,),
    "emit_batch": (16,),
}


def time_shape(process, sqrt_s, pdf, shape: dict, n_events: int, precision=G.GAPS_MIXED,
               first: int = 1 << 44, reps: int = 1, mix=None, learned=None,
               schedule=G.GAPS_SCHED_PERSISTENT) -> dict:
    """Shower time of one launch shape; mix: rows of a mixed batch; learned:
    (params, log_margins) of the learned proposal."""
    uses_pdf = process or (mix and any(r[0] for r in mix))
    cfg = G.make_config(process, sqrt_s, pdf_grid=pdf if uses_pdf else None, nmax=128,
                        precision=precision, schedule=schedule, mix=mix, **shape)
    ctx = G.gaps_init(cfg)
    try:
        if learned is not None:
            G.gaps_set_learned_proposal(ctx, *learned)
        buf = G.EventBuffers.allocate(n_events, 128)
        ev = buf.view()
        s = torch.cuda.current_stream()
        best = float("inf")
        for r in range(reps + 1):
            f0 = first + r * n_events
            G.gaps_generate_hard(ctx, f0, n_events, ev, s)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(s)
            G.gaps_shower(ctx, f0, n_events, ev, s)
            b.record(s)
            torch.cuda.synchronize()
            if r:  # the first pass allocates the working set and warms up
                best = min(best, a.elapsed_time(b))
            else:
                G.gaps_reset_stats(ctx, s)
        st = G.gaps_get_stats(ctx, s)
    finally:
        G.gaps_destroy(ctx)
    return {**shape, "ms": best, "events_per_s": n_events / best * 1e3,
            "lane_efficiency": st["lane_steps"] / max(1, st["warp_steps"])}


def autotune(process, sqrt_s, pdf, n_events: int = 1 << 21, grid: dict | None = None,
             precision=G.GAPS_MIXED, mix=None, learned=None, schedule=G.GAPS_SCHED_PERSISTENT) -> dict:
    grid = grid or (WAVE_GRID if schedule == G.GAPS_SCHED_WAVE else DEFAULT_GRID)
    keys = list(grid)
    table = []
    for values in itertools.product(*(grid[k] for k in keys)):
        shape = dict(zip(keys, values))
        if shape.get("block_size", 128) * shape.get("blocks_per_sm", 1) > 2048:
            continue  # more threads than an SM holds
        table.append(time_shape(process, sqrt_s, pdf, shape, n_events, precision, mix=mix, learned=learned,
                                schedule=schedule))
    best = min(table, key=lambda r: r["ms"])
    return {"best": {k: best[k] for k in keys}, "best_events_per_s": best["events_per_s"],
            "sample_events": n_events, "table": table}
