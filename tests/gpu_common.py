"""Helpers of the GPU parity tests: run the CUDA library through its C ABI
and compare records with the FP64 oracle event by event."""
from __future__ import annotations

import numpy as np

PROCESS = {"ee91": (0, 91.2), "ee500": (0, 500.0), "pp_lo": (1, 13600.0), "pp_nlo": (2, 13600.0),
           "pp_ll": (3, 13600.0)}


def gaps():
    from paper_2511_19633_gb300 import build
    build.build()
    from paper_2511_19633_gb300 import gaps as G
    return G


def run_gpu(G, process, sqrt_s, first, n, pdf, nmax=128, seed=1, schedule=0, block_size=0,
            blocks_per_sm=0, precision=0, t_cut=1.0, obs=True, refill_period=0, emit_batch=0, mix=None,
            trial_mode=None, max_cycles=0):
    import torch
    uses_pdf = process or (mix and any(r[0] for r in mix))
    cfg = G.make_config(process, sqrt_s, pdf_grid=pdf if uses_pdf else None, nmax=nmax, seed=seed,
                        schedule=schedule, block_size=block_size, blocks_per_sm=blocks_per_sm,
                        precision=precision, t_cut=t_cut, refill_period=refill_period,
                        emit_batch=emit_batch, mix=mix, trial_mode=trial_mode, max_cycles=max_cycles)
    ctx = G.gaps_init(cfg)
    try:
        buf = G.EventBuffers.allocate(max(n, 1), nmax)
        ev = buf.view()
        G.gaps_generate_hard(ctx, first, n, ev)
        G.gaps_shower(ctx, first, n, ev)
        o = None
        if obs:
            o = torch.zeros((G.GAPS_NOBS, max(n, 1)), dtype=torch.float64, device="cuda")
            G.gaps_observables(ctx, first, n, ev, o, None)
        torch.cuda.synchronize()
        host = buf.to_host(n)
        if obs:
            host["obs"] = o[:, :n].T.cpu().numpy()
        host["stats"] = G.gaps_get_stats(ctx)
    finally:
        G.gaps_destroy(ctx)
    return host


def run_oracle(O, process, sqrt_s, first, n, pdf, nmax=128, seed=1, threads=8, t_cut=1.0):
    st = O.Settings(process=process, sqrt_s=sqrt_s, nmax=nmax, seed=seed, t_cut=t_cut)
    return O.run(st, first, n, pdf if process else None, threads=threads)


def identical(gpu, orc):
    """Indices of events whose records are not bit-identical to the oracle's."""
    n = len(gpu["npart"])
    bad = []
    for e in range(n):
        m = int(orc["npart"][e])
        same = (gpu["npart"][e] == m and gpu["status"][e] == orc["status"][e]
                and np.array_equal(gpu["flav"][e, :m], orc["flav"][e, :m])
                and np.array_equal(gpu["col"][e, :m], orc["col"][e, :m])
                and np.array_equal(gpu["acol"][e, :m], orc["acol"][e, :m])
                and np.array_equal(gpu["p"][e, :m], orc["p"][e, :m])
                and gpu["weight"][e] == orc["weight"][e])
        if not same:
            bad.append(e)
    return bad


def compare(gpu, orc, rel=1e-12):
    """Indices of events that differ: structure (multiplicity, flavours,
    colours, status, emissions) exactly; momenta to rel x the largest energy of
    the event; weight and observables to rel relative."""
    n = len(gpu["npart"])
    bad = []
    for e in range(n):
        m = int(orc["npart"][e])
        ok = (gpu["npart"][e] == m and gpu["status"][e] == orc["status"][e]
              and gpu["n_emit"][e] == orc["n_emit"][e]
              and np.array_equal(gpu["flav"][e, :m], orc["flav"][e, :m])
              and np.array_equal(gpu["col"][e, :m], orc["col"][e, :m])
              and np.array_equal(gpu["acol"][e, :m], orc["acol"][e, :m]))
        if ok:
            pg, po = gpu["p"][e, :m], orc["p"][e, :m]
            scale = max(np.abs(po[:, 0]).max(), 1e-300)
            ok = np.abs(pg - po).max() <= rel * scale
        if ok:
            wg, wo = gpu["weight"][e], orc["weight"][e]
            ok = abs(wg - wo) <= rel * max(abs(wo), 1e-300)
        if ok and "obs" in gpu:
            og, oo = gpu["obs"][e], orc["obs"][e]
            ok = np.all(np.abs(og - oo) <= 1e-9 * np.maximum(1.0, np.abs(oo)))
        if not ok:
            bad.append(e)
    return bad
