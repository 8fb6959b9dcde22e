"""Benchmark: showered events per second on GB300.

One step = one pass of the whole hot path over one batch of synthetic events:
hard process, shower and observables with histogram filling, all in the CUDA
library, with the batch's records resident in HBM. Different steps use
different event ranges (no cached work). Prints one JSON line on rank 0.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank showers its own event range (independent
events, weak scaling, no data-path collective); the time is the maximum over
ranks and the value is all ranks' events divided by it.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "showered events/sec on 1 GB300 (learned+compacted vs plain GPU) at oracle-matched chi2/ndf<1.2"

MIX_ROWS = [(2, 13600.0, 1.0, 0.5), (0, 91.2, 0.5, 0.25), (0, 500.0, 4.0, 0.25)]

WORKLOADS = {
    # name: (process, sqrt_s, events per step, chunk, precision, mixed-batch rows, description)
    "pp_nlo_1e7": (2, 13600.0, 10_000_000, 1 << 22, 1, None,
                   "NLO-matched pp -> Z at 13.6 TeV, synthetic 100x50 PDF, 1e7 events per step in "
                   "chunks of 2^22, FP32 trials/PDF + FP64 kinematics, learned initial-state proposal, "
                   "wavefront shower over live-event lists, one CUDA graph per step"),
    "pp_lo_1e6_fp64": (1, 13600.0, 1_000_000, 1_000_000, 0, None,
                       "pp -> Z at 13.6 TeV, LO + initial/final-state shower, synthetic 100x50 PDF, "
                       "1e6 events, FP64 (per-event oracle parity)"),
    "ee91_1e4_fp64": (0, 91.2, 10_000, 10_000, 0, None,
                      "e+e- -> q qbar at 91.2 GeV, final-state shower, 1e4 events, FP64"),
    "pp_ll_1e7": (3, 13600.0, 10_000_000, 1 << 22, 1, None,
                  "pp -> Z/gamma* -> e- e+ at 13.6 TeV, LO with the Z/gamma interference, dilepton "
                  "mass 66-116 GeV, initial/final-state shower, synthetic 100x50 PDF, 1e7 events per "
                  "step in chunks of 2^22, mixed precision, learned proposal, one CUDA graph per step"),
    "mix_1e8": (2, 13600.0, 100_000_000, 1 << 22, 1, MIX_ROWS,
                "mixed batch, rows drawn per event inside every launch: 50% NLO pp -> Z at 13.6 TeV "
                "(t_c 1 GeV^2), 25% e+e- at 91.2 GeV (t_c 0.5), 25% e+e- at 500 GeV (t_c 4), "
                "1e8 events in chunks of 2^22, learned proposal, one CUDA graph per step"),
}
DEFAULT_WORKLOAD = "pp_nlo_1e7"
# the kernel that dominates a step of the mixed-precision path
SHOWER_KERNEL = "k_shower_mixed"

# Algorithmic work per unit, as the scope of the measurement defines it: a
# dipole trial is a log, an exp, a log for the z sample and about 25 FMA
# (28 operations, a transcendental counting as one); an initial-state trial adds
# two bilinear PDF interpolations (about 20 operations and 4 gathers each, 48);
# an accepted emission about 300 FP64 operations of kinematics. The counts are
# the library's counters of the timed run.
ALG_OPS_PER_TRIAL = 28.0
ALG_OPS_PER_ISR_TRIAL = 48.0
ALG_OPS_PER_ACCEPT = 300.0
# FP64 path: FLOP per trial / initial-state trial / cycle / accepted emission,
# a log, exp or sqrt counting as 20 FLOP (the FP64 kernel's own arithmetic).
FLOP_PER_TRIAL = 85.0
FLOP_PER_ISR_TRIAL = 16.0
FLOP_PER_STEP = 160.0
FLOP_PER_ACCEPT = 300.0
# Mixed path, implementation count: 32-bit operations per trial (Philox-4x32-10:
# 10 rounds of two 32x32->64 products, two 3-input XORs and two key additions =
# 60; uniform, log, FMA, compare 7), per cycle (FP32 veto: limits, maps, kernel,
# two PDF interpolations, alpha_s) and per accepted emission (FP64 kinematics and
# the end-table rebuild, each operation counted once).
OPS_PER_TRIAL = 67.0
OPS_PER_STEP = 190.0
OPS_PER_ACCEPT = 1200.0
# Nominal figures, used only when the microbenchmarks cannot run: 152 SMs x
# 128 FP32 lanes x 2.07 GHz, and 1.25 TFLOP/s FP64 (dense).
LANE_PEAK_TOPS_NOMINAL = 152 * 128 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS_NOMINAL = 1.25
# DRAM bytes (read + write) per event of the shower phase (every kernel of the
# wavefront between the hard process and the observables), from one ncu
# capture of the current kernels on a 262 144-event case of the same workload
# (the traffic grows with the events showered); scaled to a chunk by its
# events. Workloads and variants without a capture report null.
SHOWER_DRAM_BYTES_PER_EVENT = {
    ("pp_nlo_1e7", True): (14015.0e6 + 4602.4e6) / 262144,   # learned proposal, wavefront
}


def fp64_flops(stats: dict) -> float:
    return (stats["trials"] * FLOP_PER_TRIAL + stats["isr_trials"] * FLOP_PER_ISR_TRIAL
            + stats["steps"] * FLOP_PER_STEP + stats["accepts"] * FLOP_PER_ACCEPT)


def implementation_ops_mixed(stats: dict) -> float:
    return stats["trials"] * OPS_PER_TRIAL + stats["steps"] * OPS_PER_STEP + stats["accepts"] * OPS_PER_ACCEPT


def algorithmic_ops(stats: dict) -> float:
    return (stats["trials"] * ALG_OPS_PER_TRIAL + stats["isr_trials"] * ALG_OPS_PER_ISR_TRIAL
            + stats["accepts"] * ALG_OPS_PER_ACCEPT)


def alu_peaks(G) -> dict:
    """Instruction throughput of the FP32, FP64, special-function and integer
    pipes, from the library's own microbenchmarks on this GPU, with the SM
    clock sampled while they run."""
    out = {}
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for name, kind, iters in (("ffma", G.GAPS_PEAK_FFMA, 32768), ("dfma", G.GAPS_PEAK_DFMA, 256),
                                  ("mufu", G.GAPS_PEAK_MUFU, 4096), ("imad", G.GAPS_PEAK_IMAD, 16384)):
            r = G.gaps_alu_peak(kind, iters)
            out[name + "_per_s"] = r["ops_per_s"]
            out[name + "_ms"] = r["ms"]
    out["clocks"] = clk.summary()
    return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_first_event(rank: int, step: int, events_per_step: int, steps_total: int) -> int:
    """Event range of (rank, step): ranks own disjoint contiguous blocks."""
    from paper_2511_19633_gb300.sharding import rank_first_event as first
    return first(rank, step, events_per_step, steps_total)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def _oracle_run(O, rows, fractions, first, n, pdf, cores, chunk=50_000):
    """Runs the oracle over n events in chunks (bounded host memory)."""
    for f0 in range(0, n, chunk):
        m = min(chunk, n - f0)
        if len(rows) == 1:
            O.run(rows[0], first + f0, m, pdf if rows[0].process else None, threads=cores)
        else:
            O.run_mix(rows, fractions, first + f0, m, pdf, threads=cores)


def _oracle_rows(O, process, sqrt_s, mix):
    if mix:
        return ([O.Settings(process=p, sqrt_s=rs, t_cut=tc, nmax=128) for p, rs, tc, _ in mix],
                [r[3] for r in mix])
    return [O.Settings(process=process, sqrt_s=sqrt_s, nmax=128)], [1.0]


def cpu_baseline(process: int, sqrt_s: float, mix=None, target_s: float = 12.0) -> dict:
    """The FP64 oracle as it stands, on all host cores, over a bounded sample."""
    from oracle import oracle as O
    from paper_2511_19633_gb300 import inputs
    pdf = inputs.synthetic_pdf_grid()
    cores = os.cpu_count() or 1
    rows, fr = _oracle_rows(O, process, sqrt_s, mix)
    probe = 500 * cores
    t0 = time.perf_counter()
    _oracle_run(O, rows, fr, 10_000_000_000, probe, pdf, cores)
    dt = time.perf_counter() - t0
    n = max(probe, int(probe * target_s / max(dt, 1e-3)))
    t0 = time.perf_counter()
    _oracle_run(O, rows, fr, 20_000_000_000, n, pdf, cores)
    dt = time.perf_counter() - t0
    # the oracle as written, on one thread, over a smaller sample
    n1 = max(200, int(n / cores * 0.4))
    t1 = time.perf_counter()
    _oracle_run(O, rows, fr, 21_000_000_000, n1, pdf, 1)
    dt1 = time.perf_counter() - t1
    return {"value": n / dt, "unit": "events/s", "cores": cores, "kind": "oracle",
            "sample": "%d events of the same workload (event ids from 2e10), %.1f s, FP64 plain bound"
                      % (n, dt),
            "single_thread": {"value": n1 / dt1, "unit": "events/s", "cores": 1,
                              "sample": "%d events (ids from 2.1e10), %.1f s" % (n1, dt1)}}


def run_reference(args, ws, rank):
    name = args.workload
    process, sqrt_s, per_step, chunk, precision, mix, desc = WORKLOADS[name]
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2511_19633_gb300 import inputs
    pdf = inputs.synthetic_pdf_grid()
    cores = os.cpu_count() or 1
    rows, fr = _oracle_rows(O, process, sqrt_s, mix)
    # each step: a sample of the workload sized to about 20 s of CPU work over all steps
    probe = 200 * cores
    t0 = time.perf_counter()
    _oracle_run(O, rows, fr, 30_000_000_000, probe, pdf, cores)
    rate = probe / (time.perf_counter() - t0)
    n = max(probe, int(rate * 20.0 / max(1, args.steps)))
    for w in range(args.warmup):
        _oracle_run(O, rows, fr, 31_000_000_000 + w * n, min(n, probe), pdf, cores)
    t0 = time.perf_counter()
    for k in range(args.steps):
        _oracle_run(O, rows, fr, 32_000_000_000 + k * n, n, pdf, cores)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "events/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": name,
                       "description": "the FP64 CPU oracle as it stands (plain certified bound, Fig. 1 "
                                      "max-veto redrawing every channel, no learned proposal, no GPU) on "
                                      "%d host threads over a bounded sample of the workload's events"
                                      % cores,
                       "events_per_step": n},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": "events/s",
                             "sample": "%d events per step on %d threads" % (n, cores)},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _plain_pass(G, ctx, ev, first, total, chunk, stream, marks=None):
    """hard + shower + observables through the per-call entry points; with
    `marks`, a pair of CUDA events around each chunk's shower is appended."""
    import torch
    for f0 in range(0, total, chunk):
        m = min(chunk, total - f0)
        G.gaps_generate_hard(ctx, first + f0, m, ev, stream)
        if marks is not None:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        G.gaps_shower(ctx, first + f0, m, ev, stream)
        if marks is not None:
            b.record(stream)
            marks.append((a, b))
        G.gaps_observables(ctx, first + f0, m, ev, None, None, stream)


def _time_variant(G, cfg, ev, first, n, chunk, stream, learned=None, fit=None):
    """Events per second of one configuration over n events (after a warm-up
    pass), the shower kernels' own time, and the shower statistics."""
    import torch
    ctx = G.gaps_init(cfg)
    try:
        if learned is not None:
            G.gaps_set_learned_proposal(ctx, *learned)
        if fit is not None:
            G.gaps_set_pdf_ratio_fit(ctx, fit)
        # every acceptance weight above one, logged with its dipole type and channel
        vlog = torch.zeros((64, 8), dtype=torch.float32, device="cuda")
        vcnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        G.gaps_set_violation_log(ctx, vlog, vcnt)
        _plain_pass(G, ctx, ev, first - (1 << 40), min(n, 1 << 16), chunk, stream)
        torch.cuda.synchronize()
        G.gaps_reset_stats(ctx, stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        marks = []
        a.record(stream)
        _plain_pass(G, ctx, ev, first, n, chunk, stream, marks)
        b.record(stream)
        torch.cuda.synchronize()
        st = G.gaps_get_stats(ctx, stream)
        nv = min(int(vcnt.item()), vlog.shape[0])
        # entries of the timed run and the warm-up before it: {eta, s, t, w, class or
        # -1 - (8 type + channel), bin, z, zeta}
        logged = [[round(float(x), 7) for x in row] for row in vlog[:nv].cpu().tolist()]
    finally:
        G.gaps_destroy(ctx)
    return {"value": n / (a.elapsed_time(b) / 1e3), "unit": "events/s", "events": n,
            "shower_ms": sum(x.elapsed_time(y) for x, y in marks),
            "steps_per_event": st["steps"] / max(1, st["events"]),
            "trials_per_event": st["trials"] / max(1, st["events"]),
            "violations": st["violations"], "violation_log": logged[:8], "stats": st}


def _pdf_ratio_fit(G, cfg, ev, first, n, stream):
    """The paper's percentile fit of the PDF ratios (App. A.2), from the ratios
    a shower with the certified bounds evaluates for n events."""
    import torch
    ctx = G.gaps_init(cfg)
    try:
        cap = 1 << 23
        samples = torch.empty((cap, 4), dtype=torch.float32, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        G.gaps_generate_hard(ctx, first, n, ev, stream)
        G.gaps_collect_pdf_ratios(ctx, first, n, ev, samples, count, keep_fraction=0.1, stream=stream)
        torch.cuda.synchronize()
        m = min(int(count.item()), cap)
        fit = G.gaps_fit_pdf_ratios(samples[:m].cpu().numpy())
    finally:
        G.gaps_destroy(ctx)
    return fit, m


def run_ours(args, ws, rank, local):
    import torch
    from paper_2511_19633_gb300 import build
    build.build()
    from paper_2511_19633_gb300 import gaps as G
    from paper_2511_19633_gb300 import inputs

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    name = args.workload
    process, sqrt_s, total, chunk, precision, mix, desc = WORKLOADS[name]
    if args.events:
        total = args.events
        chunk = min(chunk, total)
    nmax = 128
    pdf = inputs.synthetic_pdf_grid()
    uses_pdf = bool(process or (mix and any(r[0] for r in mix)))
    stream = torch.cuda.current_stream()
    mixed = precision == G.GAPS_MIXED

    # learned initial-state proposal: trained on the GPU before the timed
    # region, on shower states of events outside every timed range
    learned = None
    learned_info = None
    # the network learns the initial-state states of the workload's own
    # hadronic process (a mixed batch: its first pp row); e+e- has none
    t_proc, t_sqrt_s, t_cut = next(((r[0], r[1], r[2]) for r in mix if r[0]), (0, 0.0, 1.0)) if mix \
        else (process, sqrt_s, 1.0)
    if mixed and not args.no_learned and t_proc != 0:
        from paper_2511_19633_gb300 import learned as LP
        tcfg = G.make_config(t_proc, t_sqrt_s, pdf_grid=pdf, nmax=nmax, seed=1, t_cut=t_cut,
                             precision=G.GAPS_MIXED, schedule=G.GAPS_SCHED_PERSISTENT,
                             blocks_per_sm=4, emit_batch=8)
        tctx = G.gaps_init(tcfg)
        t0 = time.perf_counter()
        try:
            res = LP.train_and_install(tctx, first_event=(3 << 40) + (rank << 38))
        finally:
            G.gaps_destroy(tctx)
        learned = (res["params"], res["log_margins"])
        learned_info = {"train_seconds": time.perf_counter() - t0, "states": res["states"],
                        "training_rows": res["rows"], "holdout_states": res["holdout_states"],
                        "mean_bin_height": res["mean_bin_height"], "loss_first": res["loss_first"],
                        "loss_last": res["loss_last"], "cells_calibrated": res["cells_calibrated"],
                        "fit_rmse": res["fit_rmse"], "pipeline": "gaps_train_learned_proposal (one C-ABI call)"}

    # mixed precision: the wavefront schedule (default) or the persistent one;
    # FP64: persistent or one thread per event
    if mixed:
        schedule = G.GAPS_SCHED_WAVE if args.schedule == 3 else G.GAPS_SCHED_PERSISTENT
    else:
        schedule = G.GAPS_SCHED_PERSISTENT if args.schedule else G.GAPS_SCHED_PER_EVENT
    shape = {"block_size": args.block, "blocks_per_sm": args.bps, "refill_period": args.period,
             "emit_batch": args.emit_batch}
    if schedule == G.GAPS_SCHED_WAVE:
        shape.update(wave_passes=args.passes, wave_cycles=args.cycles, wave_veto_blocks_per_sm=args.veto_bps)
    tuning = None
    if mixed and not args.no_autotune:
        from paper_2511_19633_gb300 import autotune
        tuning = autotune.autotune(process, sqrt_s, pdf, n_events=1 << 21, mix=mix, learned=learned,
                                   schedule=schedule)
        shape = tuning["best"]

    def config(pdf_ptr=None, trial_mode=None, sched=None):
        sh = dict(shape)
        if sched is not None and sched != schedule:  # another schedule: its own defaults
            sh = {"block_size": 256, "blocks_per_sm": 4, "refill_period": 1, "emit_batch": 16}
        c = G.make_config(process, sqrt_s, pdf_grid=pdf if uses_pdf and pdf_ptr is None else None, nmax=nmax,
                          seed=1, precision=precision, schedule=schedule if sched is None else sched, mix=mix,
                          trial_mode=trial_mode, **sh)
        if pdf_ptr is not None:
            c.pdf_grid = pdf_ptr
        return c

    ctx = G.gaps_init(config())
    if learned is not None:
        G.gaps_set_learned_proposal(ctx, *learned)
    n_rows = len(mix) if mix else 1
    buf = G.EventBuffers.allocate(chunk, nmax)
    ev = buf.view()
    obs = torch.zeros((G.GAPS_NOBS, chunk), dtype=torch.float64, device="cuda")
    hw = torch.zeros((n_rows, G.GAPS_NHIST, G.GAPS_HIST_BINS), dtype=torch.float64, device="cuda")
    hw2 = torch.zeros_like(hw)
    hists = G.GapsHists(hw.data_ptr(), hw2.data_ptr())
    steps_total = args.warmup + args.steps
    n_chunks = (total + chunk - 1) // chunk

    def first_of(k):
        return rank_first_event(rank, k, total, steps_total)

    for k in range(args.warmup):
        G.gaps_process(ctx, first_of(k), total, ev, obs, None, hists, stream)
    torch.cuda.synchronize()
    G.gaps_reset_stats(ctx, stream)
    shower_ms = []
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        for k in range(args.steps):
            G.gaps_process(ctx, first_of(args.warmup + k), total, ev, obs, None, hists, stream)
            if k + 1 < args.steps:
                shower_ms += G.gaps_process_shower_ms(ctx)
        stop.record(stream)
        torch.cuda.synchronize()
    shower_ms += G.gaps_process_shower_ms(ctx)
    if dist:
        dist.barrier()
    ms = start.elapsed_time(stop)
    stats = G.gaps_get_stats(ctx, stream)
    if dist:
        from paper_2511_19633_gb300.sharding import max_over_ranks
        ms = max_over_ranks(ms, dist, device="cuda")
    value = total * args.steps * ws / (ms / 1e3)
    G.gaps_destroy(ctx)  # its memory (two wavefront slots) goes back before the end-to-end contexts
    # kernels per chunk: hard process, the shower's kernels, observables
    if schedule == G.GAPS_SCHED_WAVE:
        P = shape.get("wave_passes", 24)
        shower_kernels = 1 + (P + 1) * (2 if learned is not None else 1) + 2 * P + 2
    else:
        shower_kernels = 1
    launches = (2 + shower_kernels) * n_chunks * args.steps

    # end to end through the C ABI with host buffers: a fresh context per step
    # (PDF grid and network from host memory), the full path as one graph,
    # every event's observables and the histograms back into pinned host memory
    pdf_host = torch.from_numpy(pdf).pin_memory() if uses_pdf else None
    obs_host = torch.empty((G.GAPS_NOBS, total), dtype=torch.float64).pin_memory()
    h_host = torch.empty((2, n_rows, G.GAPS_NHIST, G.GAPS_HIST_BINS), dtype=torch.float64).pin_memory()
    e2e_steps = args.steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        ctx2 = G.gaps_init(config(pdf_host.data_ptr() if pdf_host is not None else None))
        if learned is not None:
            G.gaps_set_learned_proposal(ctx2, *learned)
        hw.zero_()
        hw2.zero_()
        G.gaps_process(ctx2, first_of(k) + (1 << 50), total, ev, obs, obs_host, hists, stream)
        h_host[0].copy_(hw, non_blocking=True)
        h_host[1].copy_(hw2, non_blocking=True)
        torch.cuda.synchronize()
        G.gaps_destroy(ctx2)
    e2e_s = time.perf_counter() - t0
    e2e_value = total * e2e_steps * ws / e2e_s
    h2d = (pdf.nbytes if uses_pdf else 0) + (learned[0].nbytes + learned[1].nbytes if learned else 0)
    d2h = obs_host.numel() * 8 + h_host.numel() * 8

    # comparisons on samples of the same workload: the plain GPU veto
    # algorithm (FP64, one thread per event, no compaction, plain bound: the
    # paper's layout) and the compacted mixed-precision shower without the
    # learned proposal
    plain = mixed_plain = trial_modes = persistent = None
    if not args.no_plain:
        n_plain = min(total, 1 << 19)
        cfgp = G.make_config(process, sqrt_s, pdf_grid=pdf if uses_pdf else None, nmax=nmax, seed=1,
                             precision=G.GAPS_FP64, schedule=G.GAPS_SCHED_PER_EVENT, mix=mix)
        plain = _time_variant(G, cfgp, ev, 1 << 51, n_plain, chunk, stream)
        plain["mode"] = "FP64, one thread per event, no compaction, plain bound (the paper's layout)"
        if mixed and learned is not None:
            n_mp = min(total, chunk)
            mixed_plain = _time_variant(G, config(), ev, (1 << 51) + (1 << 24), n_mp, chunk, stream)
            mixed_plain["mode"] = "same shape and precision, plain bound (no learned proposal)"
            with_l = _time_variant(G, config(), ev, (1 << 51) + (1 << 24), n_mp, chunk, stream, learned)
            mixed_plain["learned_same_events"] = with_l
            mixed_plain["learned_gain"] = with_l["value"] / mixed_plain["value"]
            # the paper's fitted PDF-ratio overestimate in place of the certified
            # bound (fit from other events; acceptance weights above one counted)
            if uses_pdf:
                fit, n_samples = _pdf_ratio_fit(G, config(), ev, (1 << 51) + (3 << 24), min(n_mp, 1 << 19), stream)
                fitted = _time_variant(G, config(), ev, (1 << 51) + (1 << 24), n_mp, chunk, stream, None, fit)
                fitted["mode"] = ("percentile-fitted PDF-ratio overestimate (App. A.2: max(P99, P99.99 eta), "
                                  "P99.99 sqrt(eta) for g <- sum q), fit from %d sampled ratios; not a strict "
                                  "bound, violations counted" % n_samples)
                fitted["gain_vs_certified"] = fitted["value"] / mixed_plain["value"]
                mixed_plain["fitted_pdf_bound"] = fitted
        if mixed and schedule == G.GAPS_SCHED_WAVE:
            # the persistent schedule (one kernel, lanes refilled) on the same events
            n_mp = min(total, chunk)
            persistent = _time_variant(G, config(sched=G.GAPS_SCHED_PERSISTENT), ev, (1 << 51) + (1 << 24), n_mp,
                                       chunk, stream, learned)
            persistent["mode"] = "persistent schedule, 256 x 4 per SM, same events and proposal"
        if mixed:
            # the trial schemes on the same events, persistent schedule: max-veto
            # redrawing every channel, max-veto keeping the losing trials,
            # generate-select, veto-max (plain bounds)
            n_tm = min(total, chunk)
            trial_modes = {}
            for mode_name, mode in (("redraw", G.GAPS_TRIALS_REDRAW), ("keep", G.GAPS_TRIALS_KEEP),
                                    ("select", G.GAPS_TRIALS_SELECT), ("vetomax", G.GAPS_TRIALS_VETOMAX)):
                lrn = None if mode == G.GAPS_TRIALS_VETOMAX else learned
                trial_modes[mode_name] = _time_variant(G, config(trial_mode=mode, sched=G.GAPS_SCHED_PERSISTENT), ev,
                                                       (1 << 51) + (2 << 24), n_tm, chunk, stream, lrn)
                trial_modes[mode_name]["learned_proposal"] = lrn is not None

    per_launch_events = total / n_chunks
    mean_shower_ms = sum(shower_ms) / max(1, len(shower_ms))
    try:
        alu = alu_peaks(G)
        lane_peak = alu["ffma_per_s"] / 1e12
        fp64_peak = 2.0 * alu["dfma_per_s"] / 1e12
    except G.GapsError as err:  # the microbenchmarks failed: nominal figures, said so
        alu = {"error": str(err), "clocks": {}}
        lane_peak, fp64_peak = LANE_PEAK_TOPS_NOMINAL, FP64_PEAK_TFLOPS_NOMINAL
    if mixed:
        ops = algorithmic_ops(stats)
        # the time the work units took: the shower launches' own CUDA-event
        # time, or with the wavefront's two streams (chunks overlap) the timed
        # region itself (hard process and observables included: a lower bound)
        overlapped = schedule == G.GAPS_SCHED_WAVE and n_chunks > 1
        busy_s = ms / 1e3 if overlapped else sum(shower_ms) / 1e3
        achieved = ops / busy_s / 1e12
        impl = implementation_ops_mixed(stats) / busy_s / 1e12
        bpe = SHOWER_DRAM_BYTES_PER_EVENT.get((name, learned is not None))
        kname = SHOWER_KERNEL if schedule != G.GAPS_SCHED_WAVE else (
            "the shower phase: k_wave_veto, k_wave_ends, k_wave_mlp, k_wave_emit, k_wave_init/final and the "
            "k_shower_mixed tail, timed together" + (
                "; chunks run on two streams, so the time is the whole timed region (hard process and "
                "observables included)" if overlapped else ""))
        roof = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": lane_peak,
                "unit": "Tops/s (operations of the scope's work units per second)",
                "frac": achieved / lane_peak,
                "traffic": None if bpe is None else bpe * per_launch_events,
                "traffic_unit": "bytes per chunk's shower phase (ncu DRAM read + write of its kernels on "
                                "262 144 events, scaled by events)",
                "peak_source": ("measured: FP32 FMA lane throughput of this GPU (gaps_alu_peak, "
                                "median SM clock %s MHz)" % alu["clocks"].get("sm_mhz"))
                if "error" not in alu else "nominal 152 x 128 lanes x 2.07 GHz (microbenchmark failed)",
                "shower_ms_per_launch": mean_shower_ms, "events_per_launch": per_launch_events,
                "ops_per_event": ops / max(1, stats["events"]),
                "implementation": {"achieved": impl, "frac": impl / lane_peak,
                                   "ops_per_event": implementation_ops_mixed(stats) / max(1, stats["events"]),
                                   "note": "Philox, end-table rebuild and FP64 kinematics counted as executed"}}
    else:
        flops = fp64_flops(stats)
        achieved = flops / (sum(shower_ms) / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": "k_shower_fp64", "achieved": achieved, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": achieved / fp64_peak, "traffic": None,
                "peak_source": "measured: FP64 FMA throughput of this GPU x 2 (gaps_alu_peak)"
                if "error" not in alu else "nominal 1.25 TFLOP/s (microbenchmark failed)",
                "shower_ms_per_launch": mean_shower_ms, "events_per_launch": per_launch_events,
                "flop_per_event": flops / max(1, stats["events"])}
    if plain is not None and plain.get("shower_ms"):
        # the FP64 paper-layout kernel against the measured FP64 pipe
        f = fp64_flops(plain["stats"]) / (plain["shower_ms"] / 1e3) / 1e12
        plain["roofline"] = {"bound": "alu", "kernel": "k_shower_fp64", "achieved": f, "peak": fp64_peak,
                             "unit": "TFLOP/s", "frac": f / fp64_peak,
                             "peak_source": "measured FP64 FMA throughput x 2 (gaps_alu_peak)"}
    peaks = measured_peaks()
    line = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if precision == 0 else "f32+f64+bf16",
        "data": "synthetic",
        "config": {"workload": name, "description": desc, "events_per_step": total, "chunk": chunk,
                   "parallelism": "independent event ranges per GPU" if ws > 1 else "single GPU",
                   "schedule": {G.GAPS_SCHED_WAVE: "wavefront passes (rebuild, network, veto, emission kernels "
                                                   "over live-event lists), persistent kernel for the last events",
                                G.GAPS_SCHED_PERSISTENT: "persistent, live-event refill",
                                G.GAPS_SCHED_PER_EVENT: "one thread per event"}[schedule],
                   "launch_shape": shape, "learned_proposal": learned is not None,
                   "cuda_graph": "one graph per step (all chunks), parameters updated in place",
                   "l2": "event records of %.1f GB per chunk rewritten every chunk (> 129 MB L2)"
                         % (chunk * nmax * 44 / 1e9)},
        "roofline": roof,
        "clocks": clk.summary(),
        "e2e": {"value": e2e_value, "unit": "events/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "plain_gpu": plain,
        "mixed_plain_bound": mixed_plain,
        "persistent_schedule": persistent,
        "trial_modes": trial_modes,
        # the paper's own GPU number for NLO pp -> Z (V100, FP64, CT14lo at 13 TeV,
        # partitioning, 128 threads per block): context, not the target
        "paper_context": {"value": 1.7e4, "unit": "events/s", "hardware": "V100, FP64",
                          "workload": "NLO pp -> Z, CT14lo, 13 TeV, 1e6 events in about 60 s (the paper's CPU vs GPU comparison)"}
        if name == "pp_nlo_1e7" else None,
        "learned": learned_info,
        "shower_stats": {k: stats[k] for k in ("events", "steps", "trials", "isr_trials", "vetoes",
                                                "accepts", "violations", "err_capacity",
                                                "err_iter_cap", "err_numeric")},
        "veto_rate": stats["vetoes"] / max(1, stats["steps"]),
        "lane_efficiency": stats["lane_steps"] / max(1, stats["warp_steps"]),
        "hbm_gbs_measured": peaks.get("hbm_gbs"),
        "alu_peaks": alu,
    }
    if tuning is not None:
        line["autotune"] = {"best": tuning["best"], "sample_events": tuning["sample_events"],
                            "candidates": len(tuning["table"])}
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(process, sqrt_s, mix)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--events", type=int, default=0, help="override events per step")
    ap.add_argument("--schedule", type=int, default=3,
                    help="mixed precision: 3 wavefront, 1 persistent; FP64: 1 persistent, 0 per event")
    ap.add_argument("--block", type=int, default=256)
    ap.add_argument("--bps", type=int, default=4)
    ap.add_argument("--passes", type=int, default=24)
    ap.add_argument("--veto-bps", type=int, default=2)
    ap.add_argument("--cycles", type=int, default=64)
    ap.add_argument("--period", type=int, default=1)
    ap.add_argument("--emit-batch", type=int, default=16)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
