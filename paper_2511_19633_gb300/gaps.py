"""Python binding of the C ABI in include/gaps.h (ctypes).

Argument marshalling only: every step of the hard process, the shower and the
observables runs in the CUDA library libgaps.so. There is no CPU fallback;
importing this module without the built library raises.
PyTorch is used for device memory and streams.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgaps.so")

GAPS_OK = 0
GAPS_ERR_INVALID_ARG = -1
GAPS_ERR_CAPACITY = -2
GAPS_ERR_ITER_CAP = -3
GAPS_ERR_NUMERIC = -4
GAPS_ERR_CUDA = -5
GAPS_ERR_NO_DEVICE = -6

GAPS_EE_QQ, GAPS_PP_Z_LO, GAPS_PP_Z_NLO, GAPS_PP_LL = 0, 1, 2, 3
GAPS_FP64, GAPS_MIXED = 0, 1
GAPS_SCHED_PER_EVENT, GAPS_SCHED_PERSISTENT, GAPS_SCHED_WARP, GAPS_SCHED_WAVE = 0, 1, 2, 3
GAPS_TRIALS_REDRAW, GAPS_TRIALS_KEEP, GAPS_TRIALS_SELECT, GAPS_TRIALS_VETOMAX = 0, 1, 2, 3
GAPS_STATUS_ACTIVE, GAPS_STATUS_DONE = 0, 1
GAPS_NOBS, GAPS_NHIST, GAPS_HIST_BINS = 8, 6, 66


GAPS_MAX_MIX = 4


class GapsMixRow(ctypes.Structure):
    _fields_ = [("process", ctypes.c_int), ("sqrt_s", ctypes.c_double), ("t_cut", ctypes.c_double),
                ("fraction", ctypes.c_double)]


class GapsConfig(ctypes.Structure):
    _fields_ = [
        ("process", ctypes.c_int), ("precision", ctypes.c_int), ("nf", ctypes.c_int),
        ("nmax_partons", ctypes.c_int), ("sqrt_s", ctypes.c_double),
        ("alpha_s_mz", ctypes.c_double), ("t_cut", ctypes.c_double), ("p_s", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("pdf_grid", ctypes.c_void_p), ("block_size", ctypes.c_int),
        ("schedule", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
        ("refill_period", ctypes.c_int), ("emit_batch", ctypes.c_int),
        ("n_mix", ctypes.c_int), ("mix", GapsMixRow * GAPS_MAX_MIX), ("trial_mode", ctypes.c_int),
        ("mll_lo", ctypes.c_double), ("mll_hi", ctypes.c_double), ("max_cycles", ctypes.c_int),
        ("wave_passes", ctypes.c_int), ("wave_cycles", ctypes.c_int),
        ("wave_veto_blocks_per_sm", ctypes.c_int),
    ]


class GapsEvents(ctypes.Structure):
    _fields_ = [
        ("capacity", ctypes.c_uint64), ("nmax", ctypes.c_int),
        ("p", ctypes.c_void_p), ("flav", ctypes.c_void_p), ("col", ctypes.c_void_p),
        ("acol", ctypes.c_void_p), ("npart", ctypes.c_void_p), ("status", ctypes.c_void_p),
        ("n_emit", ctypes.c_void_p), ("weight", ctypes.c_void_p), ("t", ctypes.c_void_p),
        ("eta", ctypes.c_void_p), ("draw", ctypes.c_void_p),
    ]


class GapsHists(ctypes.Structure):
    _fields_ = [("sumw", ctypes.c_void_p), ("sumw2", ctypes.c_void_p)]


STAT_FIELDS = ("events", "steps", "trials", "isr_trials", "vetoes", "accepts", "violations",
               "err_capacity", "err_iter_cap", "err_numeric", "lane_steps", "warp_steps", "rebuilds",
               "mlp_tiles")


class GapsStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in STAT_FIELDS]


class GapsLearnConfig(ctypes.Structure):
    _fields_ = [("first_event", ctypes.c_uint64), ("n_events", ctypes.c_uint64), ("capacity", ctypes.c_uint64),
                ("holdout_first", ctypes.c_uint64), ("holdout_events", ctypes.c_uint64),
                ("holdout_capacity", ctypes.c_uint64), ("steps", ctypes.c_uint64), ("lr", ctypes.c_float),
                ("tau", ctypes.c_float), ("seed", ctypes.c_uint64), ("slack", ctypes.c_float),
                ("min_rows", ctypes.c_uint32), ("target_floor", ctypes.c_float)]


REPORT_FIELDS = ("states", "rows", "holdout_states", "loss_first", "loss_last", "cells_calibrated",
                 "mean_bin_height", "fit_rmse")


class GapsLearnReport(ctypes.Structure):
    _fields_ = [("states", ctypes.c_uint64), ("rows", ctypes.c_uint64), ("holdout_states", ctypes.c_uint64),
                ("loss_first", ctypes.c_float), ("loss_last", ctypes.c_float), ("cells_calibrated", ctypes.c_uint32),
                ("mean_bin_height", ctypes.c_float), ("fit_rmse", ctypes.c_float)]


GAPS_MLP_PARAMS = 4545
GAPS_ISR_BINS = 8
GAPS_ISR_CLASSES = 44
GAPS_ISR_ETA_BINS = 8
# upper edges of the eta buckets on the network input ln(eta)/7 + 1 (float32)
GAPS_ISR_ETA_EDGES = (-0.6447, -0.3158, 0.0132, 0.3421, 0.6711, 0.8691, 0.9490)

EXPORTS = ("gaps_init", "gaps_generate_hard", "gaps_shower", "gaps_observables",
           "gaps_hist_binning", "gaps_get_stats", "gaps_reset_stats", "gaps_error_string",
           "gaps_destroy", "gaps_shower_static", "gaps_collect_isr_states", "gaps_isr_targets",
           "gaps_set_learned_proposal", "gaps_mlp_loss_grad", "gaps_mlp_forward", "gaps_mlp_train",
           "gaps_process", "gaps_process_shower_ms", "gaps_set_violation_log", "gaps_alu_peak",
           "gaps_train_learned_proposal", "gaps_collect_pdf_ratios", "gaps_fit_pdf_ratios",
           "gaps_set_pdf_ratio_fit")

# kinds of gaps_alu_peak (include/gaps_peaks.h)
GAPS_PEAK_FFMA, GAPS_PEAK_DFMA, GAPS_PEAK_MUFU, GAPS_PEAK_IMAD = 0, 1, 2, 3


class GapsError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__("%s failed: %s (%d)" % (where, gaps_error_string(code), code))
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libgaps.so is not built (run __graft_entry__.build()); "
                          "the shower has no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P, vp, i, u64 = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64
    lib.gaps_init.argtypes = [P(vp), P(GapsConfig)]
    lib.gaps_generate_hard.argtypes = [vp, u64, u64, P(GapsEvents), vp]
    lib.gaps_shower.argtypes = [vp, u64, u64, P(GapsEvents), vp]
    lib.gaps_observables.argtypes = [vp, u64, u64, P(GapsEvents), vp, P(GapsHists), vp]
    lib.gaps_process.argtypes = [vp, u64, u64, P(GapsEvents), vp, vp, P(GapsHists), vp]
    lib.gaps_process_shower_ms.argtypes = [vp, vp, i]
    d = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.gaps_hist_binning.argtypes = [vp, i, d, d, ip, ip, ip]
    lib.gaps_get_stats.argtypes = [vp, P(GapsStats), vp]
    lib.gaps_reset_stats.argtypes = [vp, vp]
    lib.gaps_error_string.argtypes = [i]
    lib.gaps_error_string.restype = ctypes.c_char_p
    lib.gaps_destroy.argtypes = [vp]
    lib.gaps_destroy.restype = None
    lib.gaps_shower_static.argtypes = [P(GapsConfig), u64, u64, P(GapsEvents), P(GapsStats), vp]
    f = ctypes.c_float
    lib.gaps_collect_isr_states.argtypes = [vp, u64, u64, P(GapsEvents), f, vp, u64, vp, vp]
    lib.gaps_isr_targets.argtypes = [vp, vp, u64, vp, vp, vp]
    lib.gaps_set_learned_proposal.argtypes = [vp, vp, vp]
    lib.gaps_set_violation_log.argtypes = [vp, vp, u64, vp]
    lib.gaps_mlp_loss_grad.argtypes = [vp, vp, vp, u64, f, vp, vp, vp]
    lib.gaps_mlp_forward.argtypes = [vp, vp, u64, i, vp, vp]
    lib.gaps_mlp_train.argtypes = [vp, vp, vp, vp, vp, u64, u64, f, f, u64, vp, i, vp]
    lib.gaps_alu_peak.argtypes = [i, i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
    lib.gaps_train_learned_proposal.argtypes = [vp, P(GapsLearnConfig), vp, vp, P(GapsLearnReport), vp]
    lib.gaps_collect_pdf_ratios.argtypes = [vp, u64, u64, P(GapsEvents), f, vp, u64, vp, vp]
    lib.gaps_fit_pdf_ratios.argtypes = [vp, u64, vp]
    lib.gaps_set_pdf_ratio_fit.argtypes = [vp, vp]
    return lib


_lib = _load()


def library() -> ctypes.CDLL:
    return _lib


def _check(rc: int, where: str):
    if rc != GAPS_OK:
        raise GapsError(rc, where)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# ---------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# ---------------------------------------------------------------------------
def gaps_error_string(code: int) -> str:
    return _lib.gaps_error_string(code).decode()


def gaps_init(cfg: GapsConfig) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(_lib.gaps_init(ctypes.byref(h), ctypes.byref(cfg)), "gaps_init")
    return h


def gaps_generate_hard(ctx, first_event: int, n: int, ev: GapsEvents, stream=None):
    _check(_lib.gaps_generate_hard(ctx, first_event, n, ctypes.byref(ev), _stream_ptr(stream)),
           "gaps_generate_hard")


def gaps_shower(ctx, first_event: int, n: int, ev: GapsEvents, stream=None):
    _check(_lib.gaps_shower(ctx, first_event, n, ctypes.byref(ev), _stream_ptr(stream)), "gaps_shower")


def gaps_shower_static(cfg: GapsConfig, first_event: int, n: int, ev: GapsEvents,
                       stream=None) -> dict:
    """The mixed-precision shower without any device allocation (its scratch is
    in the library's own device arrays; at most 32 partons per event). Returns
    the call's counters."""
    st = GapsStats()
    _check(_lib.gaps_shower_static(ctypes.byref(cfg), first_event, n, ctypes.byref(ev),
                                   ctypes.byref(st), _stream_ptr(stream)), "gaps_shower_static")
    return {name: int(getattr(st, name)) for name in STAT_FIELDS}


def gaps_collect_isr_states(ctx, first_event: int, n: int, ev: GapsEvents, states: torch.Tensor,
                            count: torch.Tensor, keep_fraction: float = 1.0, stream=None):
    """states: float32 [capacity, 4] device; count: int64 [1] device (incremented)."""
    _check(_lib.gaps_collect_isr_states(ctx, first_event, n, ctypes.byref(ev), float(keep_fraction),
                                        states.data_ptr(), states.shape[0], count.data_ptr(),
                                        _stream_ptr(stream)),
           "gaps_collect_isr_states")


def gaps_isr_targets(ctx, states: torch.Tensor, n_states: int, features: torch.Tensor,
                     targets: torch.Tensor, stream=None):
    _check(_lib.gaps_isr_targets(ctx, states.data_ptr(), n_states, features.data_ptr(),
                                 targets.data_ptr(), _stream_ptr(stream)), "gaps_isr_targets")


def gaps_set_learned_proposal(ctx, params, log_margins=0.0):
    """params: host float32 array of GAPS_MLP_PARAMS (copied) or None;
    log_margins: [GAPS_ISR_CLASSES][GAPS_ISR_ETA_BINS][GAPS_ISR_BINS] (or a scalar, broadcast)."""
    import numpy as np
    if params is None:
        _check(_lib.gaps_set_learned_proposal(ctx, None, None), "gaps_set_learned_proposal")
        return
    p = np.ascontiguousarray(params, dtype=np.float32)
    m = np.ascontiguousarray(np.broadcast_to(np.asarray(log_margins, dtype=np.float32),
                                             (GAPS_ISR_CLASSES, GAPS_ISR_ETA_BINS, GAPS_ISR_BINS)))
    _check(_lib.gaps_set_learned_proposal(ctx, p.ctypes.data, m.ctypes.data), "gaps_set_learned_proposal")


def gaps_train_learned_proposal(ctx, cfg: GapsLearnConfig, stream=None) -> dict:
    """The library's training pipeline of the learned proposal (collect, sort,
    targets, train, calibrate, install). Returns the report with the installed
    parameters and margins (numpy)."""
    import numpy as np
    params = np.zeros(GAPS_MLP_PARAMS, dtype=np.float32)
    margins = np.zeros((GAPS_ISR_CLASSES, GAPS_ISR_ETA_BINS, GAPS_ISR_BINS), dtype=np.float32)
    rep = GapsLearnReport()
    _check(_lib.gaps_train_learned_proposal(ctx, ctypes.byref(cfg), params.ctypes.data, margins.ctypes.data,
                                            ctypes.byref(rep), _stream_ptr(stream)), "gaps_train_learned_proposal")
    out = {n: getattr(rep, n) for n in REPORT_FIELDS}
    out["params"] = params
    out["log_margins"] = margins
    return out


def gaps_collect_pdf_ratios(ctx, first_event: int, n: int, ev: GapsEvents, samples: torch.Tensor,
                            count: torch.Tensor, keep_fraction: float = 1.0, stream=None):
    """samples: float32 [capacity, 4] device; count: int64 [1] device (incremented)."""
    _check(_lib.gaps_collect_pdf_ratios(ctx, first_event, n, ctypes.byref(ev), float(keep_fraction),
                                        samples.data_ptr(), samples.shape[0], count.data_ptr(),
                                        _stream_ptr(stream)), "gaps_collect_pdf_ratios")


def gaps_fit_pdf_ratios(samples):
    """samples: host float32 [n, 4]; returns the fit [12][12][2] (numpy)."""
    import numpy as np
    a = np.ascontiguousarray(samples, dtype=np.float32).reshape(-1, 4)
    fit = np.zeros((12, 12, 2), dtype=np.float32)
    _check(_lib.gaps_fit_pdf_ratios(a.ctypes.data if a.size else None, a.shape[0], fit.ctypes.data),
           "gaps_fit_pdf_ratios")
    return fit


def gaps_set_pdf_ratio_fit(ctx, fit):
    """fit: [12][12][2] float32 (copied) or None for the certified bounds."""
    import numpy as np
    if fit is None:
        _check(_lib.gaps_set_pdf_ratio_fit(ctx, None), "gaps_set_pdf_ratio_fit")
        return
    f = np.ascontiguousarray(fit, dtype=np.float32)
    _check(_lib.gaps_set_pdf_ratio_fit(ctx, f.ctypes.data), "gaps_set_pdf_ratio_fit")


def gaps_set_violation_log(ctx, log: torch.Tensor | None, count: torch.Tensor | None = None):
    """log: float32 [capacity, 8] device; count: int64 [1] device."""
    if log is None:
        _check(_lib.gaps_set_violation_log(ctx, None, 0, None), "gaps_set_violation_log")
        return
    _check(_lib.gaps_set_violation_log(ctx, log.data_ptr(), log.shape[0], count.data_ptr()),
           "gaps_set_violation_log")


def gaps_mlp_loss_grad(params: torch.Tensor, features: torch.Tensor, targets: torch.Tensor, tau: float,
                       grad: torch.Tensor, loss: torch.Tensor, stream=None):
    _check(_lib.gaps_mlp_loss_grad(params.data_ptr(), features.data_ptr(), targets.data_ptr(),
                                   targets.shape[0], float(tau), grad.data_ptr(), loss.data_ptr(),
                                   _stream_ptr(stream)), "gaps_mlp_loss_grad")


def gaps_mlp_forward(params: torch.Tensor, features: torch.Tensor, out: torch.Tensor, bf16: bool,
                     stream=None):
    _check(_lib.gaps_mlp_forward(params.data_ptr(), features.data_ptr(), features.shape[0], int(bf16),
                                 out.data_ptr(), _stream_ptr(stream)), "gaps_mlp_forward")


def gaps_mlp_train(params, adam_m, adam_v, features, targets, steps: int, lr: float, tau: float,
                   seed: int, loss_history=None, history_every: int = 0, stream=None):
    _check(_lib.gaps_mlp_train(params.data_ptr(), adam_m.data_ptr(), adam_v.data_ptr(), features.data_ptr(),
                               targets.data_ptr(), targets.shape[0], steps, float(lr), float(tau), seed,
                               None if loss_history is None else loss_history.data_ptr(), history_every,
                               _stream_ptr(stream)), "gaps_mlp_train")


def gaps_observables(ctx, first_event: int, n: int, ev: GapsEvents, obs: torch.Tensor | None,
                     hists: GapsHists | None, stream=None):
    _check(_lib.gaps_observables(ctx, first_event, n, ctypes.byref(ev), None if obs is None else obs.data_ptr(),
                                 None if hists is None else ctypes.byref(hists), _stream_ptr(stream)),
           "gaps_observables")


def gaps_process(ctx, first_event: int, n: int, ev: GapsEvents, obs_dev: torch.Tensor | None = None,
                 obs_host: torch.Tensor | None = None, hists: GapsHists | None = None, stream=None):
    """Whole path over n events in chunks of ev.capacity, as one CUDA graph.
    obs_dev: float64 [GAPS_NOBS, capacity] device; obs_host: pinned float64
    [GAPS_NOBS, n]."""
    _check(_lib.gaps_process(ctx, first_event, n, ctypes.byref(ev),
                             None if obs_dev is None else obs_dev.data_ptr(),
                             None if obs_host is None else obs_host.data_ptr(),
                             None if hists is None else ctypes.byref(hists), _stream_ptr(stream)),
           "gaps_process")


def gaps_process_shower_ms(ctx, max_chunks: int = 4096) -> list:
    """Per-chunk shower durations (ms) of the last gaps_process call."""
    buf = (ctypes.c_float * max_chunks)()
    k = _lib.gaps_process_shower_ms(ctx, buf, max_chunks)
    if k < 0:
        _check(k, "gaps_process_shower_ms")
    return [float(buf[c]) for c in range(k)]


def gaps_alu_peak(kind: int, iters: int = 4096, stream=None) -> dict:
    """Instruction throughput of one arithmetic pipe of the current GPU (the
    library's own microbenchmark): {"ops_per_s", "ms"}."""
    ops, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.gaps_alu_peak(kind, iters, ctypes.byref(ops), ctypes.byref(ms), _stream_ptr(stream)),
           "gaps_alu_peak")
    return {"ops_per_s": ops.value, "ms": ms.value}


def gaps_hist_binning(ctx, h: int) -> dict:
    lo, hi = ctypes.c_double(), ctypes.c_double()
    nb, ob, lg = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(_lib.gaps_hist_binning(ctx, h, ctypes.byref(lo), ctypes.byref(hi), ctypes.byref(nb),
                                  ctypes.byref(ob), ctypes.byref(lg)), "gaps_hist_binning")
    return {"lo": lo.value, "hi": hi.value, "nbins": nb.value, "obs": ob.value, "log10": bool(lg.value)}


def gaps_get_stats(ctx, stream=None) -> dict:
    st = GapsStats()
    _check(_lib.gaps_get_stats(ctx, ctypes.byref(st), _stream_ptr(stream)), "gaps_get_stats")
    return {n: int(getattr(st, n)) for n in STAT_FIELDS}


def gaps_reset_stats(ctx, stream=None):
    _check(_lib.gaps_reset_stats(ctx, _stream_ptr(stream)), "gaps_reset_stats")


def gaps_destroy(ctx):
    _lib.gaps_destroy(ctx)


# ---------------------------------------------------------------------------
# device buffers (torch-allocated) for the structure-of-arrays records
# ---------------------------------------------------------------------------
@dataclass
class EventBuffers:
    capacity: int
    nmax: int
    p: torch.Tensor       # [4][nmax][capacity] f64
    flav: torch.Tensor    # [nmax][capacity] i32
    col: torch.Tensor
    acol: torch.Tensor
    npart: torch.Tensor   # [capacity] i32
    status: torch.Tensor
    n_emit: torch.Tensor
    weight: torch.Tensor  # [capacity] f64
    t: torch.Tensor
    eta: torch.Tensor     # [2][capacity] f64
    draw: torch.Tensor    # [capacity] i64 (uint64 bits)

    @staticmethod
    def allocate(capacity: int, nmax: int, device="cuda") -> "EventBuffers":
        f64, i32 = torch.float64, torch.int32
        return EventBuffers(
            capacity, nmax,
            torch.zeros((4, nmax, capacity), dtype=f64, device=device),
            torch.zeros((nmax, capacity), dtype=i32, device=device),
            torch.zeros((nmax, capacity), dtype=i32, device=device),
            torch.zeros((nmax, capacity), dtype=i32, device=device),
            torch.zeros(capacity, dtype=i32, device=device),
            torch.zeros(capacity, dtype=i32, device=device),
            torch.zeros(capacity, dtype=i32, device=device),
            torch.zeros(capacity, dtype=f64, device=device),
            torch.zeros(capacity, dtype=f64, device=device),
            torch.zeros((2, capacity), dtype=f64, device=device),
            torch.zeros(capacity, dtype=torch.int64, device=device),
        )

    def view(self) -> GapsEvents:
        return GapsEvents(self.capacity, self.nmax, self.p.data_ptr(), self.flav.data_ptr(),
                          self.col.data_ptr(), self.acol.data_ptr(), self.npart.data_ptr(),
                          self.status.data_ptr(), self.n_emit.data_ptr(), self.weight.data_ptr(),
                          self.t.data_ptr(), self.eta.data_ptr(), self.draw.data_ptr())

    def to_host(self, n: int) -> dict:
        """Per-event arrays of the first n records, event index first (numpy)."""
        out = {
            "p": self.p[:, :, :n].permute(2, 1, 0).cpu().numpy(),
            "flav": self.flav[:, :n].T.cpu().numpy(),
            "col": self.col[:, :n].T.cpu().numpy(),
            "acol": self.acol[:, :n].T.cpu().numpy(),
            "npart": self.npart[:n].cpu().numpy(),
            "status": self.status[:n].cpu().numpy(),
            "n_emit": self.n_emit[:n].cpu().numpy(),
            "weight": self.weight[:n].cpu().numpy(),
            "t": self.t[:n].cpu().numpy(),
            "eta": self.eta[:, :n].T.cpu().numpy(),
        }
        return out


def make_config(process: int, sqrt_s: float, *, pdf_grid=None, t_cut: float = 1.0,
                alpha_s_mz: float = 0.118, nf: int = 5, nmax: int = 128, seed: int = 1,
                p_s: float = 0.5, precision: int = GAPS_FP64, block_size: int = 0,
                schedule: int = GAPS_SCHED_PER_EVENT, blocks_per_sm: int = 0,
                refill_period: int = 0, emit_batch: int = 0, mix=None, trial_mode=None,
                mll=(66.0, 116.0), max_cycles: int = 0, wave_passes: int = 0,
                wave_cycles: int = 0, wave_veto_blocks_per_sm: int = 0) -> GapsConfig:
    """Builds a gaps_config; pdf_grid is a float32 numpy array [11][100][50] that
    must stay alive until gaps_init returns (it is copied). mix: optional list of
    (process, sqrt_s, t_cut, fraction) rows of a mixed batch; they replace
    process, sqrt_s and t_cut. trial_mode: GAPS_TRIALS_*; None = KEEP for
    GAPS_MIXED with the persistent lane schedule, REDRAW otherwise. mll: the
    dilepton mass window of GAPS_PP_LL (GeV). max_cycles: veto cycles per event
    before GAPS_ERR_ITER_CAP (0 = the library default). wave_passes: passes of
    the wavefront schedule and wave_cycles: veto cycles of an event per pass (0 = the
    library defaults); wave_veto_blocks_per_sm: the veto kernel's resident blocks
    per SM (0 = 2)."""
    ptr = None if pdf_grid is None else pdf_grid.ctypes.data
    c = GapsConfig(process, precision, nf, nmax, sqrt_s, alpha_s_mz, t_cut, p_s, seed, ptr,
                   block_size, schedule, blocks_per_sm, refill_period, emit_batch)
    # kept trials by default where they apply (mixed precision, lane or wavefront schedule)
    if trial_mode is None:
        trial_mode = (GAPS_TRIALS_KEEP if precision == GAPS_MIXED
                      and schedule in (GAPS_SCHED_PERSISTENT, GAPS_SCHED_WAVE) else GAPS_TRIALS_REDRAW)
    c.trial_mode = int(trial_mode)
    c.mll_lo, c.mll_hi = float(mll[0]), float(mll[1])
    c.max_cycles = int(max_cycles)
    c.wave_passes = int(wave_passes)
    c.wave_cycles = int(wave_cycles)
    c.wave_veto_blocks_per_sm = int(wave_veto_blocks_per_sm)
    if mix:
        if len(mix) > GAPS_MAX_MIX:
            raise ValueError("at most %d rows" % GAPS_MAX_MIX)
        c.n_mix = len(mix)
        for k, (pr, rs, tc, fr) in enumerate(mix):
            c.mix[k] = GapsMixRow(int(pr), float(rs), float(tc), float(fr))
    return c
