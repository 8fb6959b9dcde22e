"""Training pipeline of the learned initial-state proposal, on the GPU.

1. collect: the plain mixed-precision shower logs the initial-state colour
   ends it meets (eta, dipole invariant, dipole type, emitter flavour);
2. targets: for every end, channel and zeta bin the library's teacher kernel
   computes the largest acceptance ratio over the bin and the scale range;
3. train: the library's own forward/backward/Adam kernels fit the
   4 -> 64 -> 64 -> 1 network with an expectile loss that keeps it above its
   targets;
4. calibrate: the BF16 tensor-core numerics of the shower are evaluated on all
   rows of the training states and of held-out states, and a margin per
   (class, eta bucket, bin) is set so that every row is covered; sparsely
   populated cells keep the plain bound;
5. install: gaps_set_learned_proposal.
The shower checks every acceptance weight; the violation count it reports
decides whether the learned run equals the plain algorithm.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import gaps as G


def init_params(seed: int = 0) -> np.ndarray:
    """He-initialised parameters in the library's layout."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, math.sqrt(2.0 / 4), (64, 4))
    W2 = rng.normal(0.0, math.sqrt(2.0 / 64), (64, 64))
    W3 = rng.normal(0.0, math.sqrt(1.0 / 64), 64)
    b1 = np.full(64, 0.1)
    b2 = np.full(64, 0.1)
    b3 = np.array([-1.0])
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3, b3]).astype(np.float32)


def collect_states(ctx, first_event: int, n_events: int, capacity: int, chunk: int = 1 << 20,
                   stream=None) -> torch.Tensor:
    """Runs the plain shower over n_events and returns up to `capacity` logged
    states [m, 4], sampled uniformly over the whole run: a pilot of 2^14
    events measures the states per event and sets the keep fraction."""
    pilot = min(n_events, 1 << 14)
    buf = G.EventBuffers.allocate(min(chunk, max(n_events, pilot)), 128)
    ev = buf.view()
    probe = torch.zeros((pilot * 64, 4), dtype=torch.float32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    G.gaps_generate_hard(ctx, first_event - pilot, pilot, ev, stream)
    G.gaps_collect_isr_states(ctx, first_event - pilot, pilot, ev, probe, count, 1.0, stream)
    torch.cuda.synchronize()
    per_event = max(1.0, int(count.item()) / pilot)
    keep = min(1.0, 0.95 * capacity / (per_event * n_events))
    states = torch.zeros((capacity, 4), dtype=torch.float32, device="cuda")
    count.zero_()
    for f0 in range(0, n_events, chunk):
        m = min(chunk, n_events - f0)
        G.gaps_generate_hard(ctx, first_event + f0, m, ev, stream)
        G.gaps_collect_isr_states(ctx, first_event + f0, m, ev, states, count, keep, stream)
    torch.cuda.synchronize()
    return _canonical_order(states[: min(int(count.item()), capacity)])


def _canonical_order(states: torch.Tensor) -> torch.Tensor:
    """The logged states in a fixed order (the shower logs them in the order of
    its atomic counter): with it the training, and so the network, is the same
    on every run."""
    if states.shape[0] == 0:
        return states
    h = states.cpu().numpy()
    order = np.lexsort((h[:, 1], h[:, 0], h[:, 3], h[:, 2]))
    return torch.from_numpy(np.ascontiguousarray(h[order])).to(states.device)


# targets below ln(1e-4) are raised to it: a higher target is still an upper
# bound, and bins that small are rarely proposed
TARGET_FLOOR = math.log(1e-4)


def make_dataset(ctx, states: torch.Tensor, stream=None):
    n = states.shape[0]
    feats = torch.zeros((n * 16, 4), dtype=torch.float32, device="cuda")
    targ = torch.zeros(n * 16, dtype=torch.float32, device="cuda")
    G.gaps_isr_targets(ctx, states, n, feats, targ, stream)
    torch.cuda.synchronize()
    return feats, torch.clamp(targ, min=TARGET_FLOOR)


def row_cell(feats: torch.Tensor) -> torch.Tensor:
    """Calibration cell (class, eta bucket, bin) of every row, from its input
    features (the same comparisons as the shower's)."""
    cls = torch.round((feats[:, 3] + 1.0) * 21.5).long()
    m = torch.round((feats[:, 2] + 1.0) * 4.0 - 0.5).long()
    edges = torch.tensor(G.GAPS_ISR_ETA_EDGES, dtype=torch.float32, device=feats.device)
    b = (feats[:, 0:1] >= edges[None, :]).sum(1)
    return (cls * G.GAPS_ISR_ETA_BINS + b) * G.GAPS_ISR_BINS + m


def train(feats: torch.Tensor, targ: torch.Tensor, steps: int = 40000, lr: float = 2e-3, tau: float = 0.97,
          seed: int = 3, params: np.ndarray | None = None, history_every: int = 500):
    P = torch.from_numpy(init_params(seed) if params is None else params).cuda()
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    hist = torch.zeros(steps // history_every + 1, dtype=torch.float32, device="cuda")
    done = 0
    # a few shorter launches with a decaying learning rate
    plan = [(steps // 2, lr), (steps // 4, lr * 0.3), (steps - steps // 2 - steps // 4, lr * 0.1)]
    for k, (s, l) in enumerate(plan):
        G.gaps_mlp_train(P, m, v, feats, targ, s, l, tau, seed + k, hist[done // history_every:],
                         history_every)
        done += s
    torch.cuda.synchronize()
    return P, hist.cpu().numpy()


def calibrate(P: torch.Tensor, sets, slack: float = 0.2, unseen: float = 30.0, min_rows: int = 64) -> dict:
    """Margins per (class, eta bucket, bin) so that exp(NN + margin) >= exp(target)
    on every row of every (features, targets) set, with the shower's BF16
    inference numerics, times (1 + slack). Cells with fewer than min_rows rows
    get `unseen` (height 1, the plain bound)."""
    ncell = G.GAPS_ISR_CLASSES * G.GAPS_ISR_ETA_BINS * G.GAPS_ISR_BINS
    gap = torch.full((ncell,), -float("inf"), device="cuda")
    rows = torch.zeros(ncell, dtype=torch.int64, device="cuda")
    outs = []
    for feats, targ in sets:
        out = torch.zeros_like(targ)
        G.gaps_mlp_forward(P, feats, out, True)
        cell = row_cell(feats)
        gap = gap.scatter_reduce(0, cell, targ - out, reduce="amax")
        rows += torch.bincount(cell, minlength=ncell)
        outs.append((out, cell, targ))
    torch.cuda.synchronize()
    seen = rows >= min_rows
    margins = torch.where(seen, gap + math.log(1.0 + slack), torch.full_like(gap, unseen))
    # how much the learned heights shrink the plain overestimate on the first set
    out, cell, targ = outs[0]
    U = torch.clamp(torch.exp(out + margins[cell]), max=1.0)
    return {"log_margins": margins.view(G.GAPS_ISR_CLASSES, G.GAPS_ISR_ETA_BINS, G.GAPS_ISR_BINS).cpu().numpy(),
            "mean_bin_height": float(U.mean().item()), "cells_seen": int(seen.sum().item()),
            "rows": int(targ.shape[0]), "fit_rmse": float(torch.sqrt(torch.mean((out - targ) ** 2)).item())}


def train_and_install(ctx, first_event: int = 3 << 40, n_events: int = 1 << 22, capacity: int = 1 << 20,
                      steps: int = 40000, holdout_events: int = 1 << 21) -> dict:
    """Collects shower states (seed offset by first_event), trains, calibrates
    on the training rows and on held-out states of other events, and installs
    the network in ctx. Returns a summary."""
    states = collect_states(ctx, first_event, n_events, capacity)
    feats, targ = make_dataset(ctx, states)
    P, hist = train(feats, targ, steps=steps)
    held = collect_states(ctx, first_event + (1 << 36), holdout_events, 2 * capacity)
    hf, ht = make_dataset(ctx, held)
    cal = calibrate(P, [(feats, targ), (hf, ht)])
    G.gaps_set_learned_proposal(ctx, P.cpu().numpy(), cal["log_margins"])
    return {"states": int(states.shape[0]), "rows": int(feats.shape[0]), "holdout_states": int(held.shape[0]),
            "loss_first": float(hist[0]),
            "loss_last": float(hist[hist > 0][-1]) if np.any(hist > 0) else None, **cal,
            "params": P.cpu().numpy()}
