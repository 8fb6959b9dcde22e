"""Training pipeline of the learned initial-state proposal, on the GPU.

1. collect: the plain mixed-precision shower logs the initial-state colour
   ends it meets (eta, dipole invariant, dipole type, emitter flavour);
2. targets: for every end, channel and zeta bin the library's teacher kernel
   computes the largest acceptance ratio over the bin and the scale range;
3. train: the library's own forward/backward/Adam kernels fit the
   4 -> 64 -> 64 -> 1 network with an expectile loss that keeps it above its
   targets;
4. calibrate: the BF16 tensor-core numerics of the shower are evaluated on all
   rows and the margin is set so that every row is covered;
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
    """Runs the plain shower over n_events and returns the logged states [m, 4]."""
    states = torch.zeros((capacity, 4), dtype=torch.float32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    buf = G.EventBuffers.allocate(min(chunk, n_events), 128)
    ev = buf.view()
    for f0 in range(0, n_events, chunk):
        m = min(chunk, n_events - f0)
        G.gaps_generate_hard(ctx, first_event + f0, m, ev, stream)
        G.gaps_collect_isr_states(ctx, first_event + f0, m, ev, states, count, stream)
        torch.cuda.synchronize()
        if int(count.item()) >= capacity:
            break
    return states[: min(int(count.item()), capacity)]


def make_dataset(ctx, states: torch.Tensor, stream=None):
    n = states.shape[0]
    feats = torch.zeros((n * 16, 4), dtype=torch.float32, device="cuda")
    targ = torch.zeros(n * 16, dtype=torch.float32, device="cuda")
    G.gaps_isr_targets(ctx, states, n, feats, targ, stream)
    torch.cuda.synchronize()
    return feats, targ


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


def calibrate(P: torch.Tensor, feats: torch.Tensor, targ: torch.Tensor, slack: float = 0.02) -> dict:
    """Margin so that exp(NN + margin) >= exp(target) on every row, with the
    shower's BF16 inference numerics."""
    out = torch.zeros_like(targ)
    G.gaps_mlp_forward(P, feats, out, True)
    torch.cuda.synchronize()
    gap = (targ - out)
    margin = float(gap.max().item()) + math.log(1.0 + slack)
    # how much the learned heights shrink the plain overestimate on the sample
    U = torch.clamp(torch.exp(out + margin), max=1.0)
    return {"log_margin": margin, "mean_bin_height": float(U.mean().item()),
            "rows": int(targ.shape[0]), "fit_rmse": float(torch.sqrt(torch.mean((out - targ) ** 2)).item())}


def train_and_install(ctx, first_event: int = 3 << 40, n_events: int = 1 << 20, capacity: int = 1 << 20,
                      steps: int = 40000) -> dict:
    """Collects shower states (seed offset by first_event), trains, calibrates
    and installs the network in ctx. Returns a summary."""
    states = collect_states(ctx, first_event, n_events, capacity)
    feats, targ = make_dataset(ctx, states)
    P, hist = train(feats, targ, steps=steps)
    cal = calibrate(P, feats, targ)
    G.gaps_set_learned_proposal(ctx, P.cpu().numpy(), cal["log_margin"])
    return {"states": int(states.shape[0]), "rows": int(feats.shape[0]), "loss_first": float(hist[0]),
            "loss_last": float(hist[hist > 0][-1]) if np.any(hist > 0) else None, **cal,
            "params": P.cpu().numpy()}
