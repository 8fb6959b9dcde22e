"""The learned initial-state proposal from Python: argument marshalling for
gaps_train_learned_proposal, which runs the whole pipeline in the library
(collection of shower states, canonical order, teacher targets, training with
the library's forward/backward/Adam kernels, calibration with the shower's
BF16 numerics, installation). The shower checks every acceptance weight; the
violation count it reports is part of every run's statistics.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import gaps as G

# the pipeline's settings for NLO pp -> Z (events of 2^40-aligned ranges
# disjoint from every measured range)
DEFAULTS = dict(first_event=3 << 40, n_events=1 << 22, capacity=1 << 20, holdout_offset=1 << 36,
                holdout_events=1 << 21, holdout_capacity=2 << 20, steps=40000, lr=2e-3, tau=0.97, seed=3,
                slack=0.2, min_rows=2048, target_floor=math.log(1e-4))


def learn_config(**kw) -> G.GapsLearnConfig:
    o = dict(DEFAULTS)
    o.update(kw)
    return G.GapsLearnConfig(int(o["first_event"]), int(o["n_events"]), int(o["capacity"]),
                             int(o["first_event"] + o["holdout_offset"]), int(o["holdout_events"]),
                             int(o["holdout_capacity"]), int(o["steps"]), float(o["lr"]), float(o["tau"]),
                             int(o["seed"]), float(o["slack"]), int(o["min_rows"]), float(o["target_floor"]))


def train_and_install(ctx, **kw) -> dict:
    """Trains, calibrates and installs the proposal in ctx (see DEFAULTS for
    the keyword arguments). Returns the library's report with "params" and
    "log_margins"."""
    return G.gaps_train_learned_proposal(ctx, learn_config(**kw))


def init_params(seed: int = 0) -> np.ndarray:
    """A random parameter vector in the library's layout, for checks of the
    network kernels (the pipeline initialises on the device)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, math.sqrt(2.0 / 4), (64, 4))
    W2 = rng.normal(0.0, math.sqrt(2.0 / 64), (64, 64))
    W3 = rng.normal(0.0, math.sqrt(1.0 / 64), 64)
    b1 = np.full(64, 0.1)
    b2 = np.full(64, 0.1)
    b3 = np.array([-1.0])
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3, b3]).astype(np.float32)


def train(feats: torch.Tensor, targ: torch.Tensor, steps: int, lr: float = 2e-3, tau: float = 0.97, seed: int = 3,
          params: np.ndarray | None = None, history_every: int = 500):
    """gaps_mlp_train in the pipeline's three learning-rate phases on given
    rows (device tensors); returns the parameters (device) and the loss
    history."""
    P = torch.from_numpy(init_params(seed) if params is None else params).cuda()
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    hist = torch.zeros(steps // history_every + 1, dtype=torch.float32, device="cuda")
    done = 0
    plan = [(steps // 2, lr), (steps // 4, lr * 0.3), (steps - steps // 2 - steps // 4, lr * 0.1)]
    for k, (s, l) in enumerate(plan):
        G.gaps_mlp_train(P, m, v, feats, targ, s, l, tau, seed + k, hist[done // history_every:], history_every)
        done += s
    torch.cuda.synchronize()
    return P, hist.cpu().numpy()
