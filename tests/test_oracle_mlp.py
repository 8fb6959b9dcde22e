"""Pins of the FP64 reference of the learned-proposal network: its analytic
backpropagation against central finite differences, and the forward pass
against a plain numpy evaluation of the same layers."""
import numpy as np
import pytest


def _params(rng):
    from oracle import oracle as O
    P = rng.normal(0, 0.4, O.MLP_PARAMS)
    return P


def test_forward_matches_numpy(oracle_mod):
    rng = np.random.default_rng(1)
    P = _params(rng)
    X = rng.normal(size=(50, 4))
    W1 = P[:256].reshape(64, 4); b1 = P[256:320]; W2 = P[320:4416].reshape(64, 64)
    b2 = P[4416:4480]; W3 = P[4480:4544]; b3 = P[4544]
    h1 = np.maximum(X @ W1.T + b1, 0)
    h2 = np.maximum(h1 @ W2.T + b2, 0)
    ref = h2 @ W3 + b3
    assert np.allclose(oracle_mod.mlp_forward(P, X), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("tau", [0.5, 0.9])
def test_backprop_matches_finite_differences(oracle_mod, tau):
    rng = np.random.default_rng(2)
    P = _params(rng)
    X = rng.normal(size=(40, 4))
    T = rng.normal(size=40)
    loss, g = oracle_mod.mlp_loss_grad(P, X, T, tau)
    h = 1e-6
    idx = np.concatenate([rng.choice(oracle_mod.MLP_PARAMS, 60, replace=False), [0, 255, 256, 4415, 4544]])
    for q in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[q] += h
        Pm[q] -= h
        fd = (oracle_mod.mlp_loss_grad(Pp, X, T, tau)[0] - oracle_mod.mlp_loss_grad(Pm, X, T, tau)[0]) / (2 * h)
        assert g[q] == pytest.approx(fd, rel=1e-5, abs=1e-8), q
