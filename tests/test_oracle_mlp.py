"""Pins of the FP64 network reference: central differences of the loss, and a
closed form (all weights zero: the output is the last bias, whose gradient
is 2 (b - mean t) / n_out on the valid columns)."""
import numpy as np

from oracle import mlp

DIMS = [(12, 8), (8, 8), (8, 6)]  # (in_pad, out_pad) per layer
N_OUT = 5


def _params(rng):
    n = sum(a * b + b for a, b in DIMS)
    return rng.normal(0, 0.5, n)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    p = _params(rng)
    x = rng.normal(size=(7, 12))
    t = rng.normal(size=(7, 6))
    L, g = mlp.loss_and_grads(p, DIMS, x, t, N_OUT)
    h = 1e-6
    for i in rng.choice(len(p), 40, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_and_grads(pp, DIMS, x, t, N_OUT)[0] - mlp.loss_and_grads(pm, DIMS, x, t, N_OUT)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd))


def test_zero_weights_closed_form():
    rng = np.random.default_rng(1)
    p = np.zeros(sum(a * b + b for a, b in DIMS))
    b_last = rng.normal(size=6)
    p[-6:] = b_last
    x = rng.normal(size=(9, 12))
    t = rng.normal(size=(9, 6))
    L, g = mlp.loss_and_grads(p, DIMS, x, t, N_OUT)
    ref = np.zeros(6)
    ref[:N_OUT] = 2.0 * (b_last[:N_OUT] - t[:, :N_OUT].mean(axis=0)) / N_OUT
    np.testing.assert_allclose(g[-6:], ref, rtol=1e-12, atol=1e-14)
    assert L == np.mean((b_last[None, :N_OUT] - t[:, :N_OUT]) ** 2)
