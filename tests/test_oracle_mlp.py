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


def _bf16(a):
    import torch
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).double().numpy()


def _f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def _emulated_gradient(p, dims, x, t, n_out, drop_dsilu_layer=None):
    """The gradient computed with the roundings of a bf16 tensor-core network
    (products of rounded values summed in FP32; h, z rounded after each
    hidden layer; dY and every dZ rounded before their products)."""
    layers = mlp.unpack(p, dims)
    L, n = len(layers), x.shape[0]
    hs, zb, h = [x], [], x
    for l, (W, b) in enumerate(layers):
        z = _f32(h @ W.T) + b
        if l < L - 1:
            zb.append(_bf16(z))
            h = _bf16(_f32(z / (1.0 + np.exp(-z))))
            hs.append(h)
        else:
            y = _f32(z)
    d = np.zeros_like(y)
    d[:, :n_out] = y[:, :n_out] - t[:, :n_out]
    dz = _bf16(2.0 * d / (n * n_out))
    out = [None] * L
    for l in range(L - 1, -1, -1):
        W = layers[l][0]
        out[l] = (_f32(dz.T @ hs[l]), _f32(dz.sum(axis=0)))
        if l > 0:
            v = _f32(dz @ W)
            ds = 1.0 if drop_dsilu_layer == l - 1 else mlp.dsilu(zb[l - 1])
            dz = _bf16(v * ds)
    return np.concatenate([np.concatenate([a.ravel(), b]) for a, b in out])


def test_rounding_sigma_covers_a_bf16_network_and_not_a_wrong_term():
    """grad_error_sigma is the tolerance of the GPU gradient test: the
    difference between a bf16-rounded evaluation and the FP64 gradient stays
    within 6 sigma per entry, while dropping silu' in one layer (a plausible
    mistake) puts entries far outside it."""
    rng = np.random.default_rng(4)
    dims = [(32, 64), (64, 64), (64, 48)]
    n_out, n = 40, 256
    p = []
    for din, dout in dims:
        p += [_bf16(rng.normal(0, 1 / np.sqrt(din), (dout, din))).ravel(), _f32(rng.normal(0, 0.1, dout))]
    p = np.concatenate(p)
    x = _bf16(rng.normal(size=(n, 32)))
    t = _f32(rng.normal(size=(n, 48)))
    _, g = mlp.loss_and_grads(p, dims, x, t, n_out)
    sig = mlp.grad_error_sigma(p, dims, x, t, n_out)
    floor = 1e-7 * np.abs(g).max()
    ratio = np.abs(_emulated_gradient(p, dims, x, t, n_out) - g) / (6.0 * sig + floor)
    assert ratio.max() <= 1.0
    assert np.median(sig[sig > 0] / np.abs(g[sig > 0])) < 0.02  # tight: a few per mille of |g|
    bad = np.abs(_emulated_gradient(p, dims, x, t, n_out, drop_dsilu_layer=0) - g) / (6.0 * sig + floor)
    assert bad.max() > 10.0
