"""FP64 reference of the warm-start network (forward, MSE loss, gradients).

TEST INFRASTRUCTURE ONLY: used by the tests to check the GPU network's
forward pass and gradients.  Plain numpy, FP64, no batching tricks.

Network (the library's layout): x -> z_l = W_l h_{l-1} + b_l, h_l = silu(z_l)
for the hidden layers, y = W_L h_{L-1} + b_L; loss = mean over the valid
rows and the n_out valid columns of (y - t)^2.  Parameters use the padded
flat layout of the library: per layer W_l [out_pad x in_pad] row-major, then
b_l [out_pad].
"""
import numpy as np


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def unpack(params, dims):
    """dims: list of (in_pad, out_pad) per layer -> [(W, b)]."""
    out, o = [], 0
    for din, dout in dims:
        W = params[o:o + din * dout].reshape(dout, din)
        o += din * dout
        b = params[o:o + dout]
        o += dout
        out.append((W.astype(np.float64), b.astype(np.float64)))
    return out


def forward(layers, x):
    hs, zs = [x], []
    h = x
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        zs.append(z)
        h = z if l == len(layers) - 1 else silu(z)
        hs.append(h)
    return hs, zs


def loss_and_grads(params, dims, x, t, n_out):
    """Mean-squared error on the first n_out columns and its gradient with
    respect to every parameter (flat layout)."""
    layers = unpack(np.asarray(params, np.float64), dims)
    x = np.asarray(x, np.float64)
    t = np.asarray(t, np.float64)
    hs, zs = forward(layers, x)
    y = hs[-1]
    n = x.shape[0]
    d = np.zeros_like(y)
    d[:, :n_out] = y[:, :n_out] - t[:, :n_out]
    loss = float(np.sum(d * d) / (n * n_out))
    g = 2.0 * d / (n * n_out)
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, b = layers[l]
        gW = g.T @ hs[l]
        gb = g.sum(axis=0)
        grads.append((gW, gb))
        if l > 0:
            g = (g @ W) * dsilu(zs[l - 1])
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat
