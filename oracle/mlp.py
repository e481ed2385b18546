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


def dsilu2(z):
    """Second derivative of silu: s (1 - s) (2 + z (1 - 2 s)), s the logistic."""
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 - s) * (2.0 + z * (1.0 - 2.0 * s))



def grad_error_sigma(params, dims, x, t, n_out, u=2.0 ** -8):
    """Standard deviation, per gradient entry, of the difference rounding makes
    to the gradient of loss_and_grads when the network is evaluated as a
    tensor-core implementation does it: inputs and weights already in a
    format of unit roundoff u (bf16: 2^-8; the FP64 reference takes the same
    rounded values), every hidden activation h_l and pre-activation z_l
    rounded after its layer, the output gradient dY and every
    back-propagated gradient dZ_l rounded before they enter a product,
    products summed in FP32 (terms of order 2^-24, left to the caller's
    floor).  Probabilistic rounding-error analysis (Higham and Mary, SIAM J.
    Sci. Comput. 41 (2019)): each rounding is an independent zero-mean error
    of variance (u |v|)^2 / 3 (round to nearest: uniform in +-u|v|), and
    variances, not absolute values, propagate through the sums:
      V(h_l)  = silu'(z_l)^2 (V(h_{l-1}) (W_l^2)^T) + u^2 h_l^2 / 3
      V(dZ_L) = s^2 V(y) + u^2 dZ_L^2 / 3,  s = 2 / (rows n_out)
      V(dZ_{l-1}) = silu'^2 (V(dZ_l) W_l^2) + (dZ_l W_l)^2 silu''^2 (V(z) + u^2 z^2 / 3)
                    + u^2 dZ_{l-1}^2 / 3
      V(dW_l) = V(dZ_l)^T h_{l-1}^2 + (dZ_l^2)^T V(h_{l-1}),  V(db_l) = sum of V(dZ_l).
    Returns sqrt(V) in the flat parameter layout; a difference of many
    standard deviations means a wrong term, not rounding."""
    layers = unpack(np.asarray(params, np.float64), dims)
    x = np.asarray(x, np.float64)
    t = np.asarray(t, np.float64)
    hs, zs = forward(layers, x)
    L = len(layers)
    n = x.shape[0]
    r = u * u / 3.0
    V = [np.zeros_like(x)]  # variance of the error of h_l (hs[l])
    Vz = []
    for l in range(L):
        W = layers[l][0]
        vz = V[-1] @ (W * W).T
        Vz.append(vz)
        V.append(dsilu(zs[l]) ** 2 * vz + r * hs[l + 1] ** 2 if l < L - 1 else vz)
    s = 2.0 / (n * n_out)
    valid = np.zeros_like(hs[-1])
    valid[:, :n_out] = 1.0
    dz = s * (hs[-1] - t) * valid
    Vd = s * s * V[-1] * valid + r * dz * dz
    out = [None] * L
    for l in range(L - 1, -1, -1):
        out[l] = (Vd.T @ hs[l] ** 2 + (dz * dz).T @ V[l], Vd.sum(axis=0))
        if l > 0:
            W = layers[l][0]
            gp = dz @ W
            z = zs[l - 1]
            dz_new = gp * dsilu(z)
            Vd = (dsilu(z) ** 2 * (Vd @ (W * W)) + gp ** 2 * dsilu2(z) ** 2 * (Vz[l - 1] + r * z * z)
                  + r * dz_new ** 2)
            dz = dz_new
    return np.sqrt(np.concatenate([np.concatenate([a.ravel(), b]) for a, b in out]))
