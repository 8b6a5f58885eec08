"""FP64 numpy oracle of the learned denoiser (not in the paper).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Network: five 3x3
convolutions with zero padding, channels 1 -> 32 -> 32 -> 32 -> 32 -> 1, ReLU
after the first four, the input added to the output.  Parameter vector
[W1 b1 W2 b2 W3 b3 W4 b4 W5 b5], each W stored [tap][out][in] with
tap = 3 (dy + 1) + (dx + 1) for the input offset (dy, dx) in {-1, 0, 1}^2.
Images are (nimg, H, W).  The backward pass is the chain rule written out;
the optimiser is Adam (Kingma & Ba 2015, Algorithm 1).
"""
from __future__ import annotations

import numpy as np

C = 32
LAYERS = [(1, C), (C, C), (C, C), (C, C), (C, 1)]  # (in, out) channels


def split(params):
    """Views of the parameter vector: list of (W[9, out, in], b[out])."""
    p = np.asarray(params, np.float64)
    out, k = [], 0
    for cin, cout in LAYERS:
        W = p[k:k + 9 * cout * cin].reshape(9, cout, cin)
        k += 9 * cout * cin
        b = p[k:k + cout]
        k += cout
        out.append((W, b))
    assert k == p.size
    return out


def param_count():
    return sum(9 * a * b + b for a, b in LAYERS)


def shift(x, dy, dx):
    """s[..., y, x] = x[..., y + dy, x + dx] with zeros outside (x: (..., H, W))."""
    H, W = x.shape[-2:]
    s = np.zeros_like(x)
    ys, yd = slice(max(dy, 0), H + min(dy, 0)), slice(max(-dy, 0), H + min(-dy, 0))
    xs, xd = slice(max(dx, 0), W + min(dx, 0)), slice(max(-dx, 0), W + min(-dx, 0))
    s[..., yd, xd] = x[..., ys, xs]
    return s


def conv(x, W, b):
    """y[n, o] = b[o] + sum_t sum_i W[t, o, i] x[n, i] shifted by tap t.  x: (N, I, H, W)."""
    y = np.zeros((x.shape[0], W.shape[1]) + x.shape[2:])
    for t in range(9):
        dy, dx = t // 3 - 1, t % 3 - 1
        y += np.einsum("oi,nihw->nohw", W[t], shift(x, dy, dx))
    return y + b[None, :, None, None]


def forward(params, x):
    """Returns (y, cache).  x: (N, H, W)."""
    layers = split(params)
    a = [x[:, None].astype(np.float64)]
    z = []
    for l, (W, b) in enumerate(layers):
        zl = conv(a[-1], W, b)
        z.append(zl)
        if l < 4:
            a.append(np.maximum(zl, 0.0))
    y = x + z[-1][:, 0]
    return y, (a, z)


def backward(params, cache, dy):
    """Gradient of sum(dy * y) with respect to the parameter vector."""
    layers = split(params)
    a, z = cache
    grads = [None] * 5
    dz = dy[:, None].astype(np.float64)               # d/dz5
    for l in range(4, -1, -1):
        W, _ = layers[l]
        x = a[l]
        dW = np.zeros_like(W)
        for t in range(9):
            dyy, dxx = t // 3 - 1, t % 3 - 1
            dW[t] = np.einsum("nohw,nihw->oi", dz, shift(x, dyy, dxx))
        grads[l] = (dW, dz.sum(axis=(0, 2, 3)))
        if l == 0:
            break
        dx_in = np.zeros_like(x)
        for t in range(9):
            dyy, dxx = t // 3 - 1, t % 3 - 1
            dx_in += shift(np.einsum("oi,nohw->nihw", W[t], dz), -dyy, -dxx)
        dz = dx_in * (z[l - 1] > 0)                  # through the ReLU of layer l-1
    return np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in grads])


def mse(y, t):
    return float(np.mean((y - t) ** 2))


def adam(params, grad, m, v, lr, b1, b2, eps, step):
    """One Adam step (Kingma & Ba 2015, Algorithm 1), in fp64: the moment
    estimates are updated with the new gradient, divided by the bias
    corrections 1 - b1^step and 1 - b2^step, and the parameters move by
    lr * m_hat / (sqrt(v_hat) + eps).  step counts from 1.  Returns the new
    (params, m, v); the inputs are left unchanged."""
    if step < 1:
        raise ValueError("step counts from 1")
    g = np.asarray(grad, np.float64)
    m_new = b1 * np.asarray(m, np.float64) + (1.0 - b1) * g
    v_new = b2 * np.asarray(v, np.float64) + (1.0 - b2) * g * g
    m_hat = m_new / (1.0 - b1 ** step)
    v_hat = v_new / (1.0 - b2 ** step)
    p_new = np.asarray(params, np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps)
    return p_new, m_new, v_new


def init_params(seed=0):
    """He-style seeded initialisation (input layer scaled by 9, hidden by 9 C);
    the last layer starts small so that the network starts near identity."""
    rng = np.random.default_rng(seed)
    out = []
    for l, (cin, cout) in enumerate(LAYERS):
        std = np.sqrt(2.0 / (9 * cin)) * (0.1 if l == 4 else 1.0)
        out.append(rng.normal(0, std, 9 * cout * cin))
        out.append(np.zeros(cout))
    return np.concatenate(out)
