"""Pins for the denoiser oracle: the convolution against scipy's correlation
and the backward pass against central finite differences."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn


def test_conv_matches_library_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 7, 9))
    W = rng.standard_normal((9, 4, 3))
    b = rng.standard_normal(4)
    y = cnn.conv(x, W, b)
    for n in range(2):
        for o in range(4):
            k = W[:, o, :].reshape(3, 3, 3)          # [dy][dx][in]
            ref = b[o] + sum(correlate2d(x[n, i], k[:, :, i], mode="same") for i in range(3))
            np.testing.assert_allclose(y[n, o], ref, rtol=1e-12, atol=1e-12)


def test_param_count_and_identity_start():
    p = cnn.init_params(1)
    assert p.size == cnn.param_count() == 9 * 32 + 32 + 3 * (9 * 32 * 32 + 32) + 9 * 32 + 1
    x = np.random.default_rng(1).standard_normal((1, 8, 8))
    zero = p.copy()
    zero[-(9 * 32 + 1):] = 0.0                        # last layer off: y = x exactly
    np.testing.assert_array_equal(cnn.forward(zero, x)[0], x)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    p = cnn.init_params(3)
    p[-(9 * 32 + 1):] = rng.normal(0, 0.05, 9 * 32 + 1)  # make every layer matter
    x = rng.standard_normal((2, 6, 7))
    t = rng.standard_normal((2, 6, 7))
    y, cache = cnn.forward(p, x)
    g = cnn.backward(p, cache, 2 * (y - t) / y.size)
    idx = rng.choice(p.size, 25, replace=False)
    for i in idx:
        e = 1e-5 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += e
        pm[i] -= e
        fd = (cnn.mse(cnn.forward(pp, x)[0], t) - cnn.mse(cnn.forward(pm, x)[0], t)) / (2 * e)
        assert abs(g[i] - fd) <= 1e-6 * abs(fd) + 1e-9, (i, g[i], fd)
