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


# ---- Adam (Kingma & Ba 2015, Algorithm 1): pinned by closed forms of the
# recursion, not by retyping it


def _run(p, grads, lr, b1, b2, eps):
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t, g in enumerate(grads, start=1):
        p, m, v = cnn.adam(p, g, m, v, lr, b1, b2, eps, t)
    return p, m, v


def test_adam_first_step_moves_by_lr_times_the_gradient_sign():
    # from zero moments the bias corrections make m_hat = g and v_hat = g^2
    g = np.array([3.0, -0.5, 2e-4, -7e-9, 0.0])
    p0 = np.array([1.0, 2.0, -1.0, 0.5, 0.25])
    p1, m1, v1 = cnn.adam(p0, g, np.zeros(5), np.zeros(5), 0.01, 0.9, 0.999, 1e-8, 1)
    np.testing.assert_allclose(p1 - p0, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-10, atol=1e-18)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-14)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12)


def test_adam_epsilon_is_added_outside_the_square_root():
    # a gradient of magnitude eps moves by exactly half the learning rate
    eps = 1e-3
    p1 = cnn.adam(np.zeros(2), np.array([eps, -eps]), np.zeros(2), np.zeros(2), 0.2, 0.9, 0.999, eps, 1)[0]
    np.testing.assert_allclose(p1, [-0.1, 0.1], rtol=1e-12)


def test_adam_constant_gradient_moves_at_a_constant_rate():
    # with g fixed, m_t = (1 - b1^t) g and v_t = (1 - b2^t) g^2: the bias
    # corrections cancel exactly at every step, so each step is lr g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3])
    T, lr, eps = 40, 1e-2, 1e-8
    pT, mT, vT = _run(np.zeros(3), [g] * T, lr, 0.9, 0.999, eps)
    np.testing.assert_allclose(pT, -T * lr * g / (np.abs(g) + eps), rtol=1e-10)
    np.testing.assert_allclose(mT, (1 - 0.9 ** T) * g, rtol=1e-12)
    np.testing.assert_allclose(vT, (1 - 0.999 ** T) * g * g, rtol=1e-10)


def test_adam_single_impulse_decays_as_the_bias_corrected_geometric_series():
    # gradient g at step 1 and zero afterwards: m_t = b1^(t-1) (1 - b1) g and
    # v_t = b2^(t-1) (1 - b2) g^2, so step t moves by
    # lr * [b1^(t-1) (1-b1) / (1-b1^t)] / sqrt(b2^(t-1) (1-b2) / (1-b2^t)) * sign(g)   (eps = 0)
    b1, b2, lr, T = 0.9, 0.999, 1.0, 12
    g = np.array([2.5, -0.04])
    p = np.zeros(2)
    m = np.zeros(2)
    v = np.zeros(2)
    steps = []
    for t in range(1, T + 1):
        p_new, m, v = cnn.adam(p, g if t == 1 else np.zeros(2), m, v, lr, b1, b2, 0.0, t)
        a = b1 ** (t - 1) * (1 - b1) / (1 - b1 ** t)
        c = np.sqrt(b2 ** (t - 1) * (1 - b2) / (1 - b2 ** t))
        np.testing.assert_allclose(p_new - p, -lr * a / c * np.sign(g), rtol=1e-11)
        steps.append(p_new - p)
        p = p_new
    # the second step worked by hand: (0.09 / 0.19) / sqrt(0.000999 / 0.001999) = 0.6700583
    np.testing.assert_allclose(steps[1], -0.6700583 * np.sign(g), rtol=2e-7)


def test_adam_is_invariant_to_the_gradient_scale_without_eps():
    rng = np.random.default_rng(4)
    grads = [rng.standard_normal(6) for _ in range(7)]
    p0 = rng.standard_normal(6)
    a = _run(p0, grads, 1e-2, 0.8, 0.95, 0.0)[0]
    b = _run(p0, [1e3 * g for g in grads], 1e-2, 0.8, 0.95, 0.0)[0]
    np.testing.assert_allclose(a, b, rtol=1e-12)
