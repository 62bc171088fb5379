"""Pins of the FP64 network reference (no GPU): library convolution and log-softmax, finite differences."""
import numpy as np
import scipy.signal
import scipy.special

from oracle import cnn


def test_conv_forward_matches_correlate2d():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 8, 8))
    W = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    for stride in (1, 2):
        y = cnn.conv_forward(x, W, b, stride)
        for bi in range(2):
            for co in range(4):
                full = sum(scipy.signal.correlate2d(x[bi, ci], W[co, ci], mode="same") for ci in range(3)) + b[co]
                np.testing.assert_allclose(y[bi, co], full[::stride, ::stride], atol=1e-12)


def test_log_softmax_and_prepare():
    rng = np.random.default_rng(2)
    z = rng.standard_normal((3, 9)) * 10
    np.testing.assert_allclose(cnn.log_softmax(z), scipy.special.log_softmax(z, axis=1), atol=1e-12)
    img = rng.standard_normal((2, 16, 16)) * 3 + 5
    x = cnn.prepare(img, 2)
    assert x.shape == (2, 1, 8, 8)
    np.testing.assert_allclose(x.mean(axis=(2, 3)), 0, atol=1e-12)
    np.testing.assert_allclose(x.var(axis=(2, 3)), 1, atol=1e-12)
    np.testing.assert_allclose(x[0, 0, 0, 0] * np.sqrt(img[0].reshape(8, 2, 8, 2).mean(axis=(1, 3)).var())
                               + img[0].reshape(8, 2, 8, 2).mean(axis=(1, 3)).mean(), img[0, :2, :2].mean(), atol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    down, C, n_q, n_d, B = 2, 3, 5, 3, 3
    imgs = rng.standard_normal((B, 32, 32))
    _, _, F, n = cnn.layout(16, C, n_q, n_d)
    theta = rng.standard_normal(n) * 0.4
    yq = rng.integers(0, n_q, B)
    yd = rng.integers(0, n_d, B)
    losses, g = cnn.loss_and_grad(theta, imgs, yq, yd, down, C, n_q, n_d)
    f = lambda t: cnn.loss_and_grad(t, imgs, yq, yd, down, C, n_q, n_d)[0].mean()
    offs, heads, _, _ = cnn.layout(16, C, n_q, n_d)
    idx = [o[0][0] for o in offs] + [o[1][0] for o in offs] + [h[0] for h in heads] + list(rng.integers(0, n, 30))
    h = 1e-6
    for i in idx:
        e = np.zeros(n)
        e[i] = h
        fd = (f(theta + e) - f(theta - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
