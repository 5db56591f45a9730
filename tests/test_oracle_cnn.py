"""Pins of the CNN oracle (oracle/cnn.py) against independent definitions:
SciPy's 2D cross-correlation, central finite differences of the loss, the
closed form of one Adam step, and planted mistakes."""
import numpy as np
import pytest

from oracle import cnn


def test_conv_matches_scipy_correlate():
    sig = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    a = rng.normal(size=(2, 3, 7, 9))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    z = cnn.conv3x3(a, W, b)
    for bi in range(2):
        for o in range(4):
            ref = b[o] + sum(sig.correlate2d(a[bi, c], W[o, c], mode="same", boundary="fill") for c in range(3))
            np.testing.assert_allclose(z[bi, o], ref, rtol=1e-12, atol=1e-12)


def test_conv_brute_force_single_point():
    rng = np.random.default_rng(1)
    a = rng.normal(size=(1, 2, 5, 5))
    W = rng.normal(size=(3, 2, 3, 3))
    b = np.zeros(3)
    z = cnn.conv3x3(a, W, b)
    i, j = 0, 4                                   # a corner: taps outside the image are zero
    ref = 0.0
    for c in range(2):
        for p in range(3):
            for q in range(3):
                ii, jj = i + p - 1, j + q - 1
                if 0 <= ii < 5 and 0 <= jj < 5:
                    ref += W[1, c, p, q] * a[0, c, ii, jj]
    assert abs(z[0, 1, i, j] - ref) < 1e-13


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    ch = (6, 5, 4, 3, 1)                          # small widths, same structure
    theta = cnn.init_params(3, ch) + 0.05 * rng.normal(size=cnn.n_params(ch))
    x = rng.normal(size=(2, 6, 6, 7))
    t = rng.normal(size=(2, 1, 6, 7))
    _, g = cnn.grad(theta, x, t, ch)
    idx = rng.choice(theta.size, size=40, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros_like(theta)
        e[k] = h
        fd = (cnn.loss(theta + e, x, t, ch) - cnn.loss(theta - e, x, t, ch)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, fd, g[k])


def test_planted_mistakes_are_caught():
    """A transposed kernel (W[o,c,q,p]) and a missing relu mask change the
    forward or the gradient beyond the pins' tolerances."""
    rng = np.random.default_rng(4)
    a = rng.normal(size=(1, 2, 6, 6))
    W = rng.normal(size=(2, 2, 3, 3))
    b = np.zeros(2)
    z = cnn.conv3x3(a, W, b)
    zt = cnn.conv3x3(a, W.transpose(0, 1, 3, 2), b)
    assert np.max(np.abs(z - zt)) > 1e-3
    ch = (6, 4, 4, 4, 1)
    theta = cnn.init_params(5, ch)
    x = rng.normal(size=(1, 6, 5, 5))
    t = rng.normal(size=(1, 1, 5, 5))
    _, g = cnn.grad(theta, x, t, ch)
    # gradient of the same network without relu (linear) differs
    y, acts = cnn.forward(theta, x, ch)
    assert np.any(acts[1] == 0.0)                 # relu is active somewhere
    k = 0
    e = np.zeros_like(theta)
    e[k] = 1e-6
    fd = (cnn.loss(theta + e, x, t, ch) - cnn.loss(theta - e, x, t, ch)) / 2e-6
    assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9


def test_adam_first_step_closed_form():
    """After one step from m = v = 0 the bias-corrected update is lr * sign(g)
    (up to eps): m_hat = g, v_hat = g^2."""
    opt = cnn.Adam(3, lr=0.01)
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    new = opt.step(theta, g)
    np.testing.assert_allclose(new, theta - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_minimises_a_quadratic():
    opt = cnn.Adam(2, lr=0.05)
    theta = np.array([3.0, -1.0])
    for _ in range(2000):
        theta = opt.step(theta, 2 * (theta - np.array([0.5, 0.25])))
    np.testing.assert_allclose(theta, [0.5, 0.25], atol=1e-3)


def test_parameter_layout():
    assert cnn.n_params() == 32 * 6 * 9 + 32 + 2 * (32 * 32 * 9 + 32) + 32 * 9 + 1
    theta = np.arange(cnn.n_params(), dtype=float)
    layers = cnn.unpack(theta)
    assert layers[0][0].shape == (32, 6, 3, 3) and layers[0][0][0, 0, 0, 0] == 0
    assert layers[0][1][0] == 32 * 6 * 9
    assert layers[3][0].shape == (1, 32, 3, 3) and layers[3][1].shape == (1,)


def test_weighted_gradient_matches_central_differences():
    rng = np.random.default_rng(6)
    ch = (6, 4, 4, 3, 1)
    theta = cnn.init_params(7, ch)
    x = rng.normal(size=(1, 6, 5, 6))
    t = rng.normal(size=(1, 1, 5, 6))
    w = (rng.random(size=t.shape) < 0.4).astype(float) * 2.5
    _, g = cnn.grad(theta, x, t, ch, w=w)
    for k in rng.choice(theta.size, size=25, replace=False):
        e = np.zeros_like(theta)
        e[k] = 1e-6
        fd = (cnn.loss(theta + e, x, t, ch, w=w) - cnn.loss(theta - e, x, t, ch, w=w)) / 2e-6
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9
    # zero weights where the target differs make those points irrelevant
    t2 = t + (w == 0) * 5.0
    assert abs(cnn.loss(theta, x, t, ch, w=w) - cnn.loss(theta, x, t2, ch, w=w)) < 1e-14
