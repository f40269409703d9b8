"""Pins of the FP64 reference network used to check the warm-start MLP (CPU only)."""
import numpy as np
from scipy import stats

from oracle import mlp


def _net(rng, dims):
    return [(rng.normal(0, 1 / np.sqrt(i), (o, i)), rng.normal(0, 0.1, o))
            for i, o in zip(dims[:-1], dims[1:])]


def test_gelu_is_x_times_normal_cdf():
    x = np.linspace(-6, 6, 97)
    np.testing.assert_allclose(mlp.gelu(x), x * stats.norm.cdf(x), rtol=1e-13, atol=1e-15)
    h = 1e-6
    fd = (x + h) * stats.norm.cdf(x + h) - (x - h) * stats.norm.cdf(x - h)
    np.testing.assert_allclose(mlp.gelu_grad(x), fd / (2 * h), rtol=1e-7, atol=1e-9)


def test_linear_network_matches_least_squares():
    rng = np.random.default_rng(1)
    X = rng.normal(size=(200, 7))
    Y = rng.normal(size=(200, 3))
    Xa = np.hstack([X, np.ones((200, 1))])
    coef, *_ = np.linalg.lstsq(Xa, Y, rcond=None)
    W, b = coef[:7].T, coef[7]
    loss, grads = mlp.loss_and_grads([(W, b)], X, Y)
    # at the least-squares solution the gradient vanishes and the loss is the residual
    assert np.abs(grads[0][0]).max() < 1e-12 and np.abs(grads[0][1]).max() < 1e-12
    assert abs(loss - np.mean((Xa @ coef - Y) ** 2)) < 1e-12
    # away from it, the gradient is the closed form 2 X^T (X W^T + b - Y) / (B n_out)
    W2 = W + 0.1
    _, g2 = mlp.loss_and_grads([(W2, b)], X, Y)
    r = X @ W2.T + b - Y
    np.testing.assert_allclose(g2[0][0], 2 * r.T @ X / r.size, rtol=1e-12)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    net = _net(rng, [9, 11, 10, 4])
    x = rng.normal(size=(13, 9))
    t = rng.normal(size=(13, 4))
    _, grads = mlp.loss_and_grads(net, x, t)
    h = 1e-6
    for li, (W, b) in enumerate(net):
        for (i, j) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (1, 2)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[i, j] += h
            Wm[i, j] -= h
            lp = mlp.loss_and_grads(net[:li] + [(Wp, b)] + net[li + 1:], x, t)[0]
            lm = mlp.loss_and_grads(net[:li] + [(Wm, b)] + net[li + 1:], x, t)[0]
            assert abs((lp - lm) / (2 * h) - grads[li][0][i, j]) < 1e-8
        bp, bm = b.copy(), b.copy()
        bp[0] += h
        bm[0] -= h
        lp = mlp.loss_and_grads(net[:li] + [(W, bp)] + net[li + 1:], x, t)[0]
        lm = mlp.loss_and_grads(net[:li] + [(W, bm)] + net[li + 1:], x, t)[0]
        assert abs((lp - lm) / (2 * h) - grads[li][1][0]) < 1e-8


def test_adamw_first_steps():
    rng = np.random.default_rng(3)
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    w1, m, v = mlp.adamw_step(w, g, np.zeros(50), np.zeros(50), 1, lr=1e-2, wd=0.1, eps=0.0)
    # bias-corrected first step: m_hat = g, v_hat = g^2, update = sign(g) + wd w
    np.testing.assert_allclose(w1, w - 1e-2 * (np.sign(g) + 0.1 * w), rtol=1e-13)
    g2 = rng.normal(size=50)
    w2, m2, v2 = mlp.adamw_step(w1, g2, m, v, 2, lr=1e-2, wd=0.0, eps=0.0)
    mh = (0.09 * g + 0.1 * g2) / (1 - 0.81)
    vh = (0.999 * 0.001 * g * g + 0.001 * g2 * g2) / (1 - 0.999 ** 2)
    np.testing.assert_allclose(w2, w1 - 1e-2 * mh / np.sqrt(vh), rtol=1e-12)
