"""Pins of the FP64 MLP oracle: backprop against central finite differences,
closed forms of the network and of Adam's first step."""
import numpy as np

from oracle import mlp


F, H = 7, 9


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init_params(F, H, 1) + rng.normal(scale=0.05, size=mlp.num_params(F, H))
    x = rng.normal(size=(11, F))
    t = rng.normal(size=11)
    _, g = mlp.gradient(theta, x, t, F, H)
    h = 1e-6
    num = np.zeros_like(theta)
    for i in range(theta.size):
        e = np.zeros_like(theta)
        e[i] = h
        num[i] = (mlp.loss(theta + e, x, t, F, H) - mlp.loss(theta - e, x, t, F, H)) / (2 * h)
    assert np.allclose(g, num, rtol=1e-5, atol=1e-8)


def test_closed_forms():
    # zero weights: the output is the last bias for every input
    theta = np.zeros(mlp.num_params(F, H))
    p = mlp.unpack(theta, F, H)
    p["b3"][0] = 1.25
    y, _ = mlp.forward(mlp.pack(p, F, H), np.random.default_rng(2).normal(size=(5, F)), F, H)
    assert np.allclose(y, 1.25)
    # identity-like path: one positive unit per layer passes x[0] through
    p = mlp.unpack(np.zeros(mlp.num_params(F, H)), F, H)
    p["W1"][0, 0] = 2.0
    p["W2"][0, 0] = 3.0
    p["W3"][0] = 0.5
    x = np.abs(np.random.default_rng(3).normal(size=(4, F)))
    y, _ = mlp.forward(mlp.pack(p, F, H), x, F, H)
    assert np.allclose(y, 3.0 * x[:, 0])
    # a negative input to that path is cut by the first ReLU
    y, _ = mlp.forward(mlp.pack(p, F, H), -x, F, H)
    assert np.allclose(y, 0.0)


def test_adam_first_step_is_lr_times_sign():
    # at t = 1, mhat = g and vhat = g^2, so the step is -lr * g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    opt = mlp.Adam(4, lr=0.01, eps=1e-8)
    new = opt.step(np.zeros(4), g)
    assert np.allclose(new, -0.01 * g / (np.abs(g) + 1e-8))


def test_training_reduces_loss_on_a_learnable_target():
    rng = np.random.default_rng(4)
    theta = mlp.init_params(F, H, 5)
    x = rng.normal(size=(64, F))
    t = np.sin(x[:, 0]) + 0.5 * x[:, 1]
    opt = mlp.Adam(theta.size, lr=3e-3)
    l0 = mlp.loss(theta, x, t, F, H)
    for _ in range(300):
        _, g = mlp.gradient(theta, x, t, F, H)
        theta = opt.step(theta, g)
    assert mlp.loss(theta, x, t, F, H) < 0.2 * l0


def _expectile_loss(theta, x, t, tau):
    y, _ = mlp.forward(theta, x, F, H)
    d = y - t
    return float(np.mean(np.where(d < 0, 2 * tau, 2 * (1 - tau)) * d ** 2))


def test_expectile_gradient_matches_finite_differences():
    # the pessimistic loss (weight 2 tau on underestimates), written out
    # here independently of mlp.gradient, against its central differences
    rng = np.random.default_rng(4)
    theta = mlp.init_params(F, H, 2) + rng.normal(scale=0.05, size=mlp.num_params(F, H))
    x = rng.normal(size=(13, F))
    t = rng.normal(size=13)
    tau = 0.8
    loss, g = mlp.gradient(theta, x, t, F, H, tau=tau)
    assert abs(loss - _expectile_loss(theta, x, t, tau)) < 1e-12
    h = 1e-6
    num = np.zeros_like(theta)
    for i in range(theta.size):
        e = np.zeros_like(theta)
        e[i] = h
        num[i] = (_expectile_loss(theta + e, x, t, tau) - _expectile_loss(theta - e, x, t, tau)) / (2 * h)
    assert np.allclose(g, num, rtol=1e-5, atol=1e-8)


def test_expectile_of_a_constant_network():
    # a network that outputs its last bias c everywhere: the loss is least
    # where c is the tau-expectile of the targets, the root of
    # tau * sum_{t > c} (t - c) = (1 - tau) * sum_{t < c} (c - t); tau = 0.5
    # gives the mean, larger tau a larger value (pessimism)
    rng = np.random.default_rng(5)
    t = rng.exponential(size=40)
    x = rng.normal(size=(40, F))
    for tau in (0.5, 0.75, 0.9):
        lo, hi = t.min(), t.max()
        for _ in range(200):  # bisection on the defining equation
            c = 0.5 * (lo + hi)
            f = tau * np.sum(np.maximum(t - c, 0)) - (1 - tau) * np.sum(np.maximum(c - t, 0))
            lo, hi = (c, hi) if f > 0 else (lo, c)
        theta = np.zeros(mlp.num_params(F, H))
        p = mlp.unpack(theta, F, H)
        p["b3"][0] = c
        theta = mlp.pack(p, F, H)
        _, g = mlp.gradient(theta, x, t, F, H, tau=tau)
        gb3 = mlp.unpack(g, F, H)["b3"][0]
        assert abs(gb3) < 1e-9
        if tau == 0.5:
            assert abs(c - t.mean()) < 1e-9
        else:
            assert c > t.mean()


def test_half_expectile_is_the_mean_squared_error():
    rng = np.random.default_rng(6)
    theta = mlp.init_params(F, H, 3)
    x = rng.normal(size=(9, F))
    t = rng.normal(size=9)
    l1, g1 = mlp.gradient(theta, x, t, F, H)
    y, _ = mlp.forward(theta, x, F, H)
    assert abs(l1 - np.mean((y - t) ** 2)) < 1e-12
    l2, g2 = mlp.gradient(theta, x, t, F, H, tau=0.5)
    assert np.array_equal(g1, g2) and l1 == l2
