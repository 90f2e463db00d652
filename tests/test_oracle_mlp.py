"""Pins of the oracle's proposal-network forward / backward pass."""
import math

import numpy as np

from oracle import sofa_oracle as orc


def params(rng, d, h, C, scale=0.3):
    return {
        "W1": rng.standard_normal((d, h)) * scale, "b1": rng.standard_normal(h) * 0.1,
        "W2": rng.standard_normal((h, h)) * scale, "b2": rng.standard_normal(h) * 0.1,
        "W3": rng.standard_normal((h, C)) * scale, "b3": rng.standard_normal(C) * 0.1,
    }


def test_gelu_closed_values():
    assert orc.gelu(np.array([0.0]))[0] == 0.0
    # GELU(x) - GELU(-x) = x  (Phi(x) + Phi(-x) = 1)
    x = np.linspace(-4, 4, 17)
    assert np.allclose(orc.gelu(x) - orc.gelu(-x), x, atol=1e-15)
    # Phi(1) = 0.841344746068543 (standard normal table)
    assert abs(orc.gelu(np.array([1.0]))[0] - 0.841344746068543) < 1e-12


def test_zero_weights_uniform_softmax():
    C, B = 10, 6
    p = {k: np.zeros_like(v) for k, v in params(np.random.default_rng(0), 4, 5, C).items()}
    x = np.random.default_rng(1).standard_normal((B, 4))
    y = np.arange(B) % C
    loss, g = orc.mlp_loss_grad(p, x, y)
    assert abs(loss - math.log(C)) < 1e-14
    expect = np.full(C, B / C)
    np.add.at(expect, y, -1.0)
    assert np.allclose(g["b3"], expect / B, atol=1e-15)


def test_finite_differences():
    rng = np.random.default_rng(2)
    p = params(rng, 5, 7, 6)
    x = rng.standard_normal((9, 5))
    y = rng.integers(0, 6, 9)
    _, g = orc.mlp_loss_grad(p, x, y)
    h = 1e-6
    for key in p:
        flat = p[key].reshape(-1)
        for i in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[i]
            flat[i] = old + h
            lp, _ = orc.mlp_loss_grad(p, x, y)
            flat[i] = old - h
            lm, _ = orc.mlp_loss_grad(p, x, y)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[key].reshape(-1)[i]) < 1e-7 + 1e-6 * abs(fd), key


def test_adam_first_step_is_lr_sign():
    # with bias correction the first Adam step is lr * g / (|g| + eps) ~ lr * sign(g)
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    out = orc.adam_step(p, g, m, v, 1, lr=0.01)
    assert np.allclose(out["w"] - p["w"], -0.01 * np.sign(g["w"]), atol=1e-7)


def test_forward_orientation_closed_form():
    """x @ W with W stored [d_in, d_out]: a tiny network with a non-symmetric
    middle layer.  x = (1, 2), W1 = I, W2 = [[0, 1], [0, 0]], W3 = I, zero
    biases: a1 = (1, 2), h1 = (Phi(1), 2 Phi(2)), a2 = (0, h1[0]),
    logits = h2 = (0, h1[0] Phi(h1[0])), with Phi the standard normal CDF."""
    Phi = lambda v: 0.5 * (1.0 + math.erf(v / math.sqrt(2.0)))
    p = {"W1": np.eye(2), "b1": np.zeros(2), "W2": np.array([[0.0, 1.0], [0.0, 0.0]]), "b2": np.zeros(2),
         "W3": np.eye(2), "b3": np.zeros(2)}
    logits, _ = orc.mlp_forward(p, np.array([[1.0, 2.0]]))
    h10 = Phi(1.0)
    assert abs(logits[0, 0]) < 1e-15
    assert abs(logits[0, 1] - h10 * Phi(h10)) < 1e-12
