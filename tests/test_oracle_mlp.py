"""Pins of the FP64 warm-start network oracle: backpropagation against central
finite differences, the loss of an exactly representable map, and Adam's
first step (whose bias-corrected update is lr * sign(g) up to eps)."""

import numpy as np

from oracle import mlp


def _small(seed=0):
    rng = np.random.default_rng(seed)
    p = mlp.init(5, 7, 4, rng)
    for k in p:  # nonzero biases so every term of the backward pass is exercised
        if k.startswith("b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1
    X = rng.standard_normal((6, 5))
    Y = rng.standard_normal((6, 4))
    return p, X, Y


def test_backprop_matches_finite_differences():
    p, X, Y = _small()
    _, g = mlp.gradients(p, X, Y)
    h = 1e-6
    for k in p:
        num = np.zeros_like(p[k])
        it = np.nditer(p[k], flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = p[k][idx]
            p[k][idx] = old + h
            lp = mlp.loss(p, X, Y)
            p[k][idx] = old - h
            lm = mlp.loss(p, X, Y)
            p[k][idx] = old
            num[idx] = (lp - lm) / (2 * h)
        assert np.allclose(g[k], num, rtol=1e-5, atol=1e-8), k


def test_loss_zero_for_representable_map():
    p, X, _ = _small(1)
    y, _ = mlp.forward(p, X)
    assert mlp.loss(p, X, y) == 0.0
    lval, g = mlp.gradients(p, X, y)
    assert lval == 0.0 and all(np.all(v == 0) for v in g.values())


def test_adam_first_step_is_signed_lr():
    p, X, Y = _small(2)
    _, g = mlp.gradients(p, X, Y)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    p0 = {k: x.copy() for k, x in p.items()}
    mlp.adam_step(p, g, m, v, 1, 1e-3)
    for k in p:
        step = p0[k] - p[k]
        big = np.abs(g[k]) > 1e-6
        assert np.allclose(step[big], 1e-3 * np.sign(g[k][big]), rtol=1e-4)


def test_bf16_rounding_is_correct():
    # exact for numbers with at most 8 significant bits, ties to even, relative error <= 2^-8 (unit roundoff)
    assert np.array_equal(mlp.bf16(np.array([1.0, -0.75, 3.5, 1024.0])), [1.0, -0.75, 3.5, 1024.0])
    assert mlp.bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0  # tie -> even (1.0)
    assert mlp.bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6  # tie -> even (odd mantissa bit set)
    x = np.random.default_rng(0).standard_normal(10000)
    assert np.all(np.abs(mlp.bf16(x) - x) <= 2.0 ** -8 * np.abs(x) * (1 + 1e-6))
