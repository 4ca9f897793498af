"""P10: the FP64 MLP restatement against central finite differences and closed forms."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_gelu_closed_forms():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    # GELU(x) - GELU(-x) = x (from erf odd)
    x = np.linspace(-4, 4, 17)
    np.testing.assert_allclose(mlp.gelu(x) - mlp.gelu(-x), x, atol=1e-15)
    # derivative by central differences
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_grad(x), (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h), atol=1e-8)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init(3) + rng.normal(0, 0.05, mlp.N_PARAMS)
    X = rng.uniform(-1, 1, (7, mlp.N_IN))
    t = rng.uniform(0, 1, 7)
    loss, g = mlp.loss_and_grad(p, X, t)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    idx = np.concatenate([idx, [mlp.N_PARAMS - 1, mlp.N_PARAMS - 2, 0]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss_and_grad(p + e, X, t)[0] - mlp.loss_and_grad(p - e, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_layout_and_bf16_rounding():
    assert mlp.N_PARAMS == 64 * 40 + 64 + 2 * (64 * 64 + 64) + 64 + 1
    p = mlp.init(1)
    assert np.array_equal(mlp.flatten(mlp.unflatten(p)), p)
    # bfloat16 keeps 8 significant bits: 1 + 2^-8 rounds to even (1.0), 1 + 3 * 2^-8 up
    v = np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0])
    np.testing.assert_array_equal(mlp.bf16_round(v), [1.0, 1.0 + 2 ** -6, -2.5, 0.0])
