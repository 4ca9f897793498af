"""FP64 NumPy restatement of the isovalue-guess MLP — TEST INFRASTRUCTURE ONLY.

Architecture (the learned part of the method): 40 inputs -> 64 -> 64 -> 64 -> 1, GELU (exact erf
form) after each hidden layer, output = normalised isovalue position t = (c - phi_min) /
(phi_max - phi_min). Loss: mean squared error on t.

Parameter vector layout (float32 on the device, float64 here), row-major:
  W1 [64][40], b1 [64], W2 [64][64], b2 [64], W3 [64][64], b3 [64], w4 [64], b4 [1]
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_H = 40, 64
SHAPES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_H, N_H)),
          ("b3", (N_H,)), ("w4", (N_H,)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)

_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def unflatten(p: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(p[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def flatten(P: dict) -> np.ndarray:
    return np.concatenate([np.asarray(P[name], np.float64).ravel() for name, _ in SHAPES])


def init(seed: int) -> np.ndarray:
    """Seeded initial parameters (normal, fan-in scaled; zero biases, output bias 0.5)."""
    rng = np.random.default_rng(seed)
    P = {"W1": rng.normal(0, 1 / math.sqrt(N_IN), (N_H, N_IN)), "b1": np.zeros(N_H),
         "W2": rng.normal(0, 1 / math.sqrt(N_H), (N_H, N_H)), "b2": np.zeros(N_H),
         "W3": rng.normal(0, 1 / math.sqrt(N_H), (N_H, N_H)), "b3": np.zeros(N_H),
         "w4": rng.normal(0, 1 / math.sqrt(N_H), N_H), "b4": np.array([0.5])}
    return flatten(P)


def forward(p: np.ndarray, X: np.ndarray):
    """Output [n] and the cache for backward."""
    P = unflatten(p)
    Z1 = X @ P["W1"].T + P["b1"]
    H1 = gelu(Z1)
    Z2 = H1 @ P["W2"].T + P["b2"]
    H2 = gelu(Z2)
    Z3 = H2 @ P["W3"].T + P["b3"]
    H3 = gelu(Z3)
    y = H3 @ P["w4"] + P["b4"][0]
    return y, (X, Z1, H1, Z2, H2, Z3, H3)


def loss_and_grad(p: np.ndarray, X: np.ndarray, t: np.ndarray):
    """Mean squared error and its gradient with respect to the parameter vector."""
    P = unflatten(p)
    y, (X, Z1, H1, Z2, H2, Z3, H3) = forward(p, X)
    n = len(t)
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    g = {"w4": H3.T @ dy, "b4": np.array([dy.sum()])}
    dZ3 = np.outer(dy, P["w4"]) * gelu_grad(Z3)
    g["W3"], g["b3"] = dZ3.T @ H2, dZ3.sum(0)
    dZ2 = (dZ3 @ P["W3"]) * gelu_grad(Z2)
    g["W2"], g["b2"] = dZ2.T @ H1, dZ2.sum(0)
    dZ1 = (dZ2 @ P["W2"]) * gelu_grad(Z1)
    g["W1"], g["b1"] = dZ1.T @ X, dZ1.sum(0)
    return loss, flatten(g)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (nearest even) and back, elementwise."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
