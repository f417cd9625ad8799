"""FP64 reference of the warm-start network (oracle; test infrastructure only).

The learned warm start maps the parameters theta of a parametric SOS program
to a predicted HSDE iterate.  The network is a plain multilayer perceptron

    h1 = relu(X W1^T + b1),  h2 = relu(h1 W2^T + b2),  Yhat = h2 W3^T + b3,

trained on the mean squared error  L = sum((Yhat - Y)^2) / (B * n_out)  with
Adam (Kingma & Ba: beta1 = 0.9, beta2 = 0.999, eps = 1e-8, bias-corrected
moments).  Weights are stored as [n_out x n_in] (row = output unit).
Everything here is FP64 NumPy, written out step by step so that it can be
checked by finite differences.
"""

from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np

Params = Dict[str, np.ndarray]
LAYERS = ("1", "2", "3")


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64:
    keep the top 16 bits of the float32 pattern after adding the rounding
    bias 0x7FFF + (bit 16)."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _mm(a: np.ndarray, b: np.ndarray, round_operands: bool) -> np.ndarray:
    if round_operands:  # operands rounded to bfloat16, products and sums exact (FP64)
        return bf16(a) @ bf16(b)
    return a @ b


def forward(p: Params, X: np.ndarray, round_operands: bool = False) -> Tuple[np.ndarray, List[np.ndarray]]:
    r = round_operands
    z1 = _mm(X, p["W1"].T, r) + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = _mm(h1, p["W2"].T, r) + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = _mm(h2, p["W3"].T, r) + p["b3"]
    return y, [X, z1, h1, z2, h2]


def loss(p: Params, X: np.ndarray, Y: np.ndarray) -> float:
    y, _ = forward(p, X)
    return float(np.sum((y - Y) ** 2) / Y.size)


def gradients(p: Params, X: np.ndarray, Y: np.ndarray, round_operands: bool = False) -> Tuple[float, Params]:
    """Loss and its gradient with respect to every parameter (backpropagation).
    ``round_operands`` rounds the two operands of every matrix product to
    bfloat16 (a model of tensor-core arithmetic); all else stays FP64."""
    r = round_operands
    y, (X0, z1, h1, z2, h2) = forward(p, X, r)
    dy = 2.0 * (y - Y) / Y.size
    g: Params = {}
    g["W3"] = _mm(dy.T, h2, r)
    g["b3"] = dy.sum(axis=0)
    dh2 = _mm(dy, p["W3"], r)
    dz2 = dh2 * (z2 > 0)
    g["W2"] = _mm(dz2.T, h1, r)
    g["b2"] = dz2.sum(axis=0)
    dh1 = _mm(dz2, p["W2"], r)
    dz1 = dh1 * (z1 > 0)
    g["W1"] = _mm(dz1.T, X0, r)
    g["b1"] = dz1.sum(axis=0)
    return float(np.sum((y - Y) ** 2) / Y.size), g


def adam_step(p: Params, g: Params, m: Params, v: Params, t: int, lr: float,
              b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update in place; t counts steps from 1."""
    for k in p:
        m[k] = b1 * m[k] + (1 - b1) * g[k]
        v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k]
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def init(n_in: int, n_hidden: int, n_out: int, rng: np.random.Generator) -> Params:
    """He-uniform weights, zero biases."""
    p: Params = {}
    dims = [(n_hidden, n_in), (n_hidden, n_hidden), (n_out, n_hidden)]
    for name, (o, i) in zip(LAYERS, dims):
        bound = np.sqrt(6.0 / i)
        p["W" + name] = rng.uniform(-bound, bound, size=(o, i))
        p["b" + name] = np.zeros(o)
    return p
