"""FP64 NumPy oracle of the rank / expansion predictor (test infrastructure only).

The predictor is a small multilayer perceptron that maps a node's sketched
singular-value spectrum to (a) its truncation rank as a fraction of the
largest possible rank and (b) whether an incoming batch will expand the node.
It is not part of the paper; its definition here is the contract the GPU
kernels are checked against:

  parameters  W1 [H, F], b1 [H], W2 [H, H], b2 [H], W3 [2, H], b3 [2]
              (H = 128 hidden units, F = 66 inputs), flattened in that order,
              row-major, as the master copy in float32;
  forward     x~ = bf16(x); a1 = bf16(W1) x~ + b1; h1 = bf16(relu(a1));
              a2 = bf16(W2) h1 + b2; h2 = bf16(relu(a2)); o = bf16(W3) h2 + b3;
              o0 = predicted rank fraction, o1 = logit of "expands";
  loss        mean over the batch of (o0 - t0)^2 + log(1 + exp(o1)) - t1 o1;
  gradients   of that loss with respect to the rounded weights, in the
              arithmetic of the forward pass (straight through the rounding),
              applied to the master copy;
  Adam        m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
              w -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

bf16(x) is round-to-nearest-even of a float32 to its 16 high-order bits. With
``rounding=False`` every bf16() is the identity and the arithmetic is plain
float64 (used to pin the gradients against finite differences).
"""
from __future__ import annotations

import numpy as np

F_IN = 66
HIDDEN = 128
N_OUT = 2


def param_shapes(f_in: int = F_IN, hidden: int = HIDDEN):
    return [(hidden, f_in), (hidden,), (hidden, hidden), (hidden,), (N_OUT, hidden), (N_OUT,)]


def n_params(f_in: int = F_IN, hidden: int = HIDDEN) -> int:
    return int(sum(np.prod(s) for s in param_shapes(f_in, hidden)))


def unflatten(p: np.ndarray, f_in: int = F_IN, hidden: int = HIDDEN):
    out, o = [], 0
    for s in param_shapes(f_in, hidden):
        k = int(np.prod(s))
        out.append(np.asarray(p[o:o + k]).reshape(s))
        o += k
    return out


def init_params(seed: int, f_in: int = F_IN, hidden: int = HIDDEN) -> np.ndarray:
    """U(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases, float32 (the master copy)."""
    rng = np.random.default_rng(seed)
    fans = [f_in, f_in, hidden, hidden, hidden, hidden]
    parts = [rng.uniform(-1.0 / np.sqrt(fan), 1.0 / np.sqrt(fan), size=s).astype(np.float32)
             for s, fan in zip(param_shapes(f_in, hidden), fans)]
    return np.concatenate([q.ravel() for q in parts]).astype(np.float32)


def bf16(x: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even of float32 values to bfloat16, returned as float32."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(a.shape)


def forward(p: np.ndarray, X: np.ndarray, rounding: bool = True):
    """Outputs [B, 2] and the intermediates needed by backward()."""
    r = bf16 if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = (np.asarray(q, dtype=np.float64) for q in unflatten(p))
    Wr = [np.asarray(r(W), dtype=np.float64) for W in (W1, W2, W3)]
    x = np.asarray(r(X), dtype=np.float64)
    a1 = x @ Wr[0].T + b1
    h1 = np.asarray(r(np.maximum(a1, 0.0)), dtype=np.float64)
    a2 = h1 @ Wr[1].T + b2
    h2 = np.asarray(r(np.maximum(a2, 0.0)), dtype=np.float64)
    o = h2 @ Wr[2].T + b3
    return o, (x, a1, h1, a2, h2, Wr)


def loss(o: np.ndarray, T: np.ndarray) -> float:
    B = o.shape[0]
    sq = (o[:, 0] - T[:, 0]) ** 2
    bce = np.logaddexp(0.0, o[:, 1]) - T[:, 1] * o[:, 1]
    return float(np.sum(sq + bce) / B)


def backward(p: np.ndarray, X: np.ndarray, T: np.ndarray, rounding: bool = True):
    """(loss, flat gradient) of the mean loss with respect to the (rounded) weights."""
    o, (x, a1, h1, a2, h2, Wr) = forward(p, X, rounding)
    B = o.shape[0]
    dO = np.empty_like(o)
    dO[:, 0] = 2.0 * (o[:, 0] - T[:, 0]) / B
    dO[:, 1] = (1.0 / (1.0 + np.exp(-o[:, 1])) - T[:, 1]) / B
    dW3 = dO.T @ h2
    db3 = dO.sum(axis=0)
    da2 = (dO @ Wr[2]) * (a2 > 0)
    dW2 = da2.T @ h1
    db2 = da2.sum(axis=0)
    da1 = (da2 @ Wr[1]) * (a1 > 0)
    dW1 = da1.T @ x
    db1 = da1.sum(axis=0)
    g = np.concatenate([q.ravel() for q in (dW1, db1, dW2, db2, dW3, db3)])
    return loss(o, T), g


def adam_step(p: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, t: int, lr: float,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (t counts from 1); returns the new (p, m, v) in float64."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
