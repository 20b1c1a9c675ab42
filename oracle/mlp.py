"""FP64 reference of the candidate-proposal MLP -- TEST INFRASTRUCTURE ONLY.

The proposal network is not part of the paper: it is the learned pruning
stage layered on the exact method (a small MLP that scores each window
candidate so that only the best few enter the recursion). This module is the
plain numpy definition its CUDA training and inference kernels are checked
against:

  x  = [f_i (F), f'_j (F), dx/100, dy/100, dt/w]        (input, 2F + 3)
  z1 = W1 x + b1,  h1 = relu(z1)                         (hidden 128)
  z2 = W2 h1 + b2, h2 = relu(z2)                         (hidden 128)
  z3 = w3 . h2 + b3,  s = sigmoid(z3)                    (keep score)
  loss = mean over the batch of softplus(z3) - y z3      (binary cross-entropy with logits)

with dx = x'_j - x_i, dy = y'_j - y_i, dt = t'_j - (t_i + o) and w the window
half-width. Gradients are written out by the chain rule; Adam follows Kingma
and Ba (2015), bias-corrected. forward_bf16 / backward_bf16 are the same
definitions with the operands of the tensor-core products rounded to BF16
(the kernels' arithmetic up to FP32 accumulation order). Only tests/ and
bench.py's CPU legs import it.
"""
from __future__ import annotations

import numpy as np

H = 128


def init(rng: np.random.Generator, d_in: int, hidden: int = H):
    """He-style initialisation; returns a dict of FP64 arrays."""
    return {
        "W1": rng.standard_normal((hidden, d_in)) * np.sqrt(2.0 / d_in),
        "b1": np.zeros(hidden),
        "W2": rng.standard_normal((hidden, hidden)) * np.sqrt(2.0 / hidden),
        "b2": np.zeros(hidden),
        "w3": rng.standard_normal(hidden) * np.sqrt(1.0 / hidden),
        "b3": np.zeros(1),
    }


def features(model_f, scene_f, model_xy, scene_xy, model_t, scene_t, i, j, o, window):
    """Input rows for (model point i, scene point j, offset o) triples (arrays of equal length)."""
    i, j, o = np.asarray(i), np.asarray(j), np.asarray(o)
    d = np.stack([(scene_xy[j, 0] - model_xy[i, 0]) / 100.0,
                  (scene_xy[j, 1] - model_xy[i, 1]) / 100.0,
                  (scene_t[j] - (model_t[i] + o)) / float(max(window, 1))], axis=1)
    return np.concatenate([model_f[i], scene_f[j], d], axis=1).astype(np.float64)


def forward(p, x):
    z1 = x @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ p["w3"] + p["b3"][0]
    return {"z1": z1, "h1": h1, "z2": z2, "h2": h2, "z3": z3}


def score(p, x):
    return 1.0 / (1.0 + np.exp(-forward(p, x)["z3"]))


def loss(p, x, y):
    z3 = forward(p, x)["z3"]
    return float(np.mean(np.logaddexp(0.0, z3) - y * z3))


def backward(p, x, y):
    """Gradients of loss() with respect to every parameter."""
    c = forward(p, x)
    B = x.shape[0]
    dz3 = (1.0 / (1.0 + np.exp(-c["z3"])) - y) / B
    g = {"w3": c["h2"].T @ dz3, "b3": np.array([dz3.sum()])}
    dz2 = np.outer(dz3, p["w3"]) * (c["z2"] > 0)
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * (c["z1"] > 0)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return g


def bf16(x):
    """Rounds to the nearest BF16 value (8 significant bits), ties to even, returned as float64. The value is
    first taken to FP32, as the kernels hold it, then its low 16 bits are rounded away."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(p, x, rnd=bf16):
    """forward() with the operands of the two hidden layers' products rounded to BF16 first -- the inputs
    the tensor cores receive (x and W1; h1 and W2) -- and everything else in FP64. The output layer
    (w3 . h2 + b3) and the biases stay unrounded. rnd is the rounding (identity gives forward())."""
    z1 = rnd(x) @ rnd(p["W1"]).T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = rnd(h1) @ rnd(p["W2"]).T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ p["w3"] + p["b3"][0]
    return {"z1": z1, "h1": h1, "z2": z2, "h2": h2, "z3": z3}


def backward_bf16(p, x, y, rnd=bf16):
    """backward() through forward_bf16, with the operands of every product the backward pass runs on the
    tensor cores rounded to BF16: dz2 and h1 (gradient of W2), dz2 and W2 (gradient of h1), dz1 and x
    (gradient of W1). Returns (loss, gradients, scale): scale[k] is, per element of gradient k, the same
    backward pass run on absolute values (every factor replaced by its magnitude, so sums cannot cancel):
    the size of all the terms the element is built from, through every layer above it, against which
    rounding differences of that element are measured. rnd is the rounding (identity gives backward())."""
    c = forward_bf16(p, x, rnd)
    B = x.shape[0]
    z3 = c["z3"]
    loss_v = float(np.mean(np.logaddexp(0.0, z3) - y * z3))
    dz3 = (1.0 / (1.0 + np.exp(-z3)) - y) / B
    g = {"w3": c["h2"].T @ dz3, "b3": np.array([dz3.sum()])}
    scale = {"w3": np.abs(c["h2"]).T @ np.abs(dz3), "b3": np.array([np.abs(dz3).sum()])}
    dz2 = np.outer(dz3, p["w3"]) * (c["z2"] > 0)
    m2 = np.abs(dz2)
    g["b2"] = dz2.sum(axis=0)
    scale["b2"] = m2.sum(axis=0)
    A2, H1 = rnd(dz2), rnd(c["h1"])
    g["W2"] = A2.T @ H1
    scale["W2"] = m2.T @ np.abs(c["h1"])
    dh1 = A2 @ rnd(p["W2"])
    dz1 = dh1 * (c["z1"] > 0)
    m1 = (m2 @ np.abs(p["W2"])) * (c["z1"] > 0)
    g["b1"] = dz1.sum(axis=0)
    scale["b1"] = m1.sum(axis=0)
    A1, X = rnd(dz1), rnd(x)
    g["W1"] = A1.T @ X
    scale["W1"] = m1.T @ np.abs(x)
    return loss_v, g, scale


def score_split_bf16(p, x, model_xy, scene_xy, F, rnd=bf16, window=3):
    """The logit z3 as the pruning pass computes it. The first layer is split into a model-point part
    P = W1a f_i + b1 - W1c (x_i, y_i) / 100 and a scene-point part Q = W1b f'_j + W1c (x'_j, y'_j) / 100
    (both products on BF16 operands, each part rounded once to BF16), and a time term: the hidden units are
    h1 = relu(rnd(dt * rnd(W1c_t / w) + rnd(P + Q))), dt = t'_j - t_i - o the integer frame difference and
    w = window (at least 1) -- one BF16 add and one fused BF16 multiply-add per unit, as BF16x2 arithmetic
    does it. Layer 2 then runs on BF16 operands (h1 is one already), its bias b2 rounded to BF16 as well (it
    enters the tensor-core product as one more input against a constant 1), and the output layer is
    unrounded.
    x holds the rows of features() built with the same window (the dx, dy columns are not used; the positions
    come in separately). With the identity as rnd it is forward()'s z3, the split being exact algebra."""
    W1 = p["W1"]
    Wa, Wb, Wxy, Wt = W1[:, :F], W1[:, F:2 * F], W1[:, 2 * F:2 * F + 2], W1[:, 2 * F + 2]
    w = float(max(window, 1))
    P = rnd(rnd(x[:, :F]) @ rnd(Wa).T + p["b1"] - (model_xy @ Wxy.T) / 100.0)
    Q = rnd(rnd(x[:, F:2 * F]) @ rnd(Wb).T + (scene_xy @ Wxy.T) / 100.0)
    dt = rnd(np.rint(x[:, 2 * F + 2] * w))
    h1 = np.maximum(rnd(dt[:, None] * rnd(Wt / w)[None, :] + rnd(P + Q)), 0.0)
    z2 = h1 @ rnd(p["W2"]).T + rnd(p["b2"])
    return np.maximum(z2, 0.0) @ p["w3"] + p["b3"][0]


def adam(p, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step in place; state holds m, v and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m *= b1
        m += (1 - b1) * g[k]
        v *= b2
        v += (1 - b2) * g[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] -= lr * mh / (np.sqrt(vh) + eps)
    return p
