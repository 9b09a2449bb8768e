"""FP64 reference of the schedule-policy network (test infrastructure only).

The network maps six features of a level to eight outputs; outputs 0..2 are
read as the predicted log2 device time of the level under push, filtered push
and pull, and the scheduler takes the smallest.  It is fitted to per-level
traces with a masked squared error: for a row whose level ran with action a
and took log2-time y, the loss is (out[a] - y)^2; the other outputs get no
gradient from that row.

Parameter vector (the library's layout): input mean[6], input scale[6],
W1[32][6], b1[32], W2[32][32], b2[32], W3[8][32], b3[8].  Inputs are
normalised as (x - mean) / scale; both hidden layers are ReLU; the output
layer is linear.

This module writes the forward pass, the loss, its gradient by the chain rule
(backpropagation), and an Adam step (Kingma and Ba, ICLR 2015) plainly in
numpy float64.  It is pinned in tests/test_mlp_oracle.py by finite
differences and closed-form special cases.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 6, 32, 8
SHAPES = [("mu", (N_IN,)), ("sd", (N_IN,)), ("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)),
          ("b2", (N_HID,)), ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    """Views of the flat parameter vector by name."""
    out, k = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = p[k:k + size].reshape(shape)
        k += size
    return out


def features(units, groups, colours, frontier_lanes, m):
    """The six per-level features the library computes in its scheduler."""
    units = np.asarray(units, np.float64)
    groups = np.asarray(groups, np.float64)
    colours = np.asarray(colours, np.float64)
    lanes = np.asarray(frontier_lanes, np.float64)
    return np.stack([np.log2(1 + units), np.log2(1 + groups), np.log2(1 + colours), np.log2(1 + lanes),
                     np.log2(1 + 4 * groups) - np.log2(1 + float(m)),
                     np.log2(1 + colours / np.maximum(units, 1))], axis=1)


def forward(p, X):
    """Outputs [rows, 8] and the intermediate values backprop needs."""
    P = unpack(np.asarray(p, np.float64))
    Xn = (np.asarray(X, np.float64) - P["mu"]) / P["sd"]
    a1 = Xn @ P["W1"].T + P["b1"]
    h1 = np.maximum(a1, 0)
    a2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(a2, 0)
    out = h2 @ P["W3"].T + P["b3"]
    return out, (Xn, a1, h1, a2, h2)


def loss(p, X, action, y):
    """Mean over rows of (out[row, action[row]] - y[row])^2."""
    out, _ = forward(p, X)
    r = out[np.arange(len(y)), np.asarray(action)] - np.asarray(y, np.float64)
    return float(np.mean(r * r))


def loss_grad(p, X, action, y):
    """Loss and its gradient with respect to the weights and biases (the
    input mean and scale are fixed: their gradient entries are zero)."""
    P = unpack(np.asarray(p, np.float64))
    out, (Xn, a1, h1, a2, h2) = forward(p, X)
    B = len(y)
    rows = np.arange(B)
    action = np.asarray(action)
    r = out[rows, action] - np.asarray(y, np.float64)
    d_out = np.zeros_like(out)
    d_out[rows, action] = 2.0 * r / B
    g = {name: np.zeros(shape) for name, shape in SHAPES}
    g["W3"] = d_out.T @ h2
    g["b3"] = d_out.sum(0)
    d_h2 = d_out @ P["W3"]
    d_a2 = d_h2 * (a2 > 0)
    g["W2"] = d_a2.T @ h1
    g["b2"] = d_a2.sum(0)
    d_h1 = d_a2 @ P["W2"]
    d_a1 = d_h1 * (a1 > 0)
    g["W1"] = d_a1.T @ Xn
    g["b1"] = d_a1.sum(0)
    flat = np.concatenate([g[name].ravel() for name, _ in SHAPES])
    return float(np.mean(r * r)), flat


def adam_step(p, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of the weights and biases (t counts from 1); the input
    mean and scale are not trained."""
    p = np.array(p, np.float64)
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    step = lr * mh / (np.sqrt(vh) + eps)
    step[:2 * N_IN] = 0.0
    return p - step, m, v


def predict_action(p, X, allowed=(0, 1, 2)):
    """The action with the smallest predicted log-time among `allowed`."""
    out, _ = forward(p, X)
    allowed = list(allowed)
    return np.asarray(allowed)[np.argmin(out[:, allowed], axis=1)]
