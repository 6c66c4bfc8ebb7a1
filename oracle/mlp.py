"""FP64 numpy oracle of the format selector's network (test infrastructure only).

Network: 12 features -> 64 (ReLU) -> 64 (ReLU) -> C outputs, one predicted
log-time per candidate kernel class.  Loss: masked mean squared error
L = sum_{s,c} M_sc (out_sc - y_sc)^2 / sum_{s,c} M_sc, where M_sc = 0 marks a
class that was not measured for sample s.  Parameters are stored as
W1 [64, 12], b1 [64], W2 [64, 64], b2 [64], W3 [C, 64], b3 [C] (row-major,
output-major).  The update rule is Adam (Kingma and Ba, ICLR 2015).

Matrix products use numpy's matmul as a library primitive; the backward
pass is the chain rule written out layer by layer.
"""
from __future__ import annotations

import numpy as np

NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def shapes(n_in: int = 12, hidden: int = 64, n_out: int = 8):
    return dict(W1=(hidden, n_in), b1=(hidden,), W2=(hidden, hidden), b2=(hidden,),
                W3=(n_out, hidden), b3=(n_out,))


def forward(P, X):
    """Returns (out [B, C], cache)."""
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    out = h2 @ P["W3"].T + P["b3"]
    return out, (X, z1, h1, z2, h2)


def loss(P, X, Y, M):
    out, _ = forward(P, X)
    d = out - Y
    return float(np.sum(M * d * d) / np.sum(M))


def loss_and_grad(P, X, Y, M):
    """Masked MSE and its gradient with respect to every parameter."""
    out, (X, z1, h1, z2, h2) = forward(P, X)
    denom = np.sum(M)
    d = out - Y
    L = float(np.sum(M * d * d) / denom)
    dout = 2.0 * M * d / denom
    g = {}
    g["W3"] = dout.T @ h2
    g["b3"] = dout.sum(axis=0)
    dz2 = (dout @ P["W3"]) * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ P["W2"]) * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(axis=0)
    return L, g


def adam_step(P, g, state, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); ``state`` holds m and v per parameter."""
    for k in NAMES:
        m = state.setdefault("m_" + k, np.zeros_like(P[k]))
        v = state.setdefault("v_" + k, np.zeros_like(P[k]))
        m[...] = beta1 * m + (1.0 - beta1) * g[k]
        v[...] = beta2 * v + (1.0 - beta2) * g[k] * g[k]
        mh = m / (1.0 - beta1 ** t)
        vh = v / (1.0 - beta2 ** t)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)
    return P
