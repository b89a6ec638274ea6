"""CPU oracle of the configuration predictor's network -- TEST INFRASTRUCTURE ONLY.

Only the tests import this module.  A plain float64 numpy restatement of the
3-layer MLP the library trains on the GPU: x (8) -> W1, b1 -> ReLU (64) ->
W2, b2 -> ReLU (64) -> W3, b3 (OUT outputs: 6 for the configuration network,
39 for the schedule network, read off the parameter count), with the loss
    L = sum_{s,c} mask[s,c] (out[s,c] - y[s,c])^2 / sum_{s,c} mask[s,c]
and its gradient by the chain rule.  Parameters are one flat vector in the
order W1[64][8], b1[64], W2[64][64], b2[64], W3[OUT][64], b3[OUT] (row =
output unit), the layout of the library's parameter arrays.
"""

from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 8, 64, 6


def sizes(n_out: int = N_OUT):
    return [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (n_out, N_H)),
            ("b3", (n_out,))]


SIZES = sizes(N_OUT)
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)
N_HIDDEN_PARAMS = N_H * N_IN + N_H + N_H * N_H + N_H


def n_outputs(theta) -> int:
    """Output count of a parameter vector: (len - hidden parameters) / (64 + 1)."""
    n = (len(theta) - N_HIDDEN_PARAMS) // (N_H + 1)
    assert N_HIDDEN_PARAMS + n * (N_H + 1) == len(theta), "not a parameter vector of this network"
    return n


def unpack(theta: np.ndarray) -> dict:
    out, off = {}, 0
    for name, shape in sizes(n_outputs(theta)):
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[off:off + n], dtype=np.float64).reshape(shape)
        off += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([p[name].reshape(-1) for name, _ in sizes(p["b3"].shape[0])])


def forward(theta, X):
    p = unpack(theta)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    out = h2 @ p["W3"].T + p["b3"]
    return out, (X, z1, h1, z2, h2)


def loss(theta, X, Y, M):
    out, _ = forward(theta, X)
    M = np.asarray(M, dtype=np.float64)
    cnt = max(M.sum(), 1.0)
    d = (out - np.asarray(Y, dtype=np.float64)) * M
    return float((d * d).sum() / cnt)


def loss_grad(theta, X, Y, M):
    """(loss, gradient) by the chain rule, layer by layer."""
    p = unpack(theta)
    out, (X, z1, h1, z2, h2) = forward(theta, X)
    M = np.asarray(M, dtype=np.float64)
    cnt = max(M.sum(), 1.0)
    d = (out - np.asarray(Y, dtype=np.float64)) * M
    L = float((d * d).sum() / cnt)
    dout = 2.0 * d * M / cnt                 # dL/dout
    g = {"W3": dout.T @ h2, "b3": dout.sum(0)}
    dh2 = dout @ p["W3"]
    dz2 = dh2 * (z2 > 0)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (z1 > 0)
    g["W1"] = dz1.T @ X
    g["b1"] = dz1.sum(0)
    return L, pack(g)


def predict(theta, X, legal):
    """Lowest-scoring legal configuration per row (-1 if none); ties to the lower index."""
    out, _ = forward(theta, X)
    res = []
    for s in range(out.shape[0]):
        best = -1
        for c in range(out.shape[1]):
            if not (int(legal[s]) >> c) & 1:
                continue
            if best < 0 or out[s, c] < out[s, best]:
                best = c
        res.append(best)
    return np.array(res, dtype=np.int64)
