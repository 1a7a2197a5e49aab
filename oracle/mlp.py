"""Plain fp64 oracle of the learned early-stop model (a project addition; the
paper has no learned component in its method).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

Model: 2-layer perceptron with 8 inputs, 64 ReLU hidden units, one logit.
  z = x W1 + b1   (W1: [8, 64])      h = max(z, 0)
  s = h . W2 + b2 (W2: [64])         p = sigmoid(s)
Loss: mean binary cross-entropy with logits over the batch,
  L = mean( log(1 + exp(s)) - y s ).
Parameters are packed in one flat vector of 641 values:
  W1 (row-major, input-major) | b1 | W2 | b2.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 8, 64
N_PARAMS = N_IN * N_HID + N_HID + N_HID + 1


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    W1 = p[o:o + N_IN * N_HID].reshape(N_IN, N_HID)
    o += N_IN * N_HID
    b1 = p[o:o + N_HID]
    o += N_HID
    W2 = p[o:o + N_HID]
    o += N_HID
    b2 = p[o]
    return W1, b1, W2, b2


def pack(W1, b1, W2, b2):
    return np.concatenate([np.ravel(W1), b1, W2, [b2]]).astype(np.float64)


def forward(params, X):
    """Logits s for every row of X [n, 8]."""
    W1, b1, W2, b2 = unpack(params)
    X = np.asarray(X, dtype=np.float64)
    h = np.maximum(X @ W1 + b1, 0.0)
    return h @ W2 + b2


def loss_and_grad(params, X, y):
    """Mean BCE-with-logits loss and its gradient (same packing as params),
    by the chain rule written out step by step."""
    W1, b1, W2, b2 = unpack(params)
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = X.shape[0]
    z = X @ W1 + b1
    h = np.maximum(z, 0.0)
    s = h @ W2 + b2
    # log(1 + e^s) computed stably
    loss = float(np.mean(np.logaddexp(0.0, s) - y * s))
    ds = (1.0 / (1.0 + np.exp(-s)) - y) / n          # dL/ds
    gW2 = h.T @ ds
    gb2 = ds.sum()
    dh = np.outer(ds, W2)
    dz = dh * (z > 0)
    gW1 = X.T @ dz
    gb1 = dz.sum(axis=0)
    return loss, pack(gW1, gb1, gW2, gb2)


def round_f16(params):
    """The fp16 copy the search kernel reads (round to nearest even)."""
    return np.asarray(params, dtype=np.float64).astype(np.float16).astype(np.float64)


# ---------------------------------------------------------------- entry-point model
# A second 2-layer perceptron (a project addition) that picks where a search enters the
# graph: from the query vector q (d values) it scores E coarse cells of the objects.
#   x = s q                       (s: a fixed input scale, parameter 0, not trained)
#   z = x W1 + b1  (W1: [d, 64])  h = max(z, 0)
#   t = h W2 + b2  (W2: [64, E])  one logit per cell
# Loss: mean softmax cross-entropy over the batch with the cell of each query's answer as
# the label, L = mean( logsumexp(t) - t[label] ).
# Packing: s | W1 (input-major) | b1 | W2 (hidden-major) | b2.
ENTRY_HID = 64


def entry_size(d, E):
    return 1 + d * ENTRY_HID + ENTRY_HID + ENTRY_HID * E + E


def entry_unpack(params, d, E):
    p = np.asarray(params, dtype=np.float64)
    assert p.shape == (entry_size(d, E),)
    o = 0
    s = p[o]
    o += 1
    W1 = p[o:o + d * ENTRY_HID].reshape(d, ENTRY_HID)
    o += d * ENTRY_HID
    b1 = p[o:o + ENTRY_HID]
    o += ENTRY_HID
    W2 = p[o:o + ENTRY_HID * E].reshape(ENTRY_HID, E)
    o += ENTRY_HID * E
    b2 = p[o:o + E]
    return s, W1, b1, W2, b2


def entry_pack(s, W1, b1, W2, b2):
    return np.concatenate([[s], np.ravel(W1), b1, np.ravel(W2), b2]).astype(np.float64)


def entry_forward(params, Q, d, E):
    """Cell logits [n, E] for the query rows Q [n, d]."""
    s, W1, b1, W2, b2 = entry_unpack(params, d, E)
    h = np.maximum((s * np.asarray(Q, np.float64)) @ W1 + b1, 0.0)
    return h @ W2 + b2


def entry_loss_and_grad(params, Q, labels, d, E):
    """Mean softmax cross-entropy and its gradient (same packing; the scale's entry is 0,
    it is not trained), by the chain rule step by step."""
    s, W1, b1, W2, b2 = entry_unpack(params, d, E)
    X = s * np.asarray(Q, np.float64)
    y = np.asarray(labels, np.int64)
    n = X.shape[0]
    z = X @ W1 + b1
    h = np.maximum(z, 0.0)
    t = h @ W2 + b2
    tmax = t.max(axis=1, keepdims=True)
    lse = (tmax + np.log(np.exp(t - tmax).sum(axis=1, keepdims=True)))[:, 0]
    loss = float(np.mean(lse - t[np.arange(n), y]))
    prob = np.exp(t - lse[:, None])
    dt = prob.copy()
    dt[np.arange(n), y] -= 1.0
    dt /= n                                   # dL/dt
    gW2 = h.T @ dt
    gb2 = dt.sum(axis=0)
    dz = (dt @ W2.T) * (z > 0)
    gW1 = X.T @ dz
    gb1 = dz.sum(axis=0)
    return loss, entry_pack(0.0, gW1, gb1, gW2, gb2)
