"""Float64 reference of the 12-32-1 network behind the learned starting bound
(test infrastructure; only tests, the smoke check and the benchmark's CPU
baseline use it).

The paper has no learned component; this network only proposes a starting k,
and every answer is still certified by exact decide runs.

Network: z = W1 x + b1 (32), h = relu(z), yhat = W2 h + b2 (1).
Loss: mean squared error L = (1/B) * sum_b (yhat_b - y_b)^2.
Gradients (relu'(z) taken as 1 iff z > 0):
  g_b = 2 (yhat_b - y_b) / B
  dW2 = sum_b g_b h_b^T, db2 = sum_b g_b
  dz_b = (W2^T g_b) * [z_b > 0]
  dW1 = sum_b dz_b x_b^T, db1 = sum_b dz_b
Adam (Kingma & Ba 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
  p -= lr * (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps).

Flat parameter layout (449 values): W1 row-major [32][12], b1[32], W2[32],
b2[1].
"""

from __future__ import annotations

import numpy as np

N_IN, N_HID = 12, 32
N_PARAMS = N_HID * N_IN + N_HID + N_HID + 1


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + N_HID * N_IN].reshape(N_HID, N_IN); o += N_HID * N_IN
    b1 = p[o:o + N_HID]; o += N_HID
    W2 = p[o:o + N_HID]; o += N_HID
    b2 = p[o]
    return W1, b1, W2, b2


def forward(p: np.ndarray, X: np.ndarray):
    W1, b1, W2, b2 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z = X @ W1.T + b1
    h = np.maximum(z, 0.0)
    yhat = h @ W2 + b2
    return z, h, yhat


def loss(p, X, y) -> float:
    _, _, yhat = forward(p, X)
    d = yhat - np.asarray(y, dtype=np.float64)
    return float(np.mean(d * d))


def grad(p: np.ndarray, X: np.ndarray, y: np.ndarray) -> np.ndarray:
    W1, b1, W2, b2 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    z, h, yhat = forward(p, X)
    B = X.shape[0]
    g = 2.0 * (yhat - np.asarray(y, dtype=np.float64)) / B
    dW2 = h.T @ g
    db2 = g.sum()
    dz = np.outer(g, W2) * (z > 0)
    dW1 = dz.T @ X
    db1 = dz.sum(axis=0)
    return np.concatenate([dW1.reshape(-1), db1, dW2, [db2]])


def adam_step(p, g, m, v, t, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    p = p - lr * mhat / (np.sqrt(vhat) + eps)
    return p, m, v
