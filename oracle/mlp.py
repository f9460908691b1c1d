"""CPU oracle for the learned row-size predictor (test infrastructure).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Plain numpy in
float64.

The paper sizes every output row exactly with a symbolic pass (Sec. 2.2);
the learned form replaces that pass, for rows it predicts well, by a small
multilayer perceptron 6 -> 64 -> 64 -> 1 with ReLU hidden layers, trained
with mean-squared error on log1p(n_nz) and the Adam update rule (Kingma &
Ba, 2015). This module states each piece in its plain textbook form:

- ``features``   per row of C = A*B, six numbers: log1p(nnz of the A row),
                 log1p(n_prod of the row), log1p of the max / mean / min
                 length of the B rows it references (0 when the A row is
                 empty) and log((i+1)/M) for row i of M.
- ``forward``    h1 = relu(X W1 + b1), h2 = relu(h1 W2 + b2), y = h2 w3 + b3.
- ``loss``       mean((y - t)^2).
- ``backward``   gradients of ``loss`` by the chain rule.
- ``adam``       one Adam step with bias correction.
- ``sizes``      predicted row size: ceil(expm1(y) * (1 + margin)), at least 1.

Parameter layout (4673 numbers in one flat vector, in this order):
W1 (6x64 row-major), b1 (64), W2 (64x64 row-major), b2 (64), w3 (64), b3 (1).
"""

from __future__ import annotations

import numpy as np

D_IN, H1, H2 = 6, 64, 64
SHAPES = [("W1", (D_IN, H1)), ("b1", (H1,)), ("W2", (H1, H2)), ("b2", (H2,)),
          ("w3", (H2,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 4673


def unpack(theta: np.ndarray) -> dict:
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.size == N_PARAMS, theta.size
    out, off = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[off:off + n].reshape(shape)
        off += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel()
                           for name, _ in SHAPES])


def features(A, B) -> np.ndarray:
    """(M, 6) float64 row features of C = A*B."""
    M = A.rows
    arpt = np.asarray(A.rpt, dtype=np.int64)
    brpt = np.asarray(B.rpt, dtype=np.int64)
    blen = np.diff(brpt)
    X = np.zeros((M, D_IN), dtype=np.float64)
    for i in range(M):
        ks = A.col[arpt[i]:arpt[i + 1]]
        lens = blen[ks] if ks.size else np.zeros(0, dtype=np.int64)
        X[i, 0] = np.log1p(ks.size)
        X[i, 1] = np.log1p(lens.sum())
        if ks.size:
            X[i, 2] = np.log1p(lens.max())
            X[i, 3] = np.log1p(lens.sum() / ks.size)
            X[i, 4] = np.log1p(lens.min())
        X[i, 5] = np.log((i + 1) / M)
    return X


def forward(theta: np.ndarray, X: np.ndarray):
    """Returns (y, cache) with y of shape (n,)."""
    p = unpack(theta)
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["w3"] + p["b3"][0]
    return y, (X, z1, h1, z2, h2)


def loss(y: np.ndarray, t: np.ndarray) -> float:
    d = y - t
    return float(np.mean(d * d))


def backward(theta: np.ndarray, X: np.ndarray, t: np.ndarray):
    """(loss, gradient as a flat 4673 vector) of mean((y - t)^2)."""
    p = unpack(theta)
    y, (X, z1, h1, z2, h2) = forward(theta, X)
    n = X.shape[0]
    dy = 2.0 * (y - t) / n                    # d loss / d y
    g = {}
    g["w3"] = h2.T @ dy
    g["b3"] = np.array([dy.sum()])
    dh2 = np.outer(dy, p["w3"])
    dz2 = dh2 * (z2 > 0)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"].T
    dz1 = dh1 * (z1 > 0)
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return loss(y, t), pack(g)


def adam(theta, grad, m, v, step: int, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (step counts from 1). Returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    theta = theta - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


def sizes(y: np.ndarray, margin: float) -> np.ndarray:
    """Predicted row sizes from log1p-space outputs."""
    s = np.ceil(np.expm1(np.asarray(y, dtype=np.float64)) * (1.0 + margin))
    return np.maximum(s, 1.0).astype(np.int64)
