"""FP64 reference of the learned warm start: MLP, loss, gradients, Adam, POD.

The paper names learning methods only as future work (Sec. 8); these are the
textbook definitions used to check the GPU kernels:

* MLP y = W_L tanh(... tanh(W_1 x + b_1) ...) + b_L, weights W_l (out x in).
* loss L = 1 / (B n_out) sum_{i,j} w_j (y_ij - t_ij)^2.
* gradients by the chain rule (backpropagation); tanh' = 1 - tanh^2.
* Adam: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
  p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
* POD of snapshots Y (rows x cols, one snapshot per column): mean over
  columns, then the left singular vectors of the centred matrix and its
  singular values (library SVD).
* ridge least squares W = argmin |X W^T - Y|^2 + lam tr(X^T X) / n_in |W|^2
  (the linear part of the warm-start map), by the normal equations.

Parameters are packed as [W_1 (row-major), b_1, W_2, b_2, ...] in float64.
"""
import numpy as np


def layout(widths):
    offs = []
    o = 0
    for l in range(len(widths) - 1):
        wo = o
        o += widths[l] * widths[l + 1]
        bo = o
        o += widths[l + 1]
        offs.append((wo, bo))
    return offs, o


def unpack(p, widths):
    offs, _ = layout(widths)
    Ws, bs = [], []
    for l, (wo, bo) in enumerate(offs):
        Ws.append(p[wo:wo + widths[l] * widths[l + 1]].reshape(widths[l + 1], widths[l]))
        bs.append(p[bo:bo + widths[l + 1]])
    return Ws, bs


def forward(p, widths, X):
    Ws, bs = unpack(np.asarray(p, dtype=np.float64), widths)
    acts = [np.asarray(X, dtype=np.float64)]
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = acts[-1] @ W.T + b
        acts.append(np.tanh(z) if l + 1 < len(Ws) else z)
    return acts


def loss_grad(p, widths, X, T, w=None):
    """(L, dL/dp) for the weighted mean squared error."""
    p = np.asarray(p, dtype=np.float64)
    acts = forward(p, widths, X)
    Y = acts[-1]
    B, n_out = Y.shape
    wv = np.ones(n_out) if w is None else np.asarray(w, dtype=np.float64)
    D = Y - np.asarray(T, dtype=np.float64)
    L = float(np.sum(wv * D * D) / (B * n_out))
    Ws, _ = unpack(p, widths)
    offs, n = layout(widths)
    g = np.zeros(n)
    dz = 2.0 * wv * D / (B * n_out)
    for l in range(len(Ws) - 1, -1, -1):
        wo, bo = offs[l]
        g[wo:wo + Ws[l].size] = (dz.T @ acts[l]).ravel()
        g[bo:bo + Ws[l].shape[0]] = dz.sum(axis=0)
        if l > 0:
            da = dz @ Ws[l]
            dz = da * (1.0 - acts[l] ** 2)
    return L, g


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    p = p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return p, m, v


def pod(Y, r):
    """Mean, the r leading left singular vectors and singular values of Y - mean."""
    Y = np.asarray(Y, dtype=np.float64)
    mean = Y.mean(axis=1)
    U, s, _ = np.linalg.svd(Y - mean[:, None], full_matrices=False)
    return mean, U[:, :r], s[:r]


def linear_fit(X, Y, ridge):
    """W (n_out x n_in) of ridge least squares, normal equations in FP64."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    G = X.T @ X
    n = G.shape[0]
    return np.linalg.solve(G + ridge * np.trace(G) / n * np.eye(n), X.T @ Y).T
