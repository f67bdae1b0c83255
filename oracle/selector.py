"""FP64 oracle of the kernel-selection path: matrix features, the 16-64-64-24 MLP, its
masked squared-error loss, gradients and Adam steps.

TEST INFRASTRUCTURE ONLY (like the rest of this package).  Plain numpy in float64, written
from the definitions: each feature is its formula over the CSR arrays; the MLP is
y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 on standardised inputs; the gradients are the
chain rule written out; Adam is m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2,
w <- w - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np

F, H, V = 16, 64, 24
SIZES = [("W1", (H, F)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (V, H)), ("b3", (V,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(w):
    """Split the flat parameter vector into W1, b1, W2, b2, W3, b3."""
    w = np.asarray(w, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = w[o:o + n].reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SIZES])


def features(rowptr, colidx, M, K, N, dtype=0):
    """The 16 selector features, each from its definition (see gbsp_features)."""
    rp = np.asarray(rowptr, dtype=np.int64)
    ci = np.asarray(colidx, dtype=np.int64)
    L = np.diff(rp)
    nnz = int(L.sum())
    mean = nnz / M if M else 0.0
    var = max(float((L.astype(np.float64) ** 2).sum()) / M - mean * mean, 0.0) if M else 0.0
    sd = np.sqrt(var)
    mx = float(L.max()) if M else 0.0
    rows = np.repeat(np.arange(M, dtype=np.int64), L)
    centre = (rows * K) // M if M else rows
    d = np.abs(ci - centre)
    # consecutive entries of a row less than 8 columns apart
    same_row = rows[1:] == rows[:-1] if nnz > 1 else np.zeros(0, dtype=bool)
    gaps = np.abs(ci[1:] - ci[:-1]) if nnz > 1 else np.zeros(0, dtype=np.int64)
    pairs = int(np.maximum(L - 1, 0).sum())
    near = int(np.count_nonzero(same_row & (gaps < 8)))
    # entries (i, j) whose column j is also stored in row i + 1
    key = rows * (K + 1) + ci
    nxt = (rows - 1) * (K + 1) + ci  # an entry of row r seen from row r - 1
    vertical = int(np.count_nonzero(np.isin(key, nxt[rows > 0]) & (rows < M - 1))) if nnz else 0
    f = np.zeros(F)
    f[0] = np.log2(max(M, 1))
    f[1] = np.log2(max(K, 1))
    f[2] = np.log2(1 + nnz)
    f[3] = np.log2(max(nnz, 1) / (max(M, 1) * max(K, 1)))
    f[4] = np.log2(1 + mean)
    f[5] = np.log2(1 + sd)
    f[6] = sd / mean if mean > 0 else 0.0
    f[7] = np.log2(1 + mx)
    f[8] = mx / mean if mean > 0 else 0.0
    f[9] = np.count_nonzero(L == 0) / M if M else 0.0
    f[10] = d.sum() / nnz / K if nnz and K else 0.0
    f[11] = d.max() / K if nnz and K else 0.0
    f[12] = near / pairs if pairs else 0.0
    f[13] = vertical / nnz if nnz else 0.0
    f[14] = np.log2(max(N, 1))
    f[15] = dtype
    return f


def standardise(feats, norm):
    norm = np.asarray(norm, dtype=np.float64)
    return (np.asarray(feats, dtype=np.float64) - norm[:F]) / norm[F:]


def feature_norm(feats):
    x = np.asarray(feats, dtype=np.float64)
    mean = x.mean(axis=0)
    sd = np.sqrt(np.maximum((x * x).mean(axis=0) - mean * mean, 0.0))
    return np.concatenate([mean, np.where(sd > 0, sd, 1.0)])


def forward(w, x):
    """Returns y and the hidden activations for standardised inputs x (n x 16)."""
    p = unpack(w)
    a1 = x @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = h2 @ p["W3"].T + p["b3"]
    return y, (x, h1, h2)


def loss(w, x, targets, mask):
    y, _ = forward(w, x)
    cnt = max(float(np.sum(mask)), 1.0)
    return float(np.sum(mask * (y - targets) ** 2) / cnt)


def gradient(w, x, targets, mask):
    """Gradient of `loss` by the chain rule."""
    p = unpack(w)
    y, (x, h1, h2) = forward(w, x)
    cnt = max(float(np.sum(mask)), 1.0)
    dy = mask * 2.0 * (y - targets) / cnt
    g = {"W3": dy.T @ h2, "b3": dy.sum(axis=0)}
    d2 = (dy @ p["W3"]) * (h2 > 0)
    g["W2"], g["b2"] = d2.T @ h1, d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * (h1 > 0)
    g["W1"], g["b1"] = d1.T @ x, d1.sum(axis=0)
    return pack(g)


def train(w, adam, norm, feats, targets, mask, order, steps, batch, lr, t0=0, b1=0.9, b2=0.999, eps=1e-8):
    """`steps` Adam steps on minibatches taken in turn from `order` (wrapping)."""
    w = np.asarray(w, dtype=np.float64).copy()
    m = np.asarray(adam[:N_PARAMS], dtype=np.float64).copy()
    v = np.asarray(adam[N_PARAMS:], dtype=np.float64).copy()
    order = np.asarray(order, dtype=np.int64)
    x_all = standardise(feats, norm)
    for step in range(steps):
        base = (step * batch) % len(order)
        idx = order[(base + np.arange(batch)) % len(order)]
        g = gradient(w, x_all[idx], np.asarray(targets, np.float64)[idx], np.asarray(mask, np.float64)[idx])
        t = t0 + step + 1
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        w = w - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return w, np.concatenate([m, v])
