"""FP64 reference of the rank-predictor MLP (test infrastructure only).

Three layers, 64 hidden units: y = sigmoid(w3 . relu(W2 relu(W1 x + b1) + b2)
+ b3), trained on the oracle's ranks with the target r_i / n_i and the mean
squared error.  Only tests/ use this module: it pins the GPU forward and
backward kernels (analytic gradient here, finite differences in the tests).

Flat parameter layout (shared with the C ABI): W1 (64 x NFEAT, row-major),
b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1).
"""
import numpy as np

from .ce import NFEAT

H = 64
NPARAM = H * NFEAT + H + H * H + H + H + 1


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = theta[o:o + H * NFEAT].reshape(H, NFEAT); o += H * NFEAT
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    w3 = theta[o:o + H]; o += H
    b3 = theta[o]
    return W1, b1, W2, b2, w3, b3


def forward(theta, X):
    """Predictions y (one per row of X) and the activations."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ w3 + b3
    y = 1.0 / (1.0 + np.exp(-z3))
    return y, (z1, h1, z2, h2, z3)


def loss(theta, X, t):
    y, _ = forward(theta, X)
    return 0.5 * np.mean((y - t) ** 2)


def grad(theta, X, t):
    """Analytic gradient of :func:`loss` (backpropagation), flat layout."""
    W1, b1, W2, b2, w3, b3 = unpack(theta)
    y, (z1, h1, z2, h2, z3) = forward(theta, X)
    S = X.shape[0]
    d3 = (y - t) * y * (1.0 - y) / S            # dL/dz3
    g_w3 = h2.T @ d3
    g_b3 = d3.sum()
    d2 = np.outer(d3, w3) * (z2 > 0)            # dL/dz2
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (z1 > 0)                   # dL/dz1
    g_W1 = d1.T @ X
    g_b1 = d1.sum(axis=0)
    return np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])


def init(seed):
    """He-normal weights from numpy.random.default_rng(seed), zero biases."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((H, NFEAT)) * np.sqrt(2.0 / NFEAT)
    W2 = rng.standard_normal((H, H)) * np.sqrt(2.0 / H)
    w3 = rng.standard_normal(H) * np.sqrt(2.0 / H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), w3, [0.0]])


def training_set(factors):
    """(features, r/n) of every block with a non-empty far row."""
    X, t = [], []
    for F in factors:
        for lev in F.levels:
            for st in lev.steps:
                if st.sigma.size and st.n > 0:
                    X.append(st.features)
                    t.append(st.r / st.n)
    return np.array(X), np.array(t)
