"""FP64 CPU oracle of the learned prefilter network (test infrastructure).

f(x) = normalize(W2 gelu(W1 x + b1) + b2) with the erf form of GELU,
gelu(v) = v * Phi(v), and the pair loss
    L = sum_i w_i (f(q_i) . f(d_i) - y_i)^2 / sum_i w_i.
Gradients are central finite differences of L in FP64: they use no backward
formula, so they check the GPU's backward kernels independently.
The paper ranks with full embeddings (App. D.2 step 3); this network is the
library's compression of that stage, so its oracle is its own definition.
"""
from __future__ import annotations

import math

import numpy as np

_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(v):
    v = np.asarray(v, np.float64)
    return v * 0.5 * (1.0 + _erf(v / math.sqrt(2.0)))


def forward(params, x):
    """f of the rows of x (used as given), FP64."""
    W1, b1, W2, b2 = (np.asarray(p, np.float64) for p in params)
    h = np.asarray(x, np.float64) @ W1.T + b1
    z = gelu(h) @ W2.T + b2
    return z / np.linalg.norm(z, axis=1, keepdims=True)


def loss(params, xq, xd, y, w=None):
    s = np.sum(forward(params, xq) * forward(params, xd), axis=1)
    w = np.ones(len(y)) if w is None else np.asarray(w, np.float64)
    return float(np.sum(w * (s - np.asarray(y, np.float64)) ** 2) / np.sum(w))


def flat(params):
    return np.concatenate([np.asarray(p, np.float64).ravel() for p in params])


def unflat(vec, shapes):
    out, o = [], 0
    for s in shapes:
        n = int(np.prod(s))
        out.append(vec[o:o + n].reshape(s))
        o += n
    return out


def fd_grad(params, xq, xd, y, w=None, idx=None, eps=1e-6):
    """Central differences of `loss` with respect to the flat parameters
    [W1 | b1 | W2 | b2] at the positions `idx` (all when None)."""
    shapes = [np.shape(p) for p in params]
    base = flat(params)
    idx = np.arange(base.size) if idx is None else np.asarray(idx)
    g = np.zeros(len(idx))
    for k, i in enumerate(idx):
        up, dn = base.copy(), base.copy()
        up[i] += eps
        dn[i] -= eps
        g[k] = (loss(unflat(up, shapes), xq, xd, y, w) - loss(unflat(dn, shapes), xq, xd, y, w)) / (2 * eps)
    return g
