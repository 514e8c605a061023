"""FP64 reference of the learned-rank MLP and its training step.

TEST INFRASTRUCTURE ONLY: only tests/ may import this module.  It shares no
code with the CUDA library (paper_2405_11105_b300/csrc/k_mlp.cu).

The paper has no learned component; this network is the learned thresholding
rule of the build: per window it maps the normalised log-eigenvalue spectrum
(the curve of thresholding method 1, Eq. 6) plus the window centre to a
distribution over the cutoff k (number of rejected components).

Model (plain definitions, no fusion):
    A0 = X                                   (batch x nin), nin = Nt + 2
    Z_l = A_{l-1} W_l^T + b_l,  A_l = max(Z_l, 0)    l = 1, 2, 3 (hidden H)
    Z_4 = A_3 W_4^T + b_4                    (batch x Nt) logits over k = 0..Nt-1
    loss = mean_s [ log sum_j exp(Z_4[s, j]) - Z_4[s, k_s] ]
AdamW (decoupled weight decay on the weight matrices only):
    m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2
    p = p - lr * ( (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps) + wd * p )

Flat parameter layout (shared with the C ABI): W1 (H x nin, row-major), b1 (H),
W2 (H x H), b2, W3 (H x H), b3, W4 (Nt x H), b4 (Nt).
"""
from __future__ import annotations

import numpy as np


def shapes(nin: int, hidden: int, nout: int):
    return [("W1", (hidden, nin)), ("b1", (hidden,)), ("W2", (hidden, hidden)), ("b2", (hidden,)),
            ("W3", (hidden, hidden)), ("b3", (hidden,)), ("W4", (nout, hidden)), ("b4", (nout,))]


def unflatten(flat, nin, hidden, nout):
    out, o = {}, 0
    for name, shp in shapes(nin, hidden, nout):
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def flatten(params, nin, hidden, nout):
    return np.concatenate([np.asarray(params[name], np.float64).ravel() for name, _ in shapes(nin, hidden, nout)])


def forward(p, X):
    X = np.asarray(X, np.float64)
    Z1 = X @ p["W1"].T + p["b1"]
    A1 = np.maximum(Z1, 0.0)
    Z2 = A1 @ p["W2"].T + p["b2"]
    A2 = np.maximum(Z2, 0.0)
    Z3 = A2 @ p["W3"].T + p["b3"]
    A3 = np.maximum(Z3, 0.0)
    Z4 = A3 @ p["W4"].T + p["b4"]
    return Z4, (X, Z1, A1, Z2, A2, Z3, A3)


def loss_and_grads(p, X, k):
    """Mean softmax cross-entropy over the batch and its gradients (backpropagation)."""
    Z4, (A0, Z1, A1, Z2, A2, Z3, A3) = forward(p, X)
    k = np.asarray(k, np.int64)
    M = Z4.shape[0]
    zmax = Z4.max(axis=1, keepdims=True)
    e = np.exp(Z4 - zmax)
    s = e.sum(axis=1, keepdims=True)
    loss = float(np.mean(np.log(s[:, 0]) + zmax[:, 0] - Z4[np.arange(M), k]))
    dZ4 = e / s
    dZ4[np.arange(M), k] -= 1.0
    dZ4 /= M
    g = {"W4": dZ4.T @ A3, "b4": dZ4.sum(axis=0)}
    dZ3 = (dZ4 @ p["W4"]) * (Z3 > 0)
    g["W3"], g["b3"] = dZ3.T @ A2, dZ3.sum(axis=0)
    dZ2 = (dZ3 @ p["W3"]) * (Z2 > 0)
    g["W2"], g["b2"] = dZ2.T @ A1, dZ2.sum(axis=0)
    dZ1 = (dZ2 @ p["W2"]) * (Z1 > 0)
    g["W1"], g["b1"] = dZ1.T @ A0, dZ1.sum(axis=0)
    return loss, g


def adamw_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW update (t counts from 1); weight decay on W1..W4 only.  Returns new (p, m, v)."""
    P, Mo, V = {}, {}, {}
    for name in p:
        Mo[name] = beta1 * m[name] + (1.0 - beta1) * g[name]
        V[name] = beta2 * v[name] + (1.0 - beta2) * g[name] ** 2
        mh = Mo[name] / (1.0 - beta1 ** t)
        vh = V[name] / (1.0 - beta2 ** t)
        decay = wd if name.startswith("W") else 0.0
        P[name] = p[name] - lr * (mh / (np.sqrt(vh) + eps) + decay * p[name])
    return P, Mo, V


def features(lam_sorted, pos_z, pos_x):
    """MLP input of one window: the spectrum normalised like method 1's curve, then the
    window centre.  lam_sorted descending; y_i = log10(max(lam_i, lam_1 Nt 2^-52)), mapped
    to (y_i - y_Nt) / (y_1 - y_Nt) in [0, 1] (0 if the curve is flat)."""
    lam = np.asarray(lam_sorted, np.float64)
    n = lam.size
    y = np.log10(np.maximum(lam, lam[0] * n * 2.0 ** -52))
    span = y[0] - y[-1]
    yn = (y - y[-1]) / span if span > 0 else np.zeros(n)
    return np.concatenate([yn, [pos_z, pos_x]])
