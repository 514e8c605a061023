"""Training of the learned cutoff rule (LCF_T_LEARNED), on the GPU.

The network (include/lcf.h, lcf_mlp_*) predicts the cutoff k that thresholding
method 1 (maximum curvature of the normalised log-eigenvalue curve, Eq. 6)
picks on a fully converged EVD, from the spectrum of an EVD stopped after a
few Jacobi sweeps plus the window centre.  With it a plan runs the EVD with a
small sweep cap: the top-k (rejected) subspace and the kept eigenvalue sum
that the hard weights and alpha (Eq. 13) need converge long before the whole
spectrum does, and the rule that would read the unconverged tail is replaced
by the network.  The paper has no learned component.

Data: for every synthetic packet the library itself produces the pair
(features of the capped-sweep spectrum, method-1 cutoff of the converged
spectrum); nothing here computes the filter on the host.
"""
from __future__ import annotations

import numpy as np

from . import (LCF_EVD_PAIR, LCF_PATH_SIMT, LCF_PATH_TC, LCF_T_CURVATURE, Mlp, Plan)


def features(lam_sorted, pos_z, pos_x):
    """Network input of one window: y_i = log10 max(lambda_i, lambda_1 Nt 2^-52) mapped to
    (y_i - y_Nt) / (y_1 - y_Nt) (0 for a flat curve), then the window centre."""
    lam = np.asarray(lam_sorted, np.float64)
    n = lam.size
    fl = lam[0] * n * 2.220446049250313e-16
    y = np.log10(np.maximum(lam, fl))
    span = y[0] - y[-1]
    yn = (y - y[-1]) / span if span > 0 else np.zeros(n)
    return np.concatenate([yn, [pos_z, pos_x]]).astype(np.float32)


def window_centres(wz, wx):
    k = np.arange(wz * wx)
    return (k // wx + 0.5) / wz, (k % wx + 0.5) / wx


def make_plans(nz, nx, nt, wz, wx, fast_sweeps, beta=1.0, device=0):
    """(converged plan with method 1, capped-sweep plan with method 1) for one geometry."""
    tc = LCF_PATH_TC if nt <= 128 else LCF_PATH_SIMT
    full = Plan.make(nz, nx, nt, wz, wx, device=device, thresh_mode=LCF_T_CURVATURE, beta=beta,
                     gram_path=tc, project_path=LCF_PATH_TC, evd_path=LCF_EVD_PAIR)
    fast = Plan.make(nz, nx, nt, wz, wx, device=device, thresh_mode=LCF_T_CURVATURE, beta=beta,
                     gram_path=tc, project_path=LCF_PATH_TC, evd_path=LCF_EVD_PAIR, max_sweeps=fast_sweeps)
    return full, fast


def collect(packets, full: Plan, fast: Plan, wz, wx):
    """Features (capped-sweep spectra) and labels (converged method-1 cutoffs) of every
    window of every packet (each a [nt][nz][nx] complex64 array or device tensor)."""
    import torch
    pz, px = window_centres(wz, wx)
    X, K = [], []
    for iq in packets:
        d = iq if torch.is_tensor(iq) else torch.from_numpy(np.ascontiguousarray(iq)).cuda()
        full.filter(d)
        k_ref = full.debug()["k"].astype(np.int32)
        fast.filter(d)
        lam = fast.debug()["lam"]
        for w in range(lam.shape[0]):
            X.append(features(lam[w], pz[w], px[w]))
        K.append(k_ref)
    return np.stack(X), np.concatenate(K)


def init_params(nin, hidden, nout, seed=0):
    """He-uniform weights, zero biases, in the flat layout of lcf_mlp."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((nin, hidden), (hidden, hidden), (hidden, hidden), (hidden, nout)):
        lim = np.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, (fan_out, fan_in)).ravel())
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def train(X, K, nt, hidden=256, epochs=30, batch=512, lr=2e-3, wd=1e-4, seed=0, device=0, log=None):
    """Train a network on (X, K) with minibatch AdamW; returns the Mlp (parameters on the device)."""
    import torch
    dev = f"cuda:{device}"
    net = Mlp(nt, hidden=hidden, max_batch=batch, device=device)
    net.set_params(init_params(nt + 2, hidden, nt, seed))
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(dev)
    Kd = torch.from_numpy(np.ascontiguousarray(K, np.int32)).to(dev)
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = Xd.shape[0]
    steps = max(1, n // batch)
    total = epochs * steps
    t = 0
    for ep in range(epochs):
        order = torch.randperm(n, generator=g).to(dev)
        running = 0.0
        for s in range(steps):
            idx = order[s * batch:(s + 1) * batch]
            # cosine decay of the step size
            lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * t / total))
            running += net.loss_grad(Xd[idx], Kd[idx])
            net.adamw(lr_t, wd=wd)
            t += 1
        if log is not None:
            log(ep, running / steps)
    return net


def accuracy(net: Mlp, X, K):
    import torch
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda()
    pred = []
    for s in range(0, Xd.shape[0], net.max_batch):
        pred.append(net.forward(Xd[s:s + net.max_batch]).argmax(dim=1).cpu().numpy())
    pred = np.concatenate(pred)
    return float(np.mean(pred == np.asarray(K))), pred
