"""Pins of the FP64 MLP reference (oracle/mlp.py): backpropagation against central
finite differences, AdamW against closed forms, the loss at a known point, features."""
import numpy as np
import pytest

from oracle import mlp as M


def rand_params(rng, nin, h, nout, scale=0.5):
    return {name: rng.standard_normal(shp) * scale for name, shp in M.shapes(nin, h, nout)}


def test_backprop_matches_central_differences():
    rng = np.random.default_rng(0)
    nin, h, nout, batch = 10, 16, 8, 6
    p = rand_params(rng, nin, h, nout)
    X = rng.standard_normal((batch, nin))
    k = rng.integers(0, nout, batch)
    _, g = M.loss_and_grads(p, X, k)
    hstep = 1e-6
    worst = 0.0
    for name, shp in M.shapes(nin, h, nout):
        for _ in range(6):
            idx = tuple(int(rng.integers(0, s)) for s in shp)
            q = {n: v.copy() for n, v in p.items()}
            q[name][idx] += hstep
            lp, _ = M.loss_and_grads(q, X, k)
            q[name][idx] -= 2 * hstep
            lm, _ = M.loss_and_grads(q, X, k)
            fd = (lp - lm) / (2 * hstep)
            worst = max(worst, abs(fd - g[name][idx]) / max(abs(fd), 1e-3))
    assert worst <= 1e-6, worst


def test_loss_with_zero_output_layer_is_log_classes():
    rng = np.random.default_rng(1)
    nin, h, nout = 7, 12, 9
    p = rand_params(rng, nin, h, nout)
    p["W4"][:] = 0.0
    p["b4"][:] = 0.0
    loss, g = M.loss_and_grads(p, rng.standard_normal((4, nin)), [0, 3, 8, 1])
    assert abs(loss - np.log(nout)) <= 1e-15
    # uniform softmax: db4 = 1/nout - mean one-hot
    expect = np.full(nout, 1.0 / nout)
    for kk in [0, 3, 8, 1]:
        expect[kk] -= 0.25
    assert np.allclose(g["b4"], expect, atol=1e-15)


def test_adamw_first_step_closed_form():
    rng = np.random.default_rng(2)
    nin, h, nout = 5, 6, 4
    p = rand_params(rng, nin, h, nout)
    g = rand_params(rng, nin, h, nout)
    z = {n: np.zeros_like(v) for n, v in p.items()}
    lr, eps, wd = 1e-2, 1e-8, 0.1
    P, _, _ = M.adamw_step(p, g, z, z, 1, lr, eps=eps, wd=wd)
    for name in p:
        d = wd if name.startswith("W") else 0.0
        want = p[name] - lr * (g[name] / (np.abs(g[name]) + eps) + d * p[name])
        assert np.allclose(P[name], want, rtol=0, atol=1e-15)


def test_adamw_constant_gradient_moves_linearly():
    """With a constant gradient the bias-corrected moments equal g and g^2 exactly, so each
    step moves by lr * g / (|g| + eps) (no weight decay)."""
    rng = np.random.default_rng(3)
    nin, h, nout = 4, 5, 3
    p = rand_params(rng, nin, h, nout)
    g = rand_params(rng, nin, h, nout)
    m = {n: np.zeros_like(v) for n, v in p.items()}
    v = {n: np.zeros_like(x) for n, x in p.items()}
    q = p
    T, lr, eps = 7, 3e-3, 1e-8
    for t in range(1, T + 1):
        q, m, v = M.adamw_step(q, g, m, v, t, lr, eps=eps)
    for name in p:
        assert np.allclose(q[name], p[name] - T * lr * g[name] / (np.abs(g[name]) + eps), rtol=0, atol=1e-12)


def test_flatten_roundtrip_and_size():
    rng = np.random.default_rng(4)
    nin, h, nout = 130, 256, 128
    p = rand_params(rng, nin, h, nout)
    flat = M.flatten(p, nin, h, nout)
    assert flat.size == h * nin + h + 2 * (h * h + h) + nout * h + nout
    q = M.unflatten(flat, nin, h, nout)
    assert all(np.array_equal(p[n], q[n]) for n in p)


def test_features_normalised_curve():
    lam = np.array([1e4, 1e2, 1.0, 1e-2])
    f = M.features(lam, 0.25, 0.75)
    assert np.allclose(f, [1.0, 2.0 / 3.0, 1.0 / 3.0, 0.0, 0.25, 0.75], atol=1e-15)
    flat = M.features(np.ones(5), 0.5, 0.5)
    assert np.array_equal(flat[:5], np.zeros(5))
    # eigenvalues below lambda_1 * Nt * 2^-52 are floored
    tiny = M.features(np.array([1.0, 1e-30, 0.0]), 0.0, 0.0)
    assert tiny[1] == tiny[2] == 0.0
