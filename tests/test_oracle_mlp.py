"""Pins of the FP64 reference network of the learned degree/bounds proposer: gradients
against central finite differences, a linear special case against its closed-form gradient,
Adam's first step against its closed form, and a small regression that training solves."""
import numpy as np

import synth
from oracle import mlp

N_IN, N_H, N_OUT = 7, 6, 3


def _setup(seed=0, n=11):
    P = mlp.param_count(N_IN, N_H, N_OUT)
    p = mlp.init_params(synth.counter_uniform(seed, P), N_IN, N_H, N_OUT)
    X = synth.random_block(seed + 1, n, N_IN) * 2.0
    T = synth.random_block(seed + 2, n, N_OUT)
    w = np.array([1.0, 0.5, 2.0])
    return p, X, T, w


def test_param_count_and_packing_roundtrip():
    P = mlp.param_count(N_IN, N_H, N_OUT)
    assert P == N_H * N_IN + N_H + N_H * N_H + N_H + N_OUT * N_H + N_OUT
    p = np.arange(P, dtype=float)
    assert np.array_equal(mlp.pack(*mlp.unpack(p, N_IN, N_H, N_OUT)), p)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, N_IN, N_H, N_OUT)
    assert W1[1, 0] == N_IN and b1[0] == N_H * N_IN          # row-major W1, then b1


def test_gradient_matches_central_differences():
    p, X, T, w = _setup()
    L, g = mlp.loss_grad(p, X, T, w, N_IN, N_H, N_OUT)
    assert np.isclose(L, mlp.loss(p, X, T, w, N_IN, N_H, N_OUT))
    h = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (mlp.loss(p + e, X, T, w, N_IN, N_H, N_OUT) - mlp.loss(p - e, X, T, w, N_IN, N_H, N_OUT)) / (2 * h)
    assert np.abs(fd - g).max() <= 1e-7 * max(1.0, np.abs(g).max())


def test_linear_regime_matches_least_squares_gradient():
    """With W1, W2 tiny the tanh layers are linear to first order; with W1 = W2 = 0 the hidden
    layers are exactly tanh(b) constants and the loss is linear least squares in (W3, b3), whose
    gradient is 2/n sum_s w (y - t) [h2, 1]^T in closed form."""
    p, X, T, w = _setup(3)
    W1, b1, W2, b2, W3, b3 = mlp.unpack(p, N_IN, N_H, N_OUT)
    b1 = np.linspace(-0.5, 0.5, N_H)
    b2 = np.linspace(0.3, -0.2, N_H)
    q = mlp.pack(0 * W1, b1, 0 * W2, b2, W3, b3)
    L, g = mlp.loss_grad(q, X, T, w, N_IN, N_H, N_OUT)
    h2 = np.tanh(b2)
    y = W3 @ h2 + b3
    r = 2.0 * w * (y - T) / X.shape[0]                # n x n_out
    gW3 = np.outer(r.sum(axis=0), h2)
    gb3 = r.sum(axis=0)
    _, _, _, _, GW3, Gb3 = mlp.unpack(g, N_IN, N_H, N_OUT)
    assert np.allclose(GW3, gW3, rtol=1e-13, atol=1e-15)
    assert np.allclose(Gb3, gb3, rtol=1e-13, atol=1e-15)
    # W1 gets no gradient through a zero W2 (dh1 = dz2 W2 = 0)
    GW1 = mlp.unpack(g, N_IN, N_H, N_OUT)[0]
    assert np.all(GW1 == 0.0)


def test_adam_first_step_closed_form():
    """At t = 1 with zero moments the bias-corrected step is -lr g / (|g| + eps) elementwise."""
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p0 = np.ones(4)
    p1, m, v = mlp.adam_step(p0, g, np.zeros(4), np.zeros(4), 1, 0.01)
    assert np.allclose(p1, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_training_fits_a_smooth_map():
    """Full-batch Adam on y = (sin x1, x2 x3, x1 + x4) drives the loss down by 50x."""
    n = 256
    X = synth.random_block(7, n, N_IN) * 2.0
    T = np.stack([np.sin(X[:, 0]), X[:, 1] * X[:, 2], X[:, 0] + X[:, 3]], axis=1)
    w = np.ones(N_OUT)
    P = mlp.param_count(N_IN, 16, N_OUT)
    p = mlp.init_params(synth.counter_uniform(5, P), N_IN, 16, N_OUT)
    m = np.zeros(P)
    v = np.zeros(P)
    L0 = mlp.loss(p, X, T, w, N_IN, 16, N_OUT)
    for t in range(1, 1501):
        _, g = mlp.loss_grad(p, X, T, w, N_IN, 16, N_OUT)
        p, m, v = mlp.adam_step(p, g, m, v, t, 1e-2)
    assert mlp.loss(p, X, T, w, N_IN, 16, N_OUT) < L0 / 50
