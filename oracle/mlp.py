"""The learned degree/bounds proposer's network, FP64 reference (test infrastructure).

A three-layer perceptron x -> h1 = tanh(W1 x + b1) -> h2 = tanh(W2 h1 + b2) -> y = W3 h2 + b3
with a per-output weighted mean-squared loss and Adam (Kingma & Ba 2015) as the optimiser.
The parameters are packed in one flat vector in the order W1 (row-major, n_h x n_in), b1,
W2 (n_h x n_h), b2, W3 (n_out x n_h), b3 -- the layout the GPU kernels use.

Everything here is written from the definitions: the forward pass by matrix products, the
gradients by the chain rule written out layer by layer, Adam by its update formulas.  The
pins (tests/test_oracle_mlp.py) check the gradients against central finite differences,
a linear special case against its closed-form least-squares gradient, and Adam against its
first-step closed form.
"""
import numpy as np


def param_count(n_in, n_h, n_out):
    return n_h * n_in + n_h + n_h * n_h + n_h + n_out * n_h + n_out


def unpack(p, n_in, n_h, n_out):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + n_h * n_in].reshape(n_h, n_in); o += n_h * n_in
    b1 = p[o:o + n_h]; o += n_h
    W2 = p[o:o + n_h * n_h].reshape(n_h, n_h); o += n_h * n_h
    b2 = p[o:o + n_h]; o += n_h
    W3 = p[o:o + n_out * n_h].reshape(n_out, n_h); o += n_out * n_h
    b3 = p[o:o + n_out]; o += n_out
    assert o == p.size
    return W1, b1, W2, b2, W3, b3


def pack(W1, b1, W2, b2, W3, b3):
    return np.concatenate([np.ravel(a) for a in (W1, b1, W2, b2, W3, b3)])


def forward(p, X, n_in, n_h, n_out):
    """Outputs for the rows of X (n x n_in); also returns the hidden activations."""
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, n_h, n_out)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    y = h2 @ W3.T + b3
    return y, (X, h1, h2)


def loss(p, X, T, w, n_in, n_h, n_out):
    """L = (1/n) sum_s sum_k w_k (y_sk - t_sk)^2."""
    y, _ = forward(p, X, n_in, n_h, n_out)
    n = y.shape[0]
    return float(np.sum(np.asarray(w) * (y - T) ** 2) / n)


def loss_grad(p, X, T, w, n_in, n_h, n_out):
    """Loss and its gradient with respect to the packed parameters (chain rule by layer)."""
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, n_h, n_out)
    y, (X, h1, h2) = forward(p, X, n_in, n_h, n_out)
    n = y.shape[0]
    w = np.asarray(w, dtype=np.float64)
    L = float(np.sum(w * (y - T) ** 2) / n)
    dy = 2.0 * w * (y - T) / n            # dL/dy, n x n_out
    dW3 = dy.T @ h2
    db3 = dy.sum(axis=0)
    dh2 = dy @ W3                         # n x n_h
    dz2 = dh2 * (1.0 - h2 ** 2)           # tanh' = 1 - tanh^2
    dW2 = dz2.T @ h1
    db2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (1.0 - h1 ** 2)
    dW1 = dz1.T @ X
    db1 = dz1.sum(axis=0)
    return L, pack(dW1, db1, dW2, db2, dW3, db3)


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step number t >= 1); returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def init_params(seed_uniform, n_in, n_h, n_out):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases, from a supplied array of
    U(-1/2, 1/2) numbers of length param_count (the caller draws them)."""
    u = np.asarray(seed_uniform, dtype=np.float64) * 2.0
    W1, b1, W2, b2, W3, b3 = unpack(u, n_in, n_h, n_out)
    return pack(W1 / np.sqrt(n_in), 0 * b1, W2 / np.sqrt(n_h), 0 * b2, W3 / np.sqrt(n_h), 0 * b3)
