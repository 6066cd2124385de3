"""The learned proposer's network kernels (forward, loss gradient, Adam) through the C ABI
against the FP64 reference network on the same seeded inputs."""
import numpy as np
import pytest

import synth
from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(19, 64, 3), (7, 32, 2), (64, 128, 8)]


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_07820_gb300 as dg
    return dg


def _case(shape, n, seed):
    n_in, n_h, n_out = shape
    P = mlp.param_count(*shape)
    p = mlp.init_params(synth.counter_uniform(seed, P), *shape)
    # biases nonzero so every parameter block is exercised
    p = p + 0.05 * synth.counter_uniform(seed + 50, P)
    X = synth.random_block(seed + 1, n, n_in) * 3.0
    T = synth.random_block(seed + 2, n, n_out)
    w = 0.5 + np.abs(synth.counter_uniform(seed + 3, n_out))
    return p, X, T, w


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("n", [1, 37, 1000])
def test_forward_matches_reference(dg, shape, n):
    p, X, T, w = _case(shape, n, 11)
    assert dg.dftfe_mlp_param_count(*shape) == p.size
    Y = torch.empty((n, shape[2]), dtype=torch.float32, device="cuda")
    # the reference runs on the FP32-rounded inputs the kernel sees
    p32, X32 = p.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64)
    dg.dftfe_mlp_forward(_t(p), shape, _t(X), Y)
    ref, _ = mlp.forward(p32, X32, *shape)
    assert np.abs(Y.cpu().numpy() - ref).max() <= 2e-5 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("n", [1, 37, 1000])
def test_loss_gradient_matches_reference(dg, shape, n):
    p, X, T, w = _case(shape, n, 21)
    P = p.size
    grad = torch.empty(P, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    dg.dftfe_mlp_loss_grad(_t(p), shape, _t(X), _t(T), _t(w), loss, grad)
    f = lambda a: a.astype(np.float32).astype(np.float64)
    L, g = mlp.loss_grad(f(p), f(X), f(T), f(w), *shape)
    assert abs(loss.item() - L) <= 1e-5 * max(1.0, abs(L))
    gg = grad.cpu().numpy()
    assert np.abs(gg - g).max() <= 1e-5 * max(1.0, np.abs(g).max())
    # deterministic: a second call gives the same bits
    grad2 = torch.empty_like(grad)
    dg.dftfe_mlp_loss_grad(_t(p), shape, _t(X), _t(T), _t(w), None, grad2)
    assert torch.equal(grad, grad2)


def test_adam_matches_reference(dg):
    P = 5000
    p = synth.counter_uniform(1, P)
    m = np.zeros(P)
    v = np.zeros(P)
    tp, tm, tv = _t(p), _t(m), _t(v)
    for t in range(1, 6):
        g = synth.counter_uniform(10 + t, P) * (0.1 ** (t % 3))
        p, m, v = mlp.adam_step(p, g, m, v, t, 1e-2)
        dg.dftfe_mlp_adam(tp, _t(g), tm, tv, t, 1e-2)
    assert np.abs(tp.cpu().numpy() - p).max() <= 1e-6
    assert np.abs(tm.cpu().numpy() - m).max() <= 1e-7


def test_gpu_training_reduces_loss_like_reference(dg):
    """Full-batch Adam with the GPU kernels on the smooth map of the reference pin."""
    shape = (7, 32, 3)
    n = 256
    X = synth.random_block(7, n, 7) * 2.0
    T = np.stack([np.sin(X[:, 0]), X[:, 1] * X[:, 2], X[:, 0] + X[:, 3]], axis=1)
    P = mlp.param_count(*shape)
    p = mlp.init_params(synth.counter_uniform(5, P), *shape)
    tp, tX, tT = _t(p), _t(X), _t(T)
    tm = torch.zeros(P, dtype=torch.float32, device="cuda")
    tv = torch.zeros_like(tm)
    g = torch.empty_like(tm)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    dg.dftfe_mlp_loss_grad(tp, shape, tX, tT, None, loss, g)
    L0 = loss.item()
    for t in range(1, 1501):
        dg.dftfe_mlp_loss_grad(tp, shape, tX, tT, None, loss, g)
        dg.dftfe_mlp_adam(tp, g, tm, tv, t, 1e-2)
    dg.dftfe_mlp_loss_grad(tp, shape, tX, tT, None, loss, g)
    assert loss.item() < L0 / 50
    # the trained GPU network evaluated by the reference gives the same loss
    Lref = mlp.loss(tp.cpu().numpy().astype(np.float64), X, T, np.ones(3), *shape)
    assert abs(Lref - loss.item()) <= 1e-3 * max(Lref, 1e-6) + 1e-6
