"""GPU parity at N = 1,024 states: the widest subspace the precision form uses (32^3 cells,
1,024 states).  These sizes take the blocked Cholesky and triangular inverse (32 block
columns), the cooperative Jacobi eigensolver at 1,024 and the subspace GEMMs with eight
128-column tiles.  The system is a 4^3-cell, p = 4 box (4,096 DoFs) with wells and
projectors, small enough for the FP64 oracle (and a dense eigensolve of H~) to check every
output."""
import numpy as np
import pytest

import oracle
import synth
from systems import oracle_system, gpu_system, small_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 1024


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_07820_gb300 as dg
    return dg


@pytest.fixture(scope="module")
def pair(dg):
    c = small_case(5, n=(4, 4, 4), p=4, L=8.0, nl=True)
    om, oh = oracle_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
    mesh, ham = gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
    yield om, oh, mesh, ham
    dg.dftfe_ham_destroy(ham)
    dg.dftfe_mesh_destroy(mesh)


@pytest.fixture(scope="module")
def dense_eig(pair):
    om, oh, _, _ = pair
    return np.linalg.eigh(oh.dense())


def test_cholgs_1024_fp64(dg, pair):
    om, oh, mesh, ham = pair
    X0 = synth.random_block(61, om.ndofs, N)
    X = torch.from_numpy(X0).cuda()
    dg.dftfe_cholgs(ham, X)
    ref, _, _ = oracle.cholgs(X0)
    assert np.abs(X.cpu().numpy() - ref).max() < 1e-11


def test_cholgs_1024_mixed(dg, pair):
    """TF32x3 off-diagonal overlap and rotation: X^T X = I to FP32 level and the span of the
    oracle's orthonormal block."""
    om, oh, mesh, ham = pair
    X0 = synth.random_block(62, om.ndofs, N)
    X = torch.from_numpy(X0).cuda()
    dg.dftfe_cholgs(ham, X, dg.DFTFE_MIXED_TF32X3)
    x = X.cpu().numpy()
    assert np.abs(x.T @ x - np.eye(N)).max() < 1e-4
    ref, _, _ = oracle.cholgs(X0)
    # same span: the projections of the oracle's basis onto the GPU basis keep their norm
    P = x.T @ ref
    assert np.abs(np.linalg.svd(P, compute_uv=False) - 1.0).max() < 1e-4


def test_rayleigh_ritz_1024_fp64(dg, pair):
    om, oh, mesh, ham = pair
    Xo, _, _ = oracle.cholgs(synth.random_block(63, om.ndofs, N))
    X = torch.from_numpy(Xo.copy()).cuda()
    ev = torch.empty(N, dtype=torch.float64, device="cuda")
    W = torch.empty_like(X)
    dg.dftfe_rayleigh_ritz(ham, X, ev, W)
    Xr, Wr, theta, _ = oracle.rayleigh_ritz(oh.apply, Xo)
    assert np.abs(ev.cpu().numpy() - theta).max() < 1e-9
    # residual norms of the rotated pairs agree (unique even where vectors are not)
    r = torch.empty(N, dtype=torch.float64, device="cuda")
    dg.dftfe_residuals(ham, X, W, ev, r, 0)
    assert np.abs(r.cpu().numpy() - oracle.residuals(Xr, Wr, theta)).max() < 1e-8


def test_rayleigh_ritz_1024_mixed_near_converged(dg, pair, dense_eig):
    """The mixed scheme's regime: a basis close to the lowest 1,024 eigenvectors (a dense
    oracle eigensolve plus 1e-3 noise); Ritz values within 1e-6 Ha of the oracle's."""
    om, oh, mesh, ham = pair
    lam, V = dense_eig
    Xo, _, _ = oracle.cholgs(V[:, :N] + 1e-3 * synth.random_block(64, om.ndofs, N))
    X = torch.from_numpy(Xo.copy()).cuda()
    ev = torch.empty(N, dtype=torch.float64, device="cuda")
    dg.dftfe_rayleigh_ritz(ham, X, ev, None, dg.DFTFE_MIXED_TF32X3)
    _, _, theta, _ = oracle.rayleigh_ritz(oh.apply, Xo)
    assert np.abs(ev.cpu().numpy() - theta).max() < 1e-6


def test_pass_1024_fp64(dg, pair):
    """One FP64 pass (8 blocks of 128, degree 6) against the oracle's pass."""
    om, oh, mesh, ham = pair
    X0 = synth.random_block(65, om.ndofs, N)
    tmin, _, b = oracle.lanczos_bounds(oh.apply, synth.counter_uniform(66, om.ndofs), 20)
    bd = oracle.Bounds(tmin + 0.3 * (b - tmin), b, tmin)       # 1,024 of 4,096 states wanted
    _, _, theta, r, nb = oracle.chfsi_pass(oh, X0, 128, 6, bd)
    X = torch.from_numpy(X0).cuda()
    gb = dg.make_bounds(bd.a, bd.b, bd.a0)
    ev = torch.empty(N, dtype=torch.float64, device="cuda")
    rs = torch.empty(N, dtype=torch.float64, device="cuda")
    dg.dftfe_chfsi_pass(ham, X, 128, 6, gb, ev, rs)
    assert np.abs(ev.cpu().numpy() - theta).max() < 1e-9
    assert abs(gb.a - nb.a) < 1e-9 and abs(gb.a0 - nb.a0) < 1e-9
