"""dftfe_cholgs_noalloc: Cholesky-Gram-Schmidt for callers that cannot allocate device
memory where they orthonormalise (a fixed pool that must not grow, a framework step
that forbids cudaMalloc).  It must give dftfe_cholgs's result, call after call, from
its static scratch array.  This file is collected last on purpose."""
import ctypes as C
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-11    # the CholGS parity tolerance used by the other GPU tests


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_07820_gb300 as dg
    return dg


def test_noalloc_cholgs_matches_cholgs_on_consecutive_calls(dg):
    mesh = dg.dftfe_mesh_create(10.0, 6, 4)          # 13,824 DoFs
    ham = dg.dftfe_ham_create(mesh)
    M = dg.dftfe_mesh_info(mesh)[0]
    lib = dg.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (seed, N) in enumerate([(1, 64), (2, 37)]):     # two calls in a row, new sizes
        X0 = synth.random_block(seed, M, N) @ np.diag(np.linspace(1.0, 30.0, N))
        Xa = torch.from_numpy(X0).cuda()
        Xb = torch.from_numpy(X0).cuda()
        dg.dftfe_cholgs(ham, Xa)                                 # existing entry point
        rc = lib.dftfe_cholgs_noalloc(C.c_void_p(Xb.data_ptr()), Xb.stride(0), M, N, stream)
        assert rc == 0, dg.dftfe_last_error()
        torch.cuda.synchronize()
        a, b = Xa.cpu().numpy(), Xb.cpu().numpy()
        assert np.abs(b - a).max() <= TOL * np.abs(a).max(), f"call {call}"
        assert np.abs(b.T @ b - np.eye(N)).max() < 1e-12
    dg.dftfe_ham_destroy(ham)
    dg.dftfe_mesh_destroy(mesh)


def test_noalloc_cholgs_at_its_column_limit_on_a_non_blocking_stream(dg):
    """512 columns (the scratch bound caps the split count and the status word sits at the
    end of the array) on a stream created with non-blocking flags, twice in a row."""
    mesh = dg.dftfe_mesh_create(10.0, 6, 4)          # 13,824 DoFs
    ham = dg.dftfe_ham_create(mesh)
    M = dg.dftfe_mesh_info(mesh)[0]
    lib = dg.lib()
    s = torch.cuda.Stream()
    N = 512
    for seed in (3, 4):
        X0 = synth.random_block(seed, M, N) @ np.diag(np.linspace(1.0, 8.0, N))
        Xa = torch.from_numpy(X0).cuda()
        Xb = torch.from_numpy(X0).cuda()
        torch.cuda.synchronize()
        dg.dftfe_cholgs(ham, Xa)
        rc = lib.dftfe_cholgs_noalloc(C.c_void_p(Xb.data_ptr()), Xb.stride(0), M, N, C.c_void_p(s.cuda_stream))
        assert rc == 0, dg.dftfe_last_error()
        torch.cuda.synchronize()
        a, b = Xa.cpu().numpy(), Xb.cpu().numpy()
        assert np.abs(b - a).max() <= TOL * np.abs(a).max(), seed
    dg.dftfe_ham_destroy(ham)
    dg.dftfe_mesh_destroy(mesh)


def test_noalloc_cholgs_rejects_host_memory(dg):
    lib = dg.lib()
    M, N = 100, 4
    Xh = np.zeros((M, N))
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.dftfe_cholgs_noalloc(Xh.ctypes.data_as(C.c_void_p), N, M, N, stream)
    assert rc == 1 and "device" in dg.dftfe_last_error()


def test_noalloc_cholgs_rejects_sizes_beyond_its_scratch(dg):
    lib = dg.lib()
    M, N = 2000, 513
    X = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.dftfe_cholgs_noalloc(C.c_void_p(X.data_ptr()), N, M, N, stream)
    assert rc == 1 and "512" in dg.dftfe_last_error()
