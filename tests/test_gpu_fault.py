"""Failure detection on the GPU without a fault: the bounded grid-barrier wait of the
cooperative Jacobi eigensolver is made to run out (one arrival withheld, a spin limit of a
few microseconds).  The kernel must record DFTFE_ERR_TIMEOUT, every CTA must return, the
entry point must report the status with X unchanged, and the next normal call on the same
handle must succeed with the oracle's result."""
import numpy as np
import pytest

import oracle
import synth
from systems import oracle_system, gpu_system, small_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DFTFE_ERR_TIMEOUT = 6


@pytest.fixture(scope="module")
def dg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_07820_gb300 as dg
    return dg


def test_eigensolver_wait_times_out_and_recovers(dg):
    c = small_case(7, n=(4, 4, 4), p=4, L=8.0, nl=True)
    om, oh = oracle_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
    mesh, ham = gpu_system(c["L"], c["n"], c["p"], c["centres"], c["depth"], c["width"], c["vquad"], c["proj"])
    try:
        N = 256                                  # 128 co-resident CTAs in the eigensolver
        Xo, _, _ = oracle.cholgs(synth.random_block(71, om.ndofs, N))
        X = torch.from_numpy(Xo.copy()).cuda()
        ev = torch.empty(N, dtype=torch.float64, device="cuda")
        dg.dftfe_ham_set_wait_test(ham, spin_limit=64, withhold_arrival=True)
        with pytest.raises(dg.DftfeError) as info:
            dg.dftfe_rayleigh_ritz(ham, X, ev)
        assert info.value.code == DFTFE_ERR_TIMEOUT
        torch.cuda.synchronize()                 # the context is still usable
        assert np.array_equal(X.cpu().numpy(), Xo)          # X untouched by the failed call
        dg.dftfe_ham_set_wait_test(ham, 0, False)
        dg.dftfe_rayleigh_ritz(ham, X, ev)
        _, _, theta, _ = oracle.rayleigh_ritz(oh.apply, Xo)
        assert np.abs(ev.cpu().numpy() - theta).max() < 1e-9
    finally:
        dg.dftfe_ham_destroy(ham)
        dg.dftfe_mesh_destroy(mesh)
