"""C-ABI checks that need no GPU: the library loads, exports every declared entry
point, validates arguments on the host, and its host-side mesh geometry (a1)
matches the oracle."""
import os
import re
import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2203_07820_gb300 as dg
    return dg


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "dftfe_gb300.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dftfe_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(dg):
    syms = declared_symbols()
    assert len(syms) >= 20
    lib = dg.lib()
    for s in syms:
        assert hasattr(lib, s), s


def test_no_cpu_fallback_symbols(dg):
    # the binding holds no numerics: every public function forwards to the library
    import inspect
    src = inspect.getsource(dg)
    assert "numpy.linalg" not in src and "torch.matmul" not in src and "oracle" not in src.replace("oracle is", "")


@pytest.mark.parametrize("L,n,p,vquad", [(10.0, 2, 3, 0), ((4.0, 5.0, 6.0), (2, 3, 4), 4, 0),
                                         (7.0, 3, 6, 1), (30.0, 2, 6, 0)])
def test_mesh_geometry_matches_oracle(dg, L, n, p, vquad):
    import oracle
    mesh = dg.dftfe_mesh_create(L, n, p, vquad=vquad)
    nd, ncl, npc, nqp = dg.dftfe_mesh_info(mesh)
    om = oracle.PeriodicMesh(L, n, p)
    assert (nd, ncl, npc) == (om.ndofs, om.ncells, om.nodes_per_cell)
    x, q = dg.dftfe_mesh_coords(mesh)
    assert np.abs(x - om.node_xyz()).max() < 1e-13
    assert np.abs(q - om.quad_xyz(vquad)).max() < 1e-13
    dg.dftfe_mesh_destroy(mesh)


@pytest.mark.parametrize("kw", [dict(ncell=1), dict(degree=0), dict(degree=9), dict(vquad=2),
                                dict(nq1d=13), dict(L=-1.0)])
def test_mesh_argument_errors(dg, kw):
    args = dict(L=10.0, ncell=2, degree=3, vquad=0, nq1d=0)
    args.update(kw)
    with pytest.raises(dg.DftfeError) as e:
        dg.dftfe_mesh_create(args["L"], args["ncell"], args["degree"], args["vquad"], args["nq1d"])
    assert e.value.code == 1
    assert dg.dftfe_last_error() != ""


def test_non_periodic_rejected(dg):
    import ctypes as C
    d = dg.MeshDesc((C.c_double * 3)(5, 5, 5), (C.c_int * 3)(2, 2, 2), 3, (C.c_int * 3)(1, 0, 1), 0, 0)
    out = C.c_void_p()
    assert dg.lib().dftfe_mesh_create(C.byref(d), C.byref(out)) == 1


def test_null_arguments_rejected(dg):
    lib = dg.lib()
    assert lib.dftfe_mesh_create(None, None) == 1
    assert lib.dftfe_mesh_info(None, None, None, None, None) == 1
    assert lib.dftfe_ham_apply(None, None, 0, None, 0, 0, 0) == 1
    assert lib.dftfe_chfsi_pass(None, None, 0, 0, 0, 0, None, None, None, 0) == 1
    assert lib.dftfe_random_uniform(None, -1, 0, 0, None) == 1


def _g1_tilde(L, n, p):
    """m^-1/2 G1 m^-1/2 for the 1D periodic mesh, G1 assembled from int l_a l_b' = w_a l_b'(x_a)."""
    from oracle.basis import gll_rule, lagrange_deriv_table
    x, w = gll_rule(p)
    D = lagrange_deriv_table(x, x)
    h = L / n
    g = n * p
    G1 = np.zeros((g, g))
    m1 = np.zeros(g)
    for c in range(n):
        idx = [(c * p + a) % g for a in range(p + 1)]
        G1[np.ix_(idx, idx)] += w[:, None] * D
        m1[idx] += w * h / 2
    s = 1.0 / np.sqrt(m1)
    return s[:, None] * G1 * s[None, :]


@pytest.mark.parametrize("L,n,p,k", [((6.0, 7.0, 8.0), (3, 4, 5), 4, (0.3, -0.7, 1.1)),
                                     ((5.0, 5.0, 9.0), (3, 3, 3), 6, (0.25, 0.0, -0.4)),
                                     ((4.0, 6.0, 5.0), (2, 2, 3), 3, (0.5, 0.2, 0.1)),
                                     ((3.0, 4.0, 5.0), (2, 3, 4), 1, (0.7, -0.1, 0.3)),
                                     ((6.0, 6.0, 7.0), (2, 3, 2), 8, (0.2, 0.4, -0.6))])
def test_kpoint_stencil_table_matches_1d_assembly(dg, L, n, p, k):
    """The library's k.grad stencil (host table, no GPU) against the 1D periodic operator
    assembled here: every entry k_d G~1_d(i, i + o), summed where two offsets reach the same
    node (two cells per axis)."""
    mesh = dg.dftfe_mesh_create(L, n, p)
    tab = dg.dftfe_mesh_kpoint_stencil(mesh, k, p)
    dg.dftfe_mesh_destroy(mesh)
    for d in range(3):
        G = k[d] * _g1_tilde(L[d], n[d], p)
        g = n[d] * p
        for c in range(n[d]):
            for a in range(p):
                i = c * p + a
                row = np.zeros(g)
                for o in range(-p, p + 1):
                    row[(i + o) % g] += tab[d, a, o + p]
                assert np.abs(row - G[i]).max() <= 1e-13 * max(1.0, np.abs(G).max()), (d, c, a)


def test_null_arguments_rejected_by_the_kpoint_graph_and_tuning_calls(dg):
    """The k-point, graph, autotuner and batch-graph entry points check their handles and
    arguments on the host (no GPU needed for the refusals)."""
    import ctypes as C
    lib = dg.lib()
    k = (C.c_double * 3)(0.1, 0.2, 0.3)
    assert lib.dftfe_ham_set_kpoint(None, k, None) == 1
    assert lib.dftfe_ham_apply_z(None, None, 0, None, 0, 0, 0) == 1
    assert lib.dftfe_lanczos_z(None, 20, None, 0, None) == 1
    assert lib.dftfe_spectrum_bounds_z(None, 20, 0, 4, None) == 1
    assert lib.dftfe_chebyshev_filter_z(None, None, 0, 0, 0, None, 0) == 1
    assert lib.dftfe_cholgs_z(None, None, 0, 0, 0) == 1
    assert lib.dftfe_rayleigh_ritz_z(None, None, 0, 0, None, None, 0, 0) == 1
    assert lib.dftfe_residuals_z(None, None, None, 0, 0, None, None, 0) == 1
    assert lib.dftfe_chfsi_pass_z(None, None, 0, 0, 0, 0, None, None, None, 0) == 1
    assert lib.dftfe_ham_use_graphs(None, 1) == 1
    assert lib.dftfe_graph_query(None, None, None) == 1
    assert lib.dftfe_ham_autotune(None, 1) == 1
    assert lib.dftfe_autotune_query(None, 8, None, None, None) == 1
    assert lib.dftfe_batch_use_graphs(None, 1) == 1
    assert lib.dftfe_batch_graph_query(None, None, None) == 1
    # the shared local operator and the split-precision tuner
    out = C.c_void_p()
    assert lib.dftfe_ham_create_shared(None, C.byref(out)) == 1 and out.value is None
    i = [C.c_int(7) for _ in range(6)]
    t = [C.c_double(7.0) for _ in range(2)]
    assert lib.dftfe_autotune_query_mixed(None, *[C.byref(x) for x in i[:3]], *[C.byref(x) for x in t]) == 1
    assert lib.dftfe_batch_autotune(None, 1) == 1
    assert lib.dftfe_batch_autotune_query(None, 0, *[C.byref(x) for x in i], *[C.byref(x) for x in t]) == 1
    assert all(x.value == 7 for x in i) and all(x.value == 7.0 for x in t)     # outputs untouched
    mesh = dg.dftfe_mesh_create(6.0, 2, 3)
    try:
        assert lib.dftfe_mesh_kpoint_stencil(mesh, None, None) == 1
        bad = np.array([0.1, np.nan, 0.0])
        out = np.zeros(3 * 3 * 7)
        assert lib.dftfe_mesh_kpoint_stencil(mesh, bad.ctypes.data_as(C.c_void_p),
                                             out.ctypes.data_as(C.c_void_p)) == 1
        assert np.all(out == 0.0)                       # outputs untouched on DFTFE_ERR_ARG
    finally:
        dg.dftfe_mesh_destroy(mesh)
