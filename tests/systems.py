"""Seeded test systems built twice from the same synth inputs: once in the oracle,
once through the C ABI (each side evaluates the model functions at its own mesh
points)."""
import math
import numpy as np

import oracle
import synth


def oracle_system(L, n, p, centres, depth, width, vquad=0, proj=None):
    m = oracle.PeriodicMesh(L, n, p)
    h = oracle.Hamiltonian(m, vquad=vquad)
    Lb = np.broadcast_to(np.asarray(L, float), (3,))
    h.set_potential(synth.gaussian_wells(m.quad_xyz(vquad).reshape(-1, 3), centres, depth, width, Lb[0]))
    if proj is not None:
        cent, w, rc, hcoup = proj
        rowptr, node, chi = synth.projector_csr(m.node_xyz(), cent, w, rc, Lb[0])
        h.set_nonlocal(hcoup, rowptr, node, chi)
    return m, h


def gpu_system(L, n, p, centres, depth, width, vquad=0, proj=None):
    import torch
    import paper_2203_07820_gb300 as dg
    mesh = dg.dftfe_mesh_create(L, n, p, vquad=vquad)
    ham = dg.dftfe_ham_create(mesh)
    nxyz, qxyz = dg.dftfe_mesh_coords(mesh)
    Lb = np.broadcast_to(np.asarray(L, float), (3,))
    v = synth.gaussian_wells(qxyz.reshape(-1, 3), centres, depth, width, Lb[0])
    dg.dftfe_ham_set_potential(ham, torch.from_numpy(v).cuda())
    if proj is not None:
        cent, w, rc, hcoup = proj
        rowptr, node, chi = synth.projector_csr(nxyz, cent, w, rc, Lb[0])
        dg.dftfe_ham_set_nonlocal(ham, hcoup, rowptr, node, chi)
    torch.cuda.synchronize()
    return mesh, ham


def small_case(seed=0, n=(4, 3, 2), p=4, L=8.0, nl=True, vquad=0):
    """A cube with a non-uniform cell count (odd axis -> 3 colours) and projectors."""
    s = synth.Stream(seed)
    cent = np.array([[L * s.uniform() for _ in range(3)] for _ in range(3)])
    proj = None
    if nl:
        hc = np.array([0.5 + 1.5 * s.uniform() for _ in range(4 * len(cent))])
        proj = (cent, 1.0, 2.5, hc)
    return dict(L=L, n=n, p=p, centres=cent, depth=2.0, width=1.0, vquad=vquad, proj=proj)


def oracle_rows(om, oh, rows, ncol, seed, with_nonlocal=True, absolute=False):
    """Rows `rows` of H~ X (or of |H~| |X|) for X = synth.random_block(seed, M, ncol),
    computed cell by cell without forming X: only the rows the touched cells need are
    generated.  The oracle's potential must be set for every touched cell."""
    rows = np.asarray(rows)
    flat = om.cell_map.ravel()
    out = np.zeros((len(rows), ncol))
    cache = {}
    for r, j in enumerate(rows):
        for s in np.nonzero(flat == j)[0]:
            c, l = divmod(int(s), om.nodes_per_cell)
            if c not in cache:
                Hc = oh.cell_matrix(c)
                Xc = synth.random_rows(seed, om.cell_map[c], ncol)
                cache[c] = (np.abs(Hc), np.abs(Xc)) if absolute else (Hc, Xc)
            Hc, Xc = cache[c]
            out[r] += Hc[l] @ Xc
    if with_nonlocal and oh.Ct is not None:
        sup = np.unique(oh.Ct.tocoo().row)
        Xs = synth.random_rows(seed, sup, ncol)
        Ct = oh.Ct.tocsr()[sup]                      # support rows only
        if absolute:
            P = np.abs(oh.h)[:, None] * (abs(Ct).T @ np.abs(Xs))
            out += abs(oh.Ct.tocsr()[rows]) @ P
        else:
            P = oh.h[:, None] * (Ct.T @ Xs)
            out += oh.Ct.tocsr()[rows] @ P
    return out
