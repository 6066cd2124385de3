"""Oracle pins: GLL/Gauss rules, Lagrange tables, mesh numbering and lumped mass."""
import os
import numpy as np
import pytest

import oracle
from oracle.basis import gll_rule, gauss_rule, lagrange_table, lagrange_deriv_table

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_gll_p4_closed_form():
    ref = np.loadtxt(os.path.join(GOLD, "gll_p4.txt"))
    x, w = gll_rule(4)
    assert np.allclose(x, ref[:, 0], atol=1e-15)
    assert np.allclose(w, ref[:, 1], atol=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
def test_gll_exactness(p):
    x, w = gll_rule(p)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(0, 2 * p):                    # exact for degree <= 2p-1
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13
    if p >= 2:   # and not for 2p+? (degree 2p is not integrated exactly)
        assert abs(np.dot(w, x ** (2 * p)) - 2.0 / (2 * p + 1)) > 1e-6


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_exactness(n):
    x, w = gauss_rule(n)
    for k in range(0, 2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 4, 6, 7])
def test_lagrange_tables(p):
    x, _ = gll_rule(p)
    assert np.allclose(lagrange_table(x, x), np.eye(p + 1), atol=1e-13)
    pts = np.linspace(-1, 1, 11)
    D = lagrange_deriv_table(x, pts)
    T = lagrange_table(x, pts)
    assert np.allclose(T.sum(axis=1), 1.0, atol=1e-13)
    assert np.allclose(D.sum(axis=1), 0.0, atol=1e-11)          # derivative of a constant
    for k in range(1, p + 1):                                    # exact for degree <= p
        assert np.allclose(T @ x ** k, pts ** k, atol=1e-12)
        assert np.allclose(D @ x ** k, k * pts ** (k - 1), atol=1e-10)


def test_mesh_numbering_multiplicity():
    m = oracle.PeriodicMesh(7.0, (2, 3, 4), 3)
    counts = np.bincount(m.cell_map.ravel(), minlength=m.ndofs)
    assert counts.sum() == m.ncells * m.nodes_per_cell
    g = m.g
    idx = np.arange(m.ndofs)
    ix, iy, iz = idx % g[0], (idx // g[0]) % g[1], idx // (g[0] * g[1])
    on = [(i % m.p == 0).astype(int) for i in (ix, iy, iz)]
    # interior node in 1 cell, face 2, edge 4, corner 8 (periodic)
    assert np.array_equal(counts, 2 ** (on[0] + on[1] + on[2]))
    # no cell lists a node twice
    for c in range(m.ncells):
        assert np.unique(m.cell_map[c]).size == m.nodes_per_cell


def test_mesh_coords_match_map():
    m = oracle.PeriodicMesh((6.0, 8.0, 10.0), (2, 2, 3), 2)
    xyz = m.node_xyz()
    q = m.quad_xyz(vquad=1)            # GLL points are the nodes
    for c in range(m.ncells):
        assert np.allclose(xyz[m.cell_map[c]], np.mod(q[c], m.L), atol=1e-12)


@pytest.mark.parametrize("p", [1, 3, 5])
def test_lumped_mass(p):
    L = np.array([4.0, 5.0, 6.0])
    m = oracle.PeriodicMesh(L, (3, 2, 4), p)
    assert abs(m.mass.sum() - np.prod(L)) < 1e-11
    # Kronecker product of independently built 1D lumped masses
    x, w = gll_rule(p)
    m1 = []
    for d in range(3):
        h = L[d] / m.n[d]
        v = np.zeros(m.g[d])
        for c in range(m.n[d]):
            for a in range(p + 1):
                v[(c * p + a) % m.g[d]] += w[a] * h / 2
        m1.append(v)
    kron = np.kron(m1[2], np.kron(m1[1], m1[0]))
    assert np.allclose(m.mass, kron, rtol=1e-14)
