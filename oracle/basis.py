"""1D ingredients of the spectral finite-element basis (oracle, FP64).

The paper's basis is C0 Lagrange polynomials on Gauss-Lobatto-Legendre (GLL)
nodes (Sec. 2.3, Eq. fem), with GLL quadrature making the mass matrix diagonal
(text after Eq. hep).  The local-potential term uses an n_q-point rule per cell
(Eq. quadLocal); the paper does not fix n_q, and it is read here as a
Gauss-Legendre rule with p+1 points per axis.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def legendre(n, x):
    """P_n(x) through numpy's Legendre series (library primitive)."""
    c = np.zeros(n + 1)
    c[n] = 1.0
    return npleg.legval(x, c)


def gll_rule(p):
    """GLL nodes (ascending) and weights for degree p (p+1 points).

    Nodes: -1, +1 and the roots of P_p'(x).  Weights: 2 / (p (p+1) P_p(x_i)^2).
    """
    c = np.zeros(p + 1)
    c[p] = 1.0
    interior = np.sort(np.real(npleg.legroots(npleg.legder(c)))) if p >= 2 else np.zeros(0)
    x = np.concatenate([[-1.0], interior, [1.0]])
    # polish the interior roots with Newton steps on P_p' (library-evaluated)
    d1 = npleg.legder(c)
    d2 = npleg.legder(c, 2)
    for _ in range(3):
        if p >= 2:
            xi = x[1:-1]
            x[1:-1] = xi - npleg.legval(xi, d1) / npleg.legval(xi, d2)
    w = 2.0 / (p * (p + 1) * legendre(p, x) ** 2)
    return x, w


def gauss_rule(n):
    """n-point Gauss-Legendre rule on [-1, 1] (library primitive)."""
    x, w = npleg.leggauss(n)
    return x, w


def lagrange_table(nodes, pts):
    """T[q, j] = l_j(pts[q]), l_j the Lagrange polynomial of `nodes` at node j."""
    nodes = np.asarray(nodes, np.float64)
    pts = np.asarray(pts, np.float64)
    n = nodes.size
    T = np.ones((pts.size, n))
    for j in range(n):
        for m in range(n):
            if m != j:
                T[:, j] *= (pts - nodes[m]) / (nodes[j] - nodes[m])
    return T


def lagrange_deriv_table(nodes, pts):
    """T[q, j] = l_j'(pts[q]) by the product rule:
    l_j'(x) = sum_{k != j} 1/(x_j - x_k) * prod_{m != j, k} (x - x_m)/(x_j - x_m)."""
    nodes = np.asarray(nodes, np.float64)
    pts = np.asarray(pts, np.float64)
    n = nodes.size
    T = np.zeros((pts.size, n))
    for j in range(n):
        for k in range(n):
            if k == j:
                continue
            term = np.full(pts.size, 1.0 / (nodes[j] - nodes[k]))
            for m in range(n):
                if m != j and m != k:
                    term = term * (pts - nodes[m]) / (nodes[j] - nodes[m])
            T[:, j] += term
    return T
