"""Chebyshev-filtered subspace iteration steps (oracle, FP64).

Filter (Eq. chebyfilter): Psi_f = T_m(Hbar) Psi_in with Hbar = (H~ - c)/e mapping
the unwanted interval [a, b] to [-1, 1], e = (b-a)/2, c = (b+a)/2, evaluated by the
three-term recurrence T_{k+1} = 2 x T_k - T_{k-1}.  The paper fixes neither c1, c2
nor a scaling; the oracle offers the unscaled recurrence and the scaled one of
Zhou & Saad (2007, the paper's ref. saad2006), which keeps the vectors O(1):
  sigma_1 = e/(a0 - c),  X_1 = sigma_1 (H~ - c) X_0 / e,
  sigma_{k+1} = 1/(2/sigma_1 - sigma_k),
  X_{k+1} = 2 sigma_{k+1} (H~ - c) X_k / e - sigma_k sigma_{k+1} X_{k-1}.
Degree m means m applications of H~.

Orthonormalisation and Rayleigh-Ritz (Alg. 2): the paper solves the GHEP
H^ Q = S Q D in the filtered basis via S = L L^T.  This build orthonormalises
first (Cholesky-Gram-Schmidt: S = X^T X = L L^T, X <- X L^-T, Alg. 2 steps 2a and
3b) and then solves the standard problem X^T H~ X = Q Theta Q^T (steps 1b, 2b-c,
3a); in exact arithmetic the Ritz pairs are identical (L^-1 H^ L^-T is step 2b).
"""
from dataclasses import dataclass
import math
import numpy as np
from scipy.linalg import solve_triangular


@dataclass
class Bounds:
    a: float            # lower end of the unwanted interval
    b: float            # upper bound of the spectrum
    a0: float = math.nan  # estimate of the lowest wanted eigenvalue (NaN: unscaled filter)


def chebyshev_filter(apply, X, degree, bounds):
    # real blocks stay float64; complex (Bloch) blocks stay complex128, the coefficients
    # are real either way
    X = np.array(X, dtype=np.result_type(np.asarray(X).dtype, np.float64), copy=True)
    if degree <= 0:
        return X
    e = (bounds.b - bounds.a) / 2.0
    c = (bounds.b + bounds.a) / 2.0
    if math.isnan(bounds.a0):
        Y = (apply(X) - c * X) / e
        for _ in range(2, degree + 1):
            Ynew = 2.0 * (apply(Y) - c * Y) / e - X
            X, Y = Y, Ynew
        return Y
    sigma = e / (bounds.a0 - c)
    sigma1 = sigma
    gamma = 2.0 / sigma1
    Y = (apply(X) - c * X) * (sigma1 / e)
    for _ in range(2, degree + 1):
        sigma2 = 1.0 / (gamma - sigma)
        Ynew = (apply(Y) - c * Y) * (2.0 * sigma2 / e) - (sigma * sigma2) * X
        X, Y = Y, Ynew
        sigma = sigma2
    return Y


def lanczos_bounds(apply, v0, k):
    """k-step Lanczos with full reorthogonalisation (twice, classical Gram-Schmidt).

    Returns (theta_min, theta_max, b) with b = theta_max + |beta_k|: the upper-bound
    estimator of Zhou and Saad (the paper's Chebyshev filtering reference), the largest Ritz
    value of T_k plus the norm of the last Lanczos residual f_k = beta_k v_{k+1}.
    """
    v = np.asarray(v0, np.float64).ravel()
    v = v / np.linalg.norm(v)
    V = [v]
    alpha, beta = [], []
    for j in range(k):
        w = apply(V[j])
        a = float(V[j] @ w)
        w = w - a * V[j]
        if j > 0:
            w = w - beta[j - 1] * V[j - 1]
        Vm = np.stack(V, axis=1)
        for _ in range(2):
            w = w - Vm @ (Vm.T @ w)
        alpha.append(a)
        bnorm = float(np.linalg.norm(w))
        beta.append(bnorm)
        if bnorm == 0.0:
            break
        V.append(w / bnorm)
    kk = len(alpha)
    T = np.diag(alpha) + np.diag(beta[:kk - 1], 1) + np.diag(beta[:kk - 1], -1)
    theta = np.linalg.eigvalsh(T)
    b = theta[-1] + abs(beta[kk - 1])
    return float(theta[0]), float(theta[-1]), float(b)


def first_pass_bounds(theta_min, b, nstates, ndofs, frac_min=0.05):
    """Bounds for the first pass from Lanczos: a0 = theta_min,
    a = theta_min + (b - theta_min) * max(4 N / M, frac_min)."""
    a = theta_min + (b - theta_min) * max(4.0 * nstates / ndofs, frac_min)
    return Bounds(a=a, b=b, a0=theta_min)


def cholgs(X):
    """S = X^T X, S = L L^T, X <- X L^-T (Alg. 2 steps 1a, 2a, 3b)."""
    X = np.asarray(X, np.float64)
    S = X.T @ X
    L = np.linalg.cholesky(S)
    return solve_triangular(L, X.T, lower=True).T, S, L


def sign_fix(Q):
    """Make the largest-|.| entry of each column positive (first such entry on ties)."""
    idx = np.argmax(np.abs(Q), axis=0)
    s = np.sign(Q[idx, np.arange(Q.shape[1])])
    s[s == 0] = 1.0
    return Q * s[None, :]


def rayleigh_ritz(apply, X):
    """W = H~ X, H^ = (X^T W + W^T X)/2 = Q Theta Q^T (ascending), X <- X Q, W <- W Q."""
    X = np.asarray(X, np.float64)
    W = apply(X)
    Hh = X.T @ W
    Hh = 0.5 * (Hh + Hh.T)
    theta, Q = np.linalg.eigh(Hh)
    Q = sign_fix(Q)
    return X @ Q, W @ Q, theta, Hh


def rrgep_alg2(apply, Psi):
    """Alg. 2 as printed (full spectrum): S = Psi^T Psi, H^ = Psi^T H~ Psi, S = L L^T,
    eigenvalues of L^-1 H^ L^-T.  Used to pin the CholGS + RR equivalence."""
    S = Psi.T @ Psi
    Hh = Psi.T @ apply(Psi)
    L = np.linalg.cholesky(S)
    A = solve_triangular(L, solve_triangular(L, Hh, lower=True).T, lower=True)
    return np.linalg.eigvalsh(0.5 * (A + A.T))


def residuals(X, W, theta, mass=None):
    """Löwdin-basis residual ||H~ x_i - theta_i x_i||_2 (x_i unit), and, if the lumped
    mass is given, the GHEP form ||H psi - theta M psi|| / ||psi|| with psi = M^-1/2 x."""
    R = W - X * theta[None, :]
    r = np.sqrt(np.sum(R * R, axis=0))
    if mass is None:
        return r
    m = np.asarray(mass)[:, None]
    num = np.sqrt(np.sum(m * R * R, axis=0))
    den = np.sqrt(np.sum(X * X / m, axis=0))
    return r, num / den


def chfsi_pass(ham, X, block, degree, bounds):
    """One pass: filter each column block, CholGS on all columns, RR, residuals,
    then the bounds update a <- theta_N, a0 <- theta_1 (b kept)."""
    X = np.array(X, dtype=np.float64, copy=True)
    N = X.shape[1]
    for j0 in range(0, N, block):
        j1 = min(N, j0 + block)
        X[:, j0:j1] = chebyshev_filter(ham.apply, X[:, j0:j1], degree, bounds)
    X, _, _ = cholgs(X)
    X, W, theta, _ = rayleigh_ritz(ham.apply, X)
    r = residuals(X, W, theta)
    nb = Bounds(a=float(theta[-1]), b=bounds.b,
                a0=bounds.a0 if math.isnan(bounds.a0) else float(theta[0]))
    return X, W, theta, r, nb
