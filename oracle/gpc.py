"""Stochastic Galerkin matrices G_l and H_l of Section 3.2.

Oracle (test infrastructure only; see oracle/__init__.py).

[G_l]_rs = <xi_l psi_r psi_s> (l = 0..m, xi_0 = 1) and [H_l]_rs = <psi_l psi_r psi_s>
(l = 1..n_xi), with psi_r the m-variate Legendre chaos, orthonormal for xi_k
i.i.d. uniform on [-sqrt 3, sqrt 3] (Section 5.1): psi_alpha(xi) = prod_k
p_{alpha_k}(xi_k) with p_n(x) = sqrt(2n+1) P_n(x / sqrt 3).  Expectations are
products of 1-D Gauss-Legendre integrals, exact for these polynomial degrees.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def p1d(n, x):
    """Orthonormal 1-D Legendre polynomial of degree n for U(-sqrt 3, sqrt 3)."""
    c = np.zeros(n + 1); c[n] = 1.0
    return np.sqrt(2 * n + 1) * npleg.legval(x / np.sqrt(3.0), c)


def _gauss(npts):
    x, w = npleg.leggauss(npts)
    return np.sqrt(3.0) * x, w / 2.0          # expectation weights sum to 1


def triple_1d(dmax):
    """T[a, b, c] = <p_a p_b p_c> and X[a, b] = <xi p_a p_b>, degrees <= dmax (1-D)."""
    x, w = _gauss(3 * dmax + 4)
    P = np.array([p1d(n, x) for n in range(dmax + 1)])
    T = np.einsum("q,aq,bq,cq->abc", w, P, P, P)
    X = np.einsum("q,q,aq,bq->ab", w, x, P, P)
    return T, X


def g_matrices(mi):
    """G_0..G_m (list of n_xi x n_xi arrays) for the multi-index set mi (n_xi x m)."""
    n, m = mi.shape
    dmax = int(mi.max()) if mi.size else 0
    T, X = triple_1d(dmax + 1)
    G = [np.eye(n)]
    for l in range(m):
        Gl = np.zeros((n, n))
        for r in range(n):
            for s in range(n):
                v = X[mi[r, l], mi[s, l]]
                for k in range(m):
                    if k != l and mi[r, k] != mi[s, k]:
                        v = 0.0
                Gl[r, s] = v
        G.append(Gl)
    return G


def h_matrices(mi):
    """H_1..H_{n_xi} as an array H[l, r, s] = <psi_l psi_r psi_s> (l indexes psi from 0)."""
    n, m = mi.shape
    dmax = int(mi.max()) if mi.size else 0
    T, X = triple_1d(dmax)
    H = np.ones((n, n, n))
    for k in range(m):
        H *= T[np.ix_(mi[:, k], mi[:, k], mi[:, k])]
    return H
