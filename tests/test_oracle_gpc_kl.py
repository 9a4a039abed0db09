"""Pins of the gPC matrices (Section 3.2) and the KL viscosity model (Section 5.1)."""
import numpy as np
import pytest
from numpy.polynomial import legendre as L
from scipy.optimize import brentq

import synth
from oracle import gpc


def _triple_exact(a, b, c):
    """<p_a p_b p_c> by exact Legendre-series multiplication (no quadrature):
    E[f(xi)] = 1/2 int_{-1}^{1} f(sqrt3 t) dt and p_n(sqrt3 t) = sqrt(2n+1) P_n(t)."""
    ea = np.zeros(a + 1); ea[a] = 1
    eb = np.zeros(b + 1); eb[b] = 1
    ec = np.zeros(c + 1); ec[c] = 1
    prod = L.legmul(L.legmul(ea, eb), ec)
    return np.sqrt((2 * a + 1) * (2 * b + 1) * (2 * c + 1)) * prod[0]


def test_triple_products_match_exact_algebra():
    T, X = gpc.triple_1d(4)
    for a in range(5):
        for b in range(5):
            for c in range(5):
                assert abs(T[a, b, c] - _triple_exact(a, b, c)) < 1e-13


def test_xi_closed_form():
    """<xi p_n p_{n+1}> = sqrt3 (n+1) / sqrt((2n+1)(2n+3)), zero unless |n - n'| = 1."""
    T, X = gpc.triple_1d(6)
    for n in range(6):
        assert abs(X[n, n + 1] - np.sqrt(3) * (n + 1) / np.sqrt((2 * n + 1) * (2 * n + 3))) < 1e-13
        for k in range(7):
            if abs(k - n) != 1:
                assert abs(X[n, k]) < 1e-13


@pytest.mark.parametrize("m,d", [(1, 2), (2, 2), (3, 3), (5, 3)])
def test_g_h_structure(m, d):
    """G_0 = H_1 = I (Section 5.2); symmetry; H_{1+l} = G_l since psi_{1+l} = xi_l."""
    mi = synth.gpc_multi_indices(m, d)
    assert mi.shape[0] == synth.n_xi(m, d)
    assert np.all(mi[0] == 0)
    assert np.array_equal(mi[1:m + 1], np.eye(m, dtype=int))
    G = gpc.g_matrices(mi)
    H = gpc.h_matrices(mi)
    n = mi.shape[0]
    assert np.array_equal(G[0], np.eye(n))
    assert np.abs(H[0] - np.eye(n)).max() < 1e-13
    for l in range(1, m + 1):
        assert np.abs(G[l] - G[l].T).max() < 1e-15
        assert np.abs(H[l] - G[l]).max() < 1e-13
    assert np.abs(H - H.transpose(1, 0, 2)).max() < 1e-13
    assert np.abs(H - H.transpose(0, 2, 1)).max() < 1e-13
    # orthonormality <psi_r psi_s> = delta_rs: column of H for the constant mode
    assert np.abs(H[:, :, 0] - np.eye(n)).max() < 1e-13


def _kl1d(a, b, count):
    """Analytic eigenvalues of exp(-|x-y|/b) on [-a, a] (Ghanem-Spanos form):
    lambda = 2c / (w^2 + c^2), c = 1/b, w from c - w tan(wa) = 0 or w + c tan(wa) = 0."""
    c = 1.0 / b
    out = []
    for k in range(count):
        lo, hi = (k * np.pi) / a + 1e-12, ((k + 0.5) * np.pi) / a - 1e-12
        w = brentq(lambda w: c - w * np.tan(w * a), lo, hi)
        out.append(2 * c / (w * w + c * c))
        lo, hi = ((k + 0.5) * np.pi) / a + 1e-12, ((k + 1) * np.pi) / a - 1e-12
        w = brentq(lambda w: w + c * np.tan(w * a), lo, hi)
        out.append(2 * c / (w * w + c * c))
    return np.sort(out)[::-1]


def test_kl_separable_rectangle_matches_analytic():
    """On [0,2] x [-1,1] the L1 exponential kernel is a product of 1-D kernels, so
    the eigenvalues are products of the analytic 1-D eigenvalues."""
    mesh = synth.channel_mesh(0.125, 2.0)
    b = 1.0
    beta, A, M = synth.kl_eigenpairs(mesh.pxy, mesh.elem_q1, mesh.h, b, 6)
    l1 = _kl1d(1.0, b, 4)
    prods = np.sort(np.outer(l1, l1).ravel())[::-1][:6]
    assert np.allclose(beta, prods, rtol=5e-3)
    # M-orthonormal modes (L2-normalised)
    assert np.abs(A.T @ M @ A - np.eye(6)).max() < 1e-10


def test_kl_trace_converges_to_area():
    """The sum of all Galerkin eigenvalues approaches int c(x, x) dx = |D| = 4 from
    below (a Galerkin projection of a positive operator), with an O(h) gap."""
    gaps = []
    for h in (0.5, 0.25, 0.125):
        mesh = synth.channel_mesh(h, 2.0)
        beta, A, M = synth.kl_eigenpairs(mesh.pxy, mesh.elem_q1, mesh.h, 1.0, mesh.n_pnodes)
        gaps.append(4.0 - beta.sum())
    assert all(g > 0 for g in gaps)
    assert 1.6 < gaps[0] / gaps[1] < 2.4 and 1.6 < gaps[1] / gaps[2] < 2.4


def test_viscosity_fields_positive_and_scaled():
    p = synth.preset("small")
    nu = p.nu
    assert nu.shape == (3, p.n_p)
    assert np.all(nu[0] == 1 / 50)
    assert np.all(nu[0] - np.sqrt(3) * np.abs(nu[1:]).sum(0) > 0)
