"""Pins of the pressure-space pieces of the mean-based PCD preconditioner
(Section 5.2, eq. mean_pcd) in the oracle.

Matrix pins are closed-form integrals of polynomials that the Q1 space and the 3 x 3
Gauss rule reproduce exactly; the preconditioner is pinned by what it is for: the
Schur complement S_0 = B (F_0 + C)^-1 B^T of a small mean problem, preconditioned by
-S_PCD,0^-1, has its spectrum in a bounded cluster away from zero on two meshes and
GMRES on it converges in a few iterations, and a planted sign error in the time
coupling C_p slows that GMRES down.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import fem
from oracle.system import Discretisation
from oracle.tt import TT


@pytest.fixture(scope="module")
def step():
    return synth.step_mesh(0.25, 5.0)


def test_pressure_stiffness_closed_forms(step):
    """A_p c = 0 for constants; p^T A_p p = integral of nu |grad p|^2 for linear p (nu
    bilinear: the Q1 mass-weighted sum of its nodal values); symmetric; one element of
    side h with nu = 1 gives the textbook bilinear stiffness [4 -1 -1 -2; ...] / 6."""
    rng = np.random.default_rng(3)
    nu = 0.5 + rng.random(step.n_pnodes)
    Ap = fem.pressure_stiffness(step, nu)
    Mp = fem.pressure_mass(step)
    one = np.ones(step.n_pnodes)
    assert np.abs(Ap @ one).max() < 1e-12
    x, y = step.pxy[:, 0], step.pxy[:, 1]
    assert abs(x @ Ap @ x - one @ Mp @ nu) < 1e-11
    assert abs(y @ Ap @ y - one @ Mp @ nu) < 1e-11
    assert abs(x @ Ap @ y) < 1e-11
    assert abs(Ap - Ap.T).max() < 1e-14
    # one element: vertices (0,0), (1,0), (0,1), (1,1) in the a + 2b order
    e = fem.pressure_stiffness(step, np.ones(step.n_pnodes))
    pn = step.elem_q1[0]
    # the element's own contribution: assemble a single-element mesh by hand
    want = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    phi, ds, dt, chi, w = fem.reference_tables()
    chi2, cs, ct = fem._pressure_tables()
    got = np.einsum("q,qi,qj->ij", w, cs, cs) + np.einsum("q,qi,qj->ij", w, ct, ct)
    assert np.abs(got - want).max() < 1e-14
    assert np.abs(chi2 - chi).max() == 0.0
    assert e.shape == (step.n_pnodes, step.n_pnodes) and pn.size == 4


def test_pressure_convection_of_polynomials(step):
    """N_p(w) p = M_p g when w . grad p = g is bilinear: w = (c1, c2) constant and p = x1
    give g = c1; the rotation w = (x2, -x1) (a Q2 field) and p = x1 give g = x2;
    w = (1, 1) and p = x1 x2 give g = x1 + x2."""
    Mp = fem.pressure_mass(step)
    xv, yv = step.xy[:, 0], step.xy[:, 1]
    x, y = step.pxy[:, 0], step.pxy[:, 1]
    one = np.ones(step.n_pnodes)
    N = fem.pressure_convection(step, 0.7 * np.ones_like(xv), -0.3 * np.ones_like(xv))
    assert np.abs(N @ x - 0.7 * (Mp @ one)).max() < 1e-13
    assert np.abs(N @ y + 0.3 * (Mp @ one)).max() < 1e-13
    assert np.abs(N @ one).max() < 1e-13
    N = fem.pressure_convection(step, yv, -xv)
    assert np.abs(N @ x - Mp @ y).max() < 1e-13
    N = fem.pressure_convection(step, np.ones_like(xv), np.ones_like(xv))
    assert np.abs(N @ (x * y) - Mp @ (x + y)).max() < 1e-13


def _small_mean_problem(h, n_t=3, tau=0.2):
    prob = synth.preset("tiny", h=h, L=2.0, m=1, d=1, n_t=n_t, tau=tau)
    d = Discretisation(prob)
    # a rank-one convection field: the Poiseuille-like inflow profile at every node,
    # constant in time and deterministic
    xy = prob.mesh.xy
    wx = np.clip(1.0 - xy[:, 1] ** 2, 0.0, None)
    w3 = np.concatenate([wx, np.zeros_like(wx)])[None, :]
    e0 = np.zeros((1, d.n_xi, 1)); e0[0, 0, 0] = 1.0
    w = TT(np.ones((d.n_t, 1)), e0, w3)
    return d, w


def _dense_op(apply, n_t, n_xi, n):
    """Columns of a linear map on full tensors (n_t, n_xi, n) given as a TT map."""
    cols = []
    for k in range(n_t * n_xi * n):
        e = np.zeros(n_t * n_xi * n); e[k] = 1.0
        E = e.reshape(n_t, n_xi, n)
        t, x, i = np.unravel_index(k, (n_t, n_xi, n))
        z = TT(np.eye(n_t)[:, [t]], np.eye(n_xi)[None, :, [x]].reshape(1, n_xi, 1), np.eye(n)[[i], :])
        cols.append(apply(z).full().reshape(-1))
        del E
    return np.array(cols).T


def _pcd_preconditioned(d, w, flip_cp=False):
    """-S_PCD,0^-1 S_0 as a dense matrix for the mean problem with field w."""
    from oracle.solver import MeanPCD
    n_t, n_xi, n_p = d.n_t, d.n_xi, d.n_p
    # S_0 = B (F_0 + C)^-1 B^T on full vectors
    F = _dense_op(lambda z: d.apply_mean(w, z), n_t, n_xi, d.n_u)
    Bb = sp.kron(sp.identity(n_t * n_xi), d.B).toarray()
    S0 = Bb @ np.linalg.solve(F, Bb.T)
    P = MeanPCD(d, w, eps=0.0, tol_inner=1e-8, maxit_inner=10)
    if flip_cp:
        orig = d.apply_mean_p
        Mp, _, _ = d.pressure_matrices()
        from oracle.tt import add, kron_apply
        d.apply_mean_p = lambda ww, p: add((1.0, orig(ww, p)),
                                           (2.0 / d.tau, kron_apply(d.C, None, Mp, p)))
    try:
        Sinv = _dense_op(lambda z: P.schur(z).scale(-1.0), n_t, n_xi, n_p)
    finally:
        if flip_cp:
            del d.apply_mean_p
    return Sinv @ S0


def _gmres_its(A, tol=1e-8):
    """Unrestarted GMRES iterations for A x = b, b a fixed random vector."""
    b = np.random.default_rng(1).standard_normal(A.shape[0])
    its = [0]
    def cb(_):
        its[0] += 1
    spla.gmres(A, b, rtol=tol, restart=A.shape[0], maxiter=1, callback=cb, callback_type="pr_norm")
    return its[0]


def test_pcd_clusters_the_mean_schur_complement():
    """The preconditioned mean Schur complement has its spectrum in a bounded cluster
    away from zero (its eigenvalues are those of the time-diagonal blocks), and GMRES on
    it needs the same number of iterations on two meshes (h = 1/2, 1/4)."""
    its = []
    for h in (0.5, 0.25):
        d, w = _small_mean_problem(h)
        A = _pcd_preconditioned(d, w)
        ev = np.linalg.eigvals(A)
        assert ev.real.min() > 0.1 and np.abs(ev).max() < 10.0
        its.append(_gmres_its(A))
    assert max(its) <= 40 and abs(its[0] - its[1]) <= 3


def test_a_sign_error_in_the_time_coupling_slows_gmres():
    """C_p enters only the blocks below the time diagonal, so it leaves the spectrum
    alone; with its sign flipped the preconditioner no longer matches the causal
    coupling of S_0, and over 6 time steps of tau = 0.05 GMRES needs clearly more
    iterations (measured 29 against 44)."""
    d, w = _small_mean_problem(0.5, n_t=6, tau=0.05)
    good = _gmres_its(_pcd_preconditioned(d, w))
    bad = _gmres_its(_pcd_preconditioned(d, w, flip_cp=True))
    assert bad >= good + 8


def test_pcd_needs_more_gmres_iterations_than_lsc():
    """Fig. 5.4: with the PCD approximation the Picard steps need more GMRES iterations
    than with LSC (tiny problem at tight truncation tolerances)."""
    from oracle.solver import picard
    prob = synth.preset("tiny")
    prob.tol.eps_gmres, prob.tol.eps_soln, prob.tol.eps_conv = 1e-8, 1e-10, 1e-8
    d = Discretisation(prob)
    _, _, lsc = picard(d, schur="lsc")
    _, _, pcd = picard(d, schur="pcd")
    assert sum(pcd["gmres_its"]) > sum(lsc["gmres_its"])
    assert pcd["picard_its"] >= lsc["picard_its"]
