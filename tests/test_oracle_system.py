"""Pins of the all-at-once operator, its Picard solution and the preconditioner
wiring against definitions written independently of the Kronecker form."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import fem
from oracle.system import Discretisation
from oracle.solver import direct_picard, gmres, _Pair, picard
from oracle.tt import TT, tt_svd


@pytest.fixture(scope="module")
def tiny():
    return Discretisation(synth.preset("tiny"))


def _rand_pair(d, seed):
    u = TT(*synth.random_tt(d.n_t, d.n_xi, d.n_u, 2, 3, seed=seed))
    p = TT(*synth.random_tt(d.n_t, d.n_xi, d.n_p, 2, 2, seed=seed + 1))
    return u, p


def test_kron_operator_matches_per_timestep_definition(tiny):
    """L(w)[u;p] assembled from eq. (N_kron) equals the block matrix built per time
    step from eq. (F^k): sum_l H_l (x) N(w_l^k) with w_l^k read from the full tensor."""
    d = tiny
    u, p = _rand_pair(d, 0)
    w = TT(*synth.random_tt(d.n_t, d.n_xi, 2 * d.n_nodes, 2, 3, seed=5))
    uo, po = d.apply(w, u, p)
    K, _ = d.full_matrix(w.vec())
    ref = K @ np.concatenate([u.vec(), p.vec()])
    n = u.vec().size
    assert np.abs(uo.vec() - ref[:n]).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(po.vec() - ref[n:]).max() < 1e-12 * np.abs(ref).max()


def test_residual_matches_definition(tiny):
    """r = f - A(w)[u;p] with w = E u + u_D, checked against the uncompressed system
    whose right-hand side carries the Dirichlet couplings of every block."""
    d = tiny
    u, p = _rand_pair(d, 3)
    (ru, rp), rn = d.residual(u, p, 0.0)
    w = d.full_velocity(u)
    K, NfD = d.full_matrix(w.vec())
    fu, fp = d.rhs()
    rhs = np.concatenate([fu.vec() - NfD @ d.uD.vec(), fp.vec()])
    ref = rhs - K @ np.concatenate([u.vec(), p.vec()])
    got = np.concatenate([ru.vec(), rp.vec()])
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()
    assert abs(rn - np.linalg.norm(ref)) < 1e-10 * rn


def _sequential_backward_euler(prob, tol=1e-13):
    """sigma = 0: plain backward-Euler time stepping of the deterministic problem,
    Dirichlet rows replaced by the boundary values (no lifting, no Kronecker form)."""
    mesh = prob.mesh
    n, D = mesh.n_nodes, mesh.dnodes
    M = fem.mass(mesh)
    A = fem.stiffness(mesh, prob.nu[0])
    Bx, By = fem.divergence(mesh)
    np_ = mesh.n_pnodes
    tau = prob.tau
    Bfull = sp.hstack([Bx, By])
    U = np.zeros(2 * n)
    dmask = np.concatenate([mesh.dirichlet, mesh.dirichlet])
    out = []
    for k in range(prob.n_t):
        g = np.concatenate([mesh.inflow, np.zeros(n)]) * prob.tprofile[k]
        Uk = U.copy(); Uk[dmask] = g[dmask]
        for _ in range(200):
            N = fem.convection(mesh, Uk[:n], Uk[n:])
            F = sp.block_diag([M / tau + A + N, M / tau + A + N]).tolil()
            rhs = np.concatenate([sp.block_diag([M, M]) @ U / tau, np.zeros(np_)])
            K = sp.bmat([[F, Bfull.T], [Bfull, None]]).tolil()
            for i in np.flatnonzero(dmask):
                K.rows[i] = [i]; K.data[i] = [1.0]; rhs[i] = g[i]
            sol = spla.spsolve(K.tocsc(), rhs)
            diff = np.linalg.norm(sol[:2 * n] - Uk)
            Uk = sol[:2 * n]
            if diff <= tol * max(1.0, np.linalg.norm(Uk)):
                break
        U = Uk
        out.append((U.copy(), sol[2 * n:].copy()))
    return out


def test_sigma_zero_reduces_to_backward_euler():
    """sigma = 0: only the psi_1 mode is nonzero and it is backward-Euler time
    stepping of the deterministic problem (the time coupling C is a lower shift)."""
    prob = synth.preset("tiny", sigma=0.0)
    d = Discretisation(prob)
    uf, pf, _ = direct_picard(d, tol=1e-13)
    seq = _sequential_backward_euler(prob)
    f, n = d.free, d.n_nodes
    for k, (U, P) in enumerate(seq):
        assert np.abs(uf[k, 0] - np.concatenate([U[f], U[f + n]])).max() < 1e-9
        assert np.abs(pf[k, 0] - P).max() < 1e-8
    assert np.abs(uf[:, 1:]).max() < 1e-12 and np.abs(pf[:, 1:]).max() < 1e-12


def test_discrete_incompressibility(tiny):
    """B u = 0 for the full velocity of every time step and gPC mode."""
    uf, pf, _ = direct_picard(tiny, tol=1e-13)
    n, f, D = tiny.n_nodes, tiny.free, tiny.dn
    W = np.zeros((tiny.n_t, tiny.n_xi, 2 * n))
    W[:, :, f] = uf[:, :, :f.size]; W[:, :, f + n] = uf[:, :, f.size:]
    lift = tiny.full_velocity(TT.zeros(tiny.n_t, tiny.n_xi, tiny.n_u)).full()
    W = W + lift
    B = sp.hstack([tiny.Bxfull, tiny.Byfull])
    div = np.einsum("pj,tsj->tsp", B.toarray(), W)
    assert np.abs(div).max() < 1e-12


def test_commutator_identity_with_time_coupling(tiny):
    """eq. (stoch_commu_2): M_p^-1 B M^-1 C - M_p^-1 C_p M_p^-1 B = 0 exactly."""
    d = tiny
    Mp = fem.pressure_mass(d.prob.mesh)
    It, Ix = sp.identity(d.n_t), sp.identity(d.n_xi)
    bB = sp.kron(sp.kron(It, Ix), d.B)
    bM = sp.kron(sp.kron(It, Ix), d.bM).tocsc()
    bMp = sp.kron(sp.kron(It, Ix), Mp).tocsc()
    bC = -sp.kron(sp.kron(d.C, Ix), d.bM) / d.tau
    bCp = -sp.kron(sp.kron(d.C, Ix), Mp) / d.tau
    X = np.random.default_rng(0).standard_normal((bB.shape[1], 3))
    lhs = spla.spsolve(bMp, bB @ spla.spsolve(bM, bC @ X))
    rhs = spla.spsolve(bMp, bCp @ spla.spsolve(bMp, bB @ X))
    assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(lhs).max()


def test_ideal_preconditioner_converges_in_two_iterations(tiny):
    """eq. (prec): with the exact block triangular P, right-preconditioned GMRES
    converges in two iterations (eigenvalue 1, Jordan blocks of order 2)."""
    d = tiny
    w = d.full_velocity(TT(*synth.random_tt(d.n_t, d.n_xi, d.n_u, 1, 2, seed=4)))
    K, _ = d.full_matrix(w.vec())
    K = K.toarray()
    n = d.n_t * d.n_xi * d.n_u
    F, Bt, B = K[:n, :n], K[:n, n:], K[n:, :n]
    S = B @ np.linalg.solve(F, Bt)
    P = np.block([[F, Bt], [np.zeros_like(B), -S]])

    def to_pair(x):
        return (tt_svd(x[:n].reshape(d.n_t, d.n_xi, d.n_u), 1e-15),
                tt_svd(x[n:].reshape(d.n_t, d.n_xi, d.n_p), 1e-15))

    def vec(v):
        return np.concatenate([v[0].vec(), v[1].vec()])

    b = to_pair(np.random.default_rng(1).standard_normal(K.shape[0]))
    z, st = gmres(lambda v: to_pair(K @ vec(v)), lambda v: to_pair(np.linalg.solve(P, vec(v))),
                  b, tol=1e-9, eps=1e-14, maxit=10, space=_Pair)
    assert st["its"] == 2
    assert np.linalg.norm(K @ vec(z) - vec(b)) < 1e-8 * np.linalg.norm(vec(b))


def test_lsc_is_exact_schur_inverse_on_its_own_terms(tiny):
    """The LSC factor chain of eq. (mean_lsc) equals the matrix product written out:
    L^-1 (B M*^-1 (F0 + C) M*^-1 B^T) L^-1 with L = B M*^-1 B^T."""
    from oracle.solver import MeanLSC
    d = tiny
    P = MeanLSC(d, None, 0.0, 1e-1, 10)
    ap = TT(*synth.random_tt(d.n_t, d.n_xi, d.n_p, 2, 2, seed=8))
    got = P.schur(ap).vec()
    It, Ix = sp.identity(d.n_t), sp.identity(d.n_xi)
    Mi = sp.diags(1 / d.Mstar_diag)
    L = (d.B @ Mi @ d.B.T).toarray()
    F0C = (sp.kron(sp.kron(It, Ix), d.bM / d.tau + d.bA[0]) - sp.kron(sp.kron(d.C, Ix), d.bM) / d.tau).toarray()
    bL = np.kron(np.eye(d.n_t * d.n_xi), L)
    bB = np.kron(np.eye(d.n_t * d.n_xi), d.B.toarray())
    bMi = np.kron(np.eye(d.n_t * d.n_xi), Mi.toarray())
    ref = -np.linalg.solve(bL, bB @ bMi @ F0C @ bMi @ bB.T @ np.linalg.solve(bL, ap.vec()))
    assert np.abs(got - ref).max() < 1e-10 * np.abs(ref).max()


def test_inner_preconditioner_solves_its_matrix(tiny):
    """M^{-1} of eq. (11_prec): (I - C)^{-1} is a cumulative sum in time."""
    from oracle.solver import MeanLSC
    d = tiny
    P = MeanLSC(d, None, 0.0, 1e-1, 10)
    z = TT(*synth.random_tt(d.n_t, d.n_xi, d.n_u, 2, 3, seed=9))
    y = P.apply_Minv(z).vec()
    It = np.eye(d.n_t)
    K = (d.bM / d.tau + d.bA[0]).toarray()
    Mfull = np.kron(np.kron(It - d.C.toarray(), np.eye(d.n_xi)), K)
    assert np.abs(Mfull @ y - z.vec()).max() < 1e-10 * np.abs(z.vec()).max()


@pytest.mark.parametrize("mean", [False, True])
def test_grouped_convection_equals_term_by_term_sum(tiny, mean):
    """conv_apply (blocks shared per diag(w1_a) and per N(w3_b)) is the same tensor
    as summing the Kronecker terms of eq. (N_kron) one at a time."""
    from oracle.tt import add
    d = tiny
    u, _ = _rand_pair(d, 11)
    w = TT(*synth.random_tt(d.n_t, d.n_xi, 2 * d.n_nodes, 2, 3, seed=12))
    grouped = d.conv_apply(w, u, mean=mean)
    literal = add(*[(1.0, t) for t in d.conv_terms(w, u, mean=mean)])
    assert grouped.ranks == (2 * u.ranks[0], 3 * u.ranks[1])
    assert np.abs(grouped.vec() - literal.vec()).max() < 1e-12 * np.abs(literal.vec()).max()


def test_batch_generator_is_seeded_and_within_ranges():
    import synth
    a = synth.batch("tiny", 4, seed=9, nu0_range=(1 / 200, 1 / 50), sigma_range=(0.05, 0.3))
    b = synth.batch("tiny", 4, seed=9, nu0_range=(1 / 200, 1 / 50), sigma_range=(0.05, 0.3))
    for x, y in zip(a, b):
        assert x.params["nu0"] == y.params["nu0"] and x.params["sigma"] == y.params["sigma"]
        assert 1 / 200 <= x.params["nu0"] <= 1 / 50 and 0.05 <= x.params["sigma"] <= 0.3
    assert len({x.params["nu0"] for x in a}) == 4
