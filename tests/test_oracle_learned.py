"""Pins of the learned mean-Oseen solve's CPU reference (oracle/learned.py):
convolution against scipy's correlation, gradients against central finite
differences, Adam's first step against its closed form, lattice layout against
the mesh, and training targets against the exact solve."""
import numpy as np
import pytest
import scipy.signal

import synth
from synth.lattice import node_lattice, scatter_nodes, gather_nodes, gaussian_residuals
from oracle import learned as L
from oracle.system import Discretisation
from oracle.solver import mean_oseen_matrix


@pytest.fixture(scope="module")
def tiny():
    prob = synth.preset("tiny")
    d = Discretisation(prob)
    return prob, d, node_lattice(prob.mesh)


def _lifting_field(d):
    """Full-node convection train of the lifting alone (u = 0)."""
    from oracle.tt import TT
    return d.full_velocity(TT.zeros(d.n_t, d.n_xi, d.n_u))


def test_conv3x3_matches_scipy_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 7, 5))
    W = rng.standard_normal((2, 3, 3, 3))
    b = rng.standard_normal(2)
    y = L.conv3x3(x, W, b)
    for o in range(2):
        want = b[o] + sum(scipy.signal.correlate2d(x[c], W[o, c], mode="same", boundary="fill")
                          for c in range(3))
        assert np.allclose(y[o], want, rtol=0, atol=1e-12)


def _tiny_net(seed=1, c_in=3, ch=3, depth=3):
    params = L.init_params(channels=ch, seed=seed, c_in=c_in, c_out=2, depth=depth)
    rng = np.random.default_rng(seed + 10)
    # biases nonzero so that every ReLU sees both signs
    return [(W, rng.standard_normal(b.shape) * 0.1) for W, b in params]


def test_network_gradients_match_central_differences():
    params = _tiny_net()
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 5, 4))
    gy = rng.standard_normal((2, 5, 4))
    f = lambda ps, xx: float(np.sum(gy * L.net_forward(ps, xx)[0]))
    _, cache = L.net_forward(params, x)
    grads, gx = L.net_backward(params, cache, gy)
    h = 1e-6
    for k in range(len(params)):
        W, b = params[k]
        for idx in [tuple(rng.integers(0, s) for s in W.shape) for _ in range(4)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h
            Wm[idx] -= h
            pp = list(params); pp[k] = (Wp, b)
            pm = list(params); pm[k] = (Wm, b)
            fd = (f(pp, x) - f(pm, x)) / (2 * h)
            assert abs(fd - grads[k][0][idx]) <= 1e-6 * max(1.0, abs(fd))
        j = int(rng.integers(0, b.size))
        bp, bm = b.copy(), b.copy()
        bp[j] += h
        bm[j] -= h
        pp = list(params); pp[k] = (W, bp)
        pm = list(params); pm[k] = (W, bm)
        fd = (f(pp, x) - f(pm, x)) / (2 * h)
        assert abs(fd - grads[k][1][j]) <= 1e-6 * max(1.0, abs(fd))
    for _ in range(4):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (f(params, xp) - f(params, xm)) / (2 * h)
        assert abs(fd - gx[idx]) <= 1e-6 * max(1.0, abs(fd))


def test_lattice_layout_matches_the_mesh(tiny):
    prob, d, lat = tiny
    mesh = prob.mesh
    assert lat.mask.sum() == mesh.n_nodes
    v = np.arange(mesh.n_nodes, dtype=float) + 1.0
    assert np.array_equal(gather_nodes(lat, scatter_nodes(lat, v)), v)
    # Q2 local node a + 3b of every element sits at lattice offset (a, b) from node 0
    for e in mesh.elem_q2:
        i0, j0 = lat.ix[e[0]], lat.iy[e[0]]
        for b in range(3):
            for a in range(3):
                assert (lat.ix[e[a + 3 * b]] - i0, lat.iy[e[a + 3 * b]] - j0) == (a, b)


def test_read_free_and_scatter_free_are_adjoint(tiny):
    prob, d, lat = tiny
    rng = np.random.default_rng(3)
    y = rng.standard_normal((2, lat.ny, lat.nx))
    g = rng.standard_normal(2 * lat.free.size)
    assert np.isclose(L.read_free(lat, y, 1.0) @ g, np.sum(y * L.scatter_free(lat, g)), rtol=1e-13)


def test_learned_solve_is_positively_homogeneous(tiny):
    prob, d, lat = tiny
    params = L.init_params(channels=4, seed=4)
    r = gaussian_residuals(d.n_v, 1, seed=5)[0]
    wavg = np.zeros(2 * d.n_nodes)
    a = L.apply_net(params, lat, r, wavg, d.n_nodes)
    assert np.allclose(L.apply_net(params, lat, 3.0 * r, wavg, d.n_nodes), 3.0 * a, rtol=1e-12, atol=0)


def test_training_targets_solve_the_mean_oseen_system(tiny):
    prob, d, lat = tiny
    w = _lifting_field(d)
    R, T = L.training_pairs(d, w, gaussian_residuals(d.n_v, 3, seed=6), smooth_sweeps=2)
    K = mean_oseen_matrix(d, w)
    nv = d.n_v
    for r, t in zip(R, T):
        for c in range(2):
            res = K @ t[c * nv:(c + 1) * nv] - r[c * nv:(c + 1) * nv]
            assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(r[c * nv:(c + 1) * nv])


def test_loss_gradient_matches_central_difference(tiny):
    prob, d, lat = tiny
    params = L.init_params(channels=4, seed=7)
    params = [(W, np.full(b.shape, 0.05)) for W, b in params]
    R, T = L.training_pairs(d, _lifting_field(d), gaussian_residuals(d.n_v, 2, seed=8))
    wavg = np.zeros(2 * d.n_nodes)
    _, grads = L.loss_and_grads(params, lat, wavg, d.n_nodes, R, T)
    rng = np.random.default_rng(9)
    h = 1e-6
    for k in (0, 3):
        W, b = params[k]
        idx = tuple(rng.integers(0, s) for s in W.shape)
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += h
        Wm[idx] -= h
        pp = list(params); pp[k] = (Wp, b)
        pm = list(params); pm[k] = (Wm, b)
        fp, _ = L.loss_and_grads(pp, lat, wavg, d.n_nodes, R, T)
        fm, _ = L.loss_and_grads(pm, lat, wavg, d.n_nodes, R, T)
        fd = (fp - fm) / (2 * h)
        assert abs(fd - grads[k][0][idx]) <= 1e-6 * max(1.0, abs(fd))


def test_adam_first_step_closed_form():
    # with zero moments, the first bias-corrected step is lr * g / (|g| + eps)
    rng = np.random.default_rng(10)
    params = [(rng.standard_normal((2, 3, 3, 3)), rng.standard_normal(2))]
    grads = [(rng.standard_normal((2, 3, 3, 3)), rng.standard_normal(2))]
    opt = L.Adam(params, lr=1e-2)
    new = opt.step(params, grads)
    for (W, b), (gW, gb), (nW, nb) in zip(params, grads, new):
        assert np.allclose(nW, W - 1e-2 * gW / (np.abs(gW) + 1e-8), rtol=0, atol=1e-15)
        assert np.allclose(nb, b - 1e-2 * gb / (np.abs(gb) + 1e-8), rtol=0, atol=1e-15)


def test_short_training_reduces_the_loss(tiny):
    prob, d, lat = tiny
    params = L.init_params(channels=8, seed=11)
    R, T = L.training_pairs(d, _lifting_field(d), gaussian_residuals(d.n_v, 6, seed=12), smooth_sweeps=1)
    wavg = np.zeros(2 * d.n_nodes)
    opt = L.Adam(params, lr=3e-3)
    first, _ = L.loss_and_grads(params, lat, wavg, d.n_nodes, R, T)
    for _ in range(25):
        loss, g = L.loss_and_grads(params, lat, wavg, d.n_nodes, R, T)
        params = opt.step(params, g)
    last, _ = L.loss_and_grads(params, lat, wavg, d.n_nodes, R, T)
    assert last < 0.7 * first


def test_learned_minv_keeps_the_train_structure(tiny):
    prob, d, lat = tiny
    params = L.init_params(channels=4, seed=13)
    rng = np.random.default_rng(14)
    z1, z2, z3 = synth.random_tt(d.n_t, d.n_xi, d.n_u, 2, 3, seed=15)
    from oracle.tt import TT
    z = TT(z1, z2, z3)
    out = L.LearnedMinv(params, d, lat, None)(z)
    assert out.ranks == z.ranks
    assert np.allclose(out.z1, np.cumsum(z1, axis=0))
    assert np.allclose(out.z3[1], L.apply_net(params, lat, z3[1], np.zeros(2 * d.n_nodes), d.n_nodes))


def test_inner_solve_falls_back_to_the_exact_preconditioner(tiny):
    """An untrained net in place of K^{-1}: every inner solve that misses its
    tolerance is redone with the exact M^{-1}, so the outer solve is unchanged."""
    from oracle.solver import MeanLSC, gmres, _Pair
    prob, d, lat = tiny
    t = prob.tol
    f = d.rhs()
    exact = MeanLSC(d, None, t.eps_gmres, t.tol_inner, t.maxit_inner)
    (ue, pe), ste = gmres(lambda v: d.apply(None, *v), exact, f, tol=t.tol_gmres, eps=t.eps_gmres,
                          maxit=t.maxit_gmres, space=_Pair)
    params = L.init_params(channels=4, seed=16)
    lp = MeanLSC(d, None, t.eps_gmres, t.tol_inner, 3, learned_minv=L.LearnedMinv(params, d, lat, None))
    lp.maxit_inner = 3
    (ul, pl), stl = gmres(lambda v: d.apply(None, *v), lp, f, tol=t.tol_gmres, eps=t.eps_gmres,
                          maxit=t.maxit_gmres, space=_Pair)
    assert lp.fallbacks >= 1
    assert stl["res"][-1] <= t.tol_gmres * stl["bnorm"]
