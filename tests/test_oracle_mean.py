"""Pins of the mean-based pieces of the preconditioner (Section 5.2, eq. 11_prec)
against definitions read off the full tensors, independent of the Kronecker
grouping the oracle uses:

* N_0 is block diagonal in time with I_{n_xi} (x) N(w_{h,1}^k) as block k, where
  w_{h,1}^k is the psi_1 (mean) mode of the convection field at time step k;
* w_avg of eq. (11_prec) is the average of those mean modes over the time steps;
* K = tau^-1 M + A_0 + N(w_avg) is the time average of the spatial blocks of
  F_0^k, because N(w) is linear in w;
* the convection field is the full velocity E u + u_D, whose Dirichlet values are
  the inflow (1 - 4 x2^2) times the time ramp in the mean mode (Section 5.1).
"""
import numpy as np
import pytest

import synth
from oracle.solver import mean_oseen_matrix, mean_velocity_field
from oracle.system import Discretisation
from oracle.tt import TT


@pytest.fixture(scope="module")
def tiny():
    return Discretisation(synth.preset("tiny"))


def _conv_field(d, seed, r1=2, r2=3):
    return TT(*synth.random_tt(d.n_t, d.n_xi, 2 * d.n_nodes, r1, r2, seed=seed))


def test_mean_convection_is_block_diagonal_in_the_mean_mode(tiny):
    """N_0(w) z: at time step k every gPC mode of z is multiplied by the bold N of
    the mean mode W[k, 0] of the full convection tensor (Section 5.2)."""
    d = tiny
    w = _conv_field(d, 21)
    z = TT(*synth.random_tt(d.n_t, d.n_xi, d.n_u, 2, 3, seed=22))
    got = d.conv_apply(w, z, mean=True).full()
    W, Z = w.full(), z.full()
    ref = np.zeros_like(Z)
    for k in range(d.n_t):
        Nk = d.conv_matrix(W[k, 0], "f", "f")
        for s in range(d.n_xi):
            ref[k, s] = Nk @ Z[k, s]
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    # the same product with another mode's field differs: the test sees the mode index
    wrong = np.zeros_like(Z)
    for k in range(d.n_t):
        Nk = d.conv_matrix(W[k, 1], "f", "f")
        for s in range(d.n_xi):
            wrong[k, s] = Nk @ Z[k, s]
    assert np.abs(got - wrong).max() > 1e-3 * np.abs(ref).max()


def test_mean_convection_equals_full_convection_for_a_deterministic_field(tiny):
    """With a convection field whose only nonzero gPC mode is psi_1, N(w) and N_0(w)
    coincide (H_1 = I, Section 5.2)."""
    d = tiny
    z1, z2, z3 = synth.random_tt(d.n_t, d.n_xi, 2 * d.n_nodes, 2, 3, seed=23)
    z2 = z2.copy()
    z2[:, 1:, :] = 0.0
    w = TT(z1, z2, z3)
    z = TT(*synth.random_tt(d.n_t, d.n_xi, d.n_u, 2, 2, seed=24))
    a = d.conv_apply(w, z, mean=True).full()
    b = d.conv_apply(w, z, mean=False).full()
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_mean_velocity_field_is_the_time_average_of_the_mean_mode(tiny):
    d = tiny
    w = _conv_field(d, 25)
    ref = w.full()[:, 0, :].mean(axis=0)
    got = mean_velocity_field(w)
    assert got.shape == (2 * d.n_nodes,)
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_mean_oseen_matrix_is_the_time_average_of_the_mean_blocks(tiny):
    """K x = (1/n_t) sum_k [(F_0 + C)(e_k (x) e_1 (x) x)] at time k, mode 1, for the
    x1-component: the shift term lands on step k+1, so block k is F_0^k alone."""
    d = tiny
    w = _conv_field(d, 26)
    K = mean_oseen_matrix(d, w)
    x = np.random.default_rng(27).standard_normal(d.n_v)
    e0 = np.zeros(d.n_xi); e0[0] = 1.0
    acc = np.zeros(d.n_v)
    for k in range(d.n_t):
        ek = np.zeros(d.n_t); ek[k] = 1.0
        z = TT.rank1(ek, e0, np.concatenate([x, np.zeros(d.n_v)]))
        out = d.apply_mean(w, z).full()
        acc += out[k, 0, :d.n_v]
        # the x2-component of a pure x1 input stays zero (bold blocks are diagonal)
        assert np.abs(out[k, 0, d.n_v:]).max() < 1e-12 * np.abs(out[k, 0, :d.n_v]).max()
    ref = acc / d.n_t
    got = K @ x
    assert np.abs(got - ref).max() < 1e-11 * np.abs(ref).max()
    # a convection-free K differs (the averaged convection is really in it)
    K0 = mean_oseen_matrix(d, None)
    assert np.abs(K0 @ x - ref).max() > 1e-6 * np.abs(ref).max()


def test_full_velocity_carries_the_inflow_lifting(tiny):
    """w = E u + u_D: free rows hold u, Dirichlet rows hold (1 - 4 x2^2)(1 - e^{-10 t_k})
    at the inlet x1 = -1 in the mean mode, and zero on the walls and other modes."""
    d = tiny
    prob = d.prob
    u = TT(*synth.random_tt(d.n_t, d.n_xi, d.n_u, 2, 3, seed=28))
    W = d.full_velocity(u).full()
    U = u.full()
    n, f, D = d.n_nodes, d.free, d.dn
    assert np.abs(W[:, :, f] - U[:, :, :d.n_v]).max() < 1e-13
    assert np.abs(W[:, :, f + n] - U[:, :, d.n_v:]).max() < 1e-13
    xy = prob.mesh.xy[D]
    t = prob.tau * np.arange(1, d.n_t + 1)
    ramp = 1.0 - np.exp(-10.0 * t)
    inlet = np.isclose(xy[:, 0], xy[:, 0].min()) & (np.abs(xy[:, 1]) < 0.5)
    prof = np.where(inlet, 1.0 - 4.0 * xy[:, 1] ** 2, 0.0)
    assert np.abs(W[:, 0, D] - ramp[:, None] * prof[None, :]).max() < 1e-13
    assert np.abs(W[:, 1:, D]).max() == 0.0
    assert np.abs(W[:, :, D + n]).max() == 0.0
    assert inlet.sum() > 0 and np.abs(prof).max() > 0.5
