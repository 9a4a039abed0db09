"""Pins of the mesh, the problem sizes and the oracle's Q2-Q1 assembly.

Every expected value here comes from the paper's printed sizes or from
closed-form integrals of polynomials that the Q2/Q1 spaces reproduce exactly.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from oracle import fem

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            out[k] = float(v)
    return out


def test_paper_problem_sizes():
    """Section 5.1: n_t=64, n_xi=20, n_u=2992, n_p=461, 4419840 unknowns."""
    g = _golden("paper_sizes.txt")
    t = _golden("table_5_1.txt")
    mesh = synth.step_mesh(t["h"], L=12.0)
    n_xi = synth.n_xi(int(t["m"]), int(t["d_psi"]))
    n_t = int(round(t["t_f"] / t["tau"]))
    assert (n_t, n_xi) == (g["n_t"], g["n_xi"])
    assert 2 * mesh.n_v == g["n_u"]
    assert mesh.n_pnodes == g["n_p"]
    assert n_t * n_xi * (2 * mesh.n_v + mesh.n_pnodes) == g["unknowns"]
    assert synth.gpc_multi_indices(3, 3).shape[0] == g["n_xi"]


def test_paper_storage_ratio():
    """Section 5.3: (n_t k1 + n_xi k1 k2 + n_u k2) / (n_t n_xi n_u) = 270748 / 3829760."""
    g = _golden("paper_sizes.txt")
    k1, k2 = g["kappa1"], g["kappa2"]
    tt = g["n_t"] * k1 + g["n_xi"] * k1 * k2 + g["n_u"] * k2
    assert tt == g["tt_storage"]
    assert g["n_t"] * g["n_xi"] * g["n_u"] == g["full_storage"]


@pytest.mark.parametrize("name,n_u,n_p,n_xi", [("small", 1312, 209, 6), ("medium", 5440, 769, 20)])
def test_preset_sizes(name, n_u, n_p, n_xi):
    """Workload sizes by exact node counting on the step with L=5."""
    h = {"small": 0.25, "medium": 0.125}[name]
    mesh = synth.step_mesh(h, 5.0)
    assert (2 * mesh.n_v, mesh.n_pnodes) == (n_u, n_p)
    assert synth.n_xi(*{"small": (2, 2), "medium": (3, 3)}[name]) == n_xi


def test_large_sizes():
    mesh = synth.step_mesh(0.0625, 5.0)
    assert (2 * mesh.n_v, mesh.n_pnodes) == (22144, 2945)
    assert synth.n_xi(5, 3) == 56


@pytest.fixture(scope="module")
def step():
    return synth.step_mesh(0.25, 5.0)


def test_mass_integrates_area(step):
    """1^T M 1 = |D| = 5*2 + 1*1 (main channel + inlet)."""
    M = fem.mass(step)
    one = np.ones(step.n_nodes)
    assert abs(one @ M @ one - 11.0) < 1e-12
    # M x . 1 = integral of x1 over the domain: main 5*2*2.5 + inlet 1*(-0.5)
    assert abs(one @ M @ step.xy[:, 0] - (25.0 - 0.5)) < 1e-12


def test_stiffness_kills_constants_and_integrates_gradients(step):
    """A c = 0 for constant c; x1^T A x1 = integral of nu; with a bilinear nu that
    is the Q1 mass-weighted sum of its nodal values."""
    rng = np.random.default_rng(0)
    nu = 0.5 + rng.random(step.n_pnodes)
    A = fem.stiffness(step, nu)
    assert np.abs(A @ np.ones(step.n_nodes)).max() < 1e-12
    x = step.xy[:, 0]
    Mp = fem.pressure_mass(step)
    assert abs(x @ A @ x - np.ones(step.n_pnodes) @ Mp @ nu) < 1e-11
    y = step.xy[:, 1]
    assert abs(x @ A @ y) < 1e-11            # grad x1 . grad x2 = 0
    assert abs((A - A.T)).max() < 1e-14


def test_divergence_of_linear_fields(step):
    """B_x1 x1 = -M_p 1 (div of (x1, 0) is 1); B_x1 x2 = 0; B_x2 x2 = -M_p 1."""
    Bx, By = fem.divergence(step)
    Mp = fem.pressure_mass(step)
    x, y = step.xy[:, 0], step.xy[:, 1]
    r = Mp @ np.ones(step.n_pnodes)
    assert np.abs(Bx @ x + r).max() < 1e-13
    assert np.abs(Bx @ y).max() < 1e-13
    assert np.abs(By @ y + r).max() < 1e-13
    # a divergence-free quadratic field (x2^2, x1^2) has zero discrete divergence
    assert np.abs(Bx @ (y ** 2) + By @ (x ** 2)).max() < 1e-13


def test_convection_of_polynomials(step):
    """N(w) v = M g when w . grad v = g lies in Q2 and the quadrature is exact:
    w=(x2,0), v=x1 gives g=x2; w=(0,x1), v=x2 gives g=x1; w=(1,1), v=x1 x2 gives x1+x2."""
    M = fem.mass(step)
    x, y = step.xy[:, 0], step.xy[:, 1]
    z = np.zeros_like(x)
    N = fem.convection(step, y, z)
    assert np.abs(N @ x - M @ y).max() < 1e-13
    N = fem.convection(step, z, x)
    assert np.abs(N @ y - M @ x).max() < 1e-13
    N = fem.convection(step, np.ones_like(x), np.ones_like(x))
    assert np.abs(N @ (x * y) - M @ (x + y)).max() < 1e-13


def test_poiseuille_is_reproduced_exactly():
    """Steady Stokes on the channel [0,2]x[-1,1]: u = (1 - x2^2, 0), p = -2 nu (x1 - 2)
    satisfies -nu lap u + grad p = 0, div u = 0 and the do-nothing outflow
    condition; both fields lie in Q2 x Q1, so the discrete solve returns them."""
    mesh = synth.channel_mesh(0.25, 2.0)
    nu = 0.05
    A = fem.stiffness(mesh, np.full(mesh.n_pnodes, nu))
    Bx, By = fem.divergence(mesh)
    f, D = mesh.free, mesh.dnodes
    n = mesh.n_nodes
    K = sp.bmat([[sp.block_diag([A[f][:, f], A[f][:, f]]), sp.hstack([Bx[:, f], By[:, f]]).T],
                 [sp.hstack([Bx[:, f], By[:, f]]), None]], format="csc")
    uD = np.concatenate([mesh.inflow[D], np.zeros(D.size)])
    AfD = sp.block_diag([A[f][:, D], A[f][:, D]])
    BD = sp.hstack([Bx[:, D], By[:, D]])
    rhs = -np.concatenate([AfD @ uD, BD @ uD])
    sol = spla.spsolve(K, rhs)
    y = mesh.xy[:, 1]
    u_exact = np.concatenate([(1 - y ** 2)[f], np.zeros(f.size)])
    p_exact = -2 * nu * (mesh.pxy[:, 0] - 2.0)
    assert np.abs(sol[:2 * f.size] - u_exact).max() < 1e-11
    assert np.abs(sol[2 * f.size:] - p_exact).max() < 1e-11


def test_step_dirichlet_set():
    """Free nodes: interior plus the open outflow segment; inflow profile 1 - 4 x2^2."""
    mesh = synth.step_mesh(0.25, 5.0)
    out = (np.abs(mesh.xy[:, 0] - 5.0) < 1e-12)
    assert not mesh.dirichlet[out & (np.abs(mesh.xy[:, 1]) < 1 - 1e-12)].any()
    assert mesh.dirichlet[out & (np.abs(mesh.xy[:, 1]) > 1 - 1e-12)].all()
    inflow = np.abs(mesh.xy[:, 0] + 1.0) < 1e-12
    assert mesh.dirichlet[inflow].all()
    assert np.allclose(mesh.inflow[inflow], 1 - 4 * mesh.xy[inflow, 1] ** 2)
    assert np.all(mesh.inflow[~inflow] == 0)
