"""Q2-Q1 Taylor-Hood matrices of Section 3.2, eq. (mat_entries) and the B definition.

Oracle (test infrastructure only; see oracle/__init__.py).

On every square element of side h, velocity basis functions are biquadratic
(9 nodes) and pressure basis functions bilinear (4 vertices).  With 3 x 3 Gauss
points per element:
    [M]_ij   = (phi_j, phi_i)
    [A_l]_ij = (nu_l grad phi_j, grad phi_i)          nu_l bilinear (nodal on Q1)
    [N(w)]_ij = (w . grad phi_j, phi_i)               w a Q2 vector field
    [B_x1]_ij = -(varphi_i, d phi_j / d x1),  [B_x2]_ij = -(varphi_i, d phi_j / d x2)
All matrices are assembled over every node, then split into free (f) and
Dirichlet (D) column / row blocks.  Elements are written out one by one, as
the definitions read.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

_G = np.array([0.5 - 0.5 * np.sqrt(0.6), 0.5, 0.5 + 0.5 * np.sqrt(0.6)])
_W = np.array([5.0, 8.0, 5.0]) / 18.0


def _quad1(s):
    """1-D quadratic Lagrange basis on nodes 0, 1/2, 1 and its derivative."""
    v = np.array([2 * (s - 0.5) * (s - 1), -4 * s * (s - 1), 2 * s * (s - 0.5)])
    dv = np.array([4 * s - 3, -8 * s + 4, 4 * s - 1])
    return v, dv


def _lin1(s):
    return np.array([1 - s, s])


def reference_tables():
    """Basis values at the 9 Gauss points of the unit square.

    Returns phi (9q, 9), dphi_s (9q, 9), dphi_t (9q, 9), chi (9q, 4), w (9q,)
    with local velocity node a + 3b and pressure vertex a + 2b.
    """
    phi = np.zeros((9, 9)); ds = np.zeros((9, 9)); dt = np.zeros((9, 9))
    chi = np.zeros((9, 4)); w = np.zeros(9)
    q = 0
    for jt in range(3):
        for js in range(3):
            s, t = _G[js], _G[jt]
            vs, dvs = _quad1(s)
            vt, dvt = _quad1(t)
            ls, lt = _lin1(s), _lin1(t)
            for b in range(3):
                for a in range(3):
                    phi[q, a + 3 * b] = vs[a] * vt[b]
                    ds[q, a + 3 * b] = dvs[a] * vt[b]
                    dt[q, a + 3 * b] = vs[a] * dvt[b]
            for b in range(2):
                for a in range(2):
                    chi[q, a + 2 * b] = ls[a] * lt[b]
            w[q] = _W[js] * _W[jt]
            q += 1
    return phi, ds, dt, chi, w


def _scatter(rows, cols, vals, shape):
    return sp.csr_matrix(sp.coo_matrix((vals, (rows, cols)), shape=shape))


def mass(mesh):
    """Scalar Q2 mass matrix M over all velocity nodes."""
    phi, ds, dt, chi, w = reference_tables()
    h = mesh.h
    R, C, V = [], [], []
    for e in range(mesh.n_elem):
        nodes = mesh.elem_q2[e]
        Me = np.einsum("q,qi,qj->ij", w, phi, phi) * h * h
        R.append(np.repeat(nodes, 9)); C.append(np.tile(nodes, 9)); V.append(Me.ravel())
    n = mesh.n_nodes
    return _scatter(np.concatenate(R), np.concatenate(C), np.concatenate(V), (n, n))


def stiffness(mesh, nu_nodal):
    """Weighted stiffness A with viscosity nu bilinear on each element (nodal on Q1)."""
    phi, ds, dt, chi, w = reference_tables()
    R, C, V = [], [], []
    for e in range(mesh.n_elem):
        nodes = mesh.elem_q2[e]
        nu_q = chi @ nu_nodal[mesh.elem_q1[e]]                    # (9q,)
        # grad phi = (1/h) (d/ds, d/dt); Jacobian h^2 cancels the 1/h^2
        Ae = np.einsum("q,qi,qj->ij", w * nu_q, ds, ds) + np.einsum("q,qi,qj->ij", w * nu_q, dt, dt)
        R.append(np.repeat(nodes, 9)); C.append(np.tile(nodes, 9)); V.append(Ae.ravel())
    n = mesh.n_nodes
    return _scatter(np.concatenate(R), np.concatenate(C), np.concatenate(V), (n, n))


def convection(mesh, wx, wy):
    """N(w)_ij = (w . grad phi_j, phi_i) for the Q2 field w given at all velocity nodes."""
    phi, ds, dt, chi, w = reference_tables()
    h = mesh.h
    R, C, V = [], [], []
    for e in range(mesh.n_elem):
        nodes = mesh.elem_q2[e]
        w1 = phi @ wx[nodes]
        w2 = phi @ wy[nodes]
        # (w . grad phi_j) phi_i |J| = (w1 dphi_j/ds + w2 dphi_j/dt) phi_i h
        Ne = (np.einsum("q,qi,qj->ij", w * w1, phi, ds) + np.einsum("q,qi,qj->ij", w * w2, phi, dt)) * h
        R.append(np.repeat(nodes, 9)); C.append(np.tile(nodes, 9)); V.append(Ne.ravel())
    n = mesh.n_nodes
    return _scatter(np.concatenate(R), np.concatenate(C), np.concatenate(V), (n, n))


def divergence(mesh):
    """(B_x1, B_x2), each n_pnodes x n_nodes: [B_xk]_ij = -(varphi_i, d phi_j / d x_k)."""
    phi, ds, dt, chi, w = reference_tables()
    h = mesh.h
    R, C, Vx, Vy = [], [], [], []
    for e in range(mesh.n_elem):
        nodes = mesh.elem_q2[e]
        pn = mesh.elem_q1[e]
        Bx = -np.einsum("q,qi,qj->ij", w, chi, ds) * h
        By = -np.einsum("q,qi,qj->ij", w, chi, dt) * h
        R.append(np.repeat(pn, 9)); C.append(np.tile(nodes, 4))
        Vx.append(Bx.ravel()); Vy.append(By.ravel())
    shape = (mesh.n_pnodes, mesh.n_nodes)
    R, C = np.concatenate(R), np.concatenate(C)
    return _scatter(R, C, np.concatenate(Vx), shape), _scatter(R, C, np.concatenate(Vy), shape)


def pressure_mass(mesh):
    """Q1 pressure mass matrix M_p (used by the commutator identity of Section 5.2)."""
    phi, ds, dt, chi, w = reference_tables()
    h = mesh.h
    R, C, V = [], [], []
    for e in range(mesh.n_elem):
        pn = mesh.elem_q1[e]
        Me = np.einsum("q,qi,qj->ij", w, chi, chi) * h * h
        R.append(np.repeat(pn, 4)); C.append(np.tile(pn, 4)); V.append(Me.ravel())
    n = mesh.n_pnodes
    return _scatter(np.concatenate(R), np.concatenate(C), np.concatenate(V), (n, n))


def _pressure_tables():
    """Bilinear basis values and derivatives (d/ds, d/dt) at the 9 Gauss points of the
    unit square, vertex a + 2b, in the point order of reference_tables()."""
    chi = np.zeros((9, 4)); cs = np.zeros((9, 4)); ct = np.zeros((9, 4))
    q = 0
    for jt in range(3):
        for js in range(3):
            s, t = _G[js], _G[jt]
            ls, lt = _lin1(s), _lin1(t)
            dl = np.array([-1.0, 1.0])
            for b in range(2):
                for a in range(2):
                    chi[q, a + 2 * b] = ls[a] * lt[b]
                    cs[q, a + 2 * b] = dl[a] * lt[b]
                    ct[q, a + 2 * b] = ls[a] * dl[b]
            q += 1
    return chi, cs, ct


def pressure_stiffness(mesh, nu_nodal):
    """Q1 pressure-space diffusion A_p (Section 5.2, the pressure analogue of A_0):
    [A_p]_ij = (nu grad varphi_j, grad varphi_i), nu bilinear (nodal on Q1), natural
    boundary conditions (no boundary terms removed or added)."""
    phi, ds, dt, chi0, w = reference_tables()
    chi, cs, ct = _pressure_tables()
    R, C, V = [], [], []
    for e in range(mesh.n_elem):
        pn = mesh.elem_q1[e]
        nu_q = chi @ nu_nodal[pn]
        # grad varphi = (1/h) (d/ds, d/dt); the Jacobian h^2 cancels the 1/h^2
        Ae = np.einsum("q,qi,qj->ij", w * nu_q, cs, cs) + np.einsum("q,qi,qj->ij", w * nu_q, ct, ct)
        R.append(np.repeat(pn, 4)); C.append(np.tile(pn, 4)); V.append(Ae.ravel())
    n = mesh.n_pnodes
    return _scatter(np.concatenate(R), np.concatenate(C), np.concatenate(V), (n, n))


def pressure_convection(mesh, wx, wy):
    """Q1 pressure-space convection N_p(w) (Section 5.2): [N_p(w)]_ij =
    (w . grad varphi_j, varphi_i) for the Q2 field w given at all velocity nodes."""
    phi, ds, dt, chi0, w = reference_tables()
    chi, cs, ct = _pressure_tables()
    h = mesh.h
    R, C, V = [], [], []
    for e in range(mesh.n_elem):
        nodes = mesh.elem_q2[e]
        pn = mesh.elem_q1[e]
        w1 = phi @ wx[nodes]
        w2 = phi @ wy[nodes]
        Ne = (np.einsum("q,qi,qj->ij", w * w1, chi, cs) + np.einsum("q,qi,qj->ij", w * w2, chi, ct)) * h
        R.append(np.repeat(pn, 4)); C.append(np.tile(pn, 4)); V.append(Ne.ravel())
    n = mesh.n_pnodes
    return _scatter(np.concatenate(R), np.concatenate(C), np.concatenate(V), (n, n))
