"""Karhunen-Loeve modes of the viscosity field (Section 5.1, problem data).

The random viscosity is nu(x, xi) = nu0 (1 + sigma sum_l sqrt(beta_l) a_l(x) xi_l)
with (beta_l, a_l) the leading eigenpairs of the exponential covariance
c(x, y) = exp(-|x - y|_1 / b) on the domain.  The paper only says the pairs come
from "a standard finite element method"; here they come from the Galerkin
eigenproblem C a = beta M a in the bilinear (Q1) space of a mesh whose element
side is `h_kl` (1/4 unless the flow mesh is coarser), with 3 x 3 Gauss points
per element for both integrals, a_l normalised in L2 and signed so that the
integral of a_l is non-negative (else its largest nodal magnitude is positive).
The resulting bilinear fields are then sampled at the flow mesh's pressure
nodes; because the meshes are nested this is exact.

This is the random-field model (an input of the discrete problem), not part
of the solver.  The output is nodal values nu_l (l = 0..m) on the flow mesh's
Q1 vertices, with nu_0 = nu0 constant.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from .mesh import Mesh, step_mesh, channel_mesh

_G = np.array([0.5 - 0.5 * np.sqrt(0.6), 0.5, 0.5 + 0.5 * np.sqrt(0.6)])
_W = np.array([5.0, 8.0, 5.0]) / 18.0


def _q1_quadrature(pxy, elem_q1, h):
    """Quadrature points, weights and the (points x nodes) bilinear evaluation matrix."""
    ne = elem_q1.shape[0]
    s, t = np.meshgrid(_G, _G, indexing="xy")          # s along x1, t along x2
    ws = np.outer(_W, _W)                                # [t, s]
    s, t, ws = s.ravel(), t.ravel(), ws.ravel()
    phi = np.stack([(1 - s) * (1 - t), s * (1 - t), (1 - s) * t, s * t], axis=1)  # (9, 4)
    x0 = pxy[elem_q1[:, 0]]                              # lower-left corners
    X = (x0[:, None, :] + h * np.stack([s, t], axis=1)[None]).reshape(-1, 2)
    W = np.tile(ws * h * h, ne)
    rows = np.repeat(np.arange(ne * 9), 4)
    cols = np.repeat(elem_q1, 9, axis=0).ravel()
    vals = np.tile(phi, (ne, 1)).ravel()
    P = np.zeros((ne * 9, pxy.shape[0]))
    np.add.at(P, (rows, cols), vals)
    return X, W, P


def kl_eigenpairs(pxy, elem_q1, h, b, m):
    """Leading m Galerkin eigenpairs (beta_l, nodal a_l) of exp(-|x-y|_1/b)."""
    X, W, P = _q1_quadrature(pxy, elem_q1, h)
    D = np.abs(X[:, None, 0] - X[None, :, 0]) + np.abs(X[:, None, 1] - X[None, :, 1])
    K = np.exp(-D / b)
    PW = P * W[:, None]
    C = PW.T @ K @ PW
    M = PW.T @ P
    C = 0.5 * (C + C.T)
    beta, A = scipy.linalg.eigh(C, M)
    idx = np.argsort(beta)[::-1][:m]
    beta, A = beta[idx], A[:, idx]
    mass1 = M.sum(axis=0)
    for l in range(A.shape[1]):
        integ = mass1 @ A[:, l]
        if abs(integ) > 1e-10 * np.abs(A[:, l]).max():
            if integ < 0:
                A[:, l] = -A[:, l]
        elif A[np.argmax(np.abs(A[:, l])), l] < 0:
            A[:, l] = -A[:, l]
    return beta, A, M


def _bilinear_sample(coarse: Mesh, field: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Evaluate a bilinear field on `coarse` (nodal values on its Q1 vertices) at pts."""
    hc = coarse.h
    out = np.empty(pts.shape[0])
    corners = coarse.pxy[coarse.elem_q1[:, 0]]
    for k, p in enumerate(pts):
        rel = (p[None, :] - corners) / hc
        inside = np.all((rel >= -1e-9) & (rel <= 1 + 1e-9), axis=1)
        e = int(np.flatnonzero(inside)[0])
        s, t = np.clip(rel[e], 0.0, 1.0)
        v = field[coarse.elem_q1[e]]
        out[k] = v[0] * (1 - s) * (1 - t) + v[1] * s * (1 - t) + v[2] * (1 - s) * t + v[3] * s * t
    return out


def viscosity_fields(mesh: Mesh, nu0: float, sigma: float, b: float, m: int,
                     h_kl: float = 0.25) -> tuple[np.ndarray, np.ndarray]:
    """Nodal viscosity fields nu_l (l = 0..m) on the flow mesh's pressure nodes.

    Returns (nu, beta): nu has shape (m + 1, n_pnodes), nu[0] = nu0 and
    nu[l] = nu0 sigma sqrt(beta_l) a_l for l >= 1.
    """
    h_kl = max(h_kl, mesh.h)
    if mesh.kind == "step":
        coarse = step_mesh(h_kl, mesh.params["L"], mesh.params["inlet_len"])
    elif mesh.kind == "channel":
        coarse = channel_mesh(h_kl, mesh.params["L"])
    else:
        raise ValueError(mesh.kind)
    nu = np.empty((m + 1, mesh.n_pnodes))
    nu[0] = nu0
    beta = np.zeros(0)
    if m > 0:
        beta, A, _ = kl_eigenpairs(coarse.pxy, coarse.elem_q1, coarse.h, b, m)
        for l in range(m):
            a = A[:, l] if coarse.h == mesh.h else _bilinear_sample(coarse, A[:, l], mesh.pxy)
            nu[l + 1] = nu0 * sigma * np.sqrt(max(beta[l], 0.0)) * a
    # nu >= nu_min > 0 for every xi in the box [-sqrt 3, sqrt 3]^m (Section 2);
    # the field is bilinear per element, so its extremes sit at the nodes.
    worst = nu[0] - np.sqrt(3.0) * np.abs(nu[1:]).sum(axis=0)
    if worst.min() <= 0:
        raise ValueError("viscosity is not positive for all xi: lower sigma")
    return nu, beta
