"""Problem presets and the conventions both solvers share.

A `Problem` is the statement of the discrete all-at-once problem of Sections 3
and 5.1: mesh, nodal viscosity fields, gPC index set, time grid, inflow time
profile and solver tolerances.  Nothing here solves or assembles anything.

Presets:
  * `tiny`   : smallest case the definition-level oracle (a sparse direct solve
               of the uncompressed all-at-once system) handles in a second;
  * `small`  : step L=5, element 1/4 (velocity spacing 1/8), m=2, d=2 (n_xi=6),
               n_t=20, tau=0.1, nu0=1/50, sigma=0.1, truncation 1e-6;
  * `medium` : element 1/8 (spacing 1/16), m=3, d=3 (n_xi=20), n_t=100,
               tau=0.05, nu0=1/100, sigma=0.2, truncation 1e-5;
  * `large`  : element 1/16 (spacing 1/32), m=5, d=3 (n_xi=56), n_t=400,
               tau=0.025, nu0=1/200, sigma=0.25, truncation 1e-5;
  * `paper`  : Table 5.1 (L=12, h=1/4, n_t=64, tau=1/64, nu0=1/50, sigma=0.01,
               b=4, m=3, d=3) with the Table 5.2 tolerances.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from itertools import product

import numpy as np

from .kl import viscosity_fields
from .mesh import Mesh, channel_mesh, step_mesh


def gpc_multi_indices(m: int, d: int) -> np.ndarray:
    """Multi-indices of the total-degree-d Legendre chaos in m variables.

    Order (a convention shared by both solvers): total degree ascending, then
    descending lexicographic within a degree, so index 0 is the constant
    (psi_1 = 1 of Section 5.2) and indices 1..m are xi_1..xi_m.
    """
    idx = [a for a in product(range(d + 1), repeat=m) if sum(a) <= d]
    idx.sort(key=lambda a: (sum(a), tuple(-x for x in a)))
    return np.array(idx, dtype=np.int64).reshape(len(idx), m)


def n_xi(m: int, d: int) -> int:
    """(m + d)! / (m! d!) (Section 5.1)."""
    from math import comb
    return comb(m + d, d)


@dataclass
class Tolerances:
    """Stopping and truncation tolerances (Table 5.2 names)."""
    tol_picard: float = 1e-5
    tol_gmres: float = 1e-1
    eps_gmres: float = 1e-3
    eps_soln: float = 1e-7
    eps_conv: float = 1e-3
    tol_inner: float = 1e-1
    maxit_picard: int = 20
    maxit_gmres: int = 50
    maxit_inner: int = 50


@dataclass
class Problem:
    name: str
    mesh: Mesh
    nu: np.ndarray            # (m+1, n_pnodes) nodal viscosity fields
    m: int
    d: int
    mi: np.ndarray            # (n_xi, m) gPC multi-indices
    n_t: int
    tau: float
    tprofile: np.ndarray      # (n_t,) inflow ramp 1 - exp(-10 t_k), t_k = k tau
    tol: Tolerances = field(default_factory=Tolerances)
    params: dict = field(default_factory=dict)

    @property
    def n_xi(self) -> int:
        return self.mi.shape[0]

    @property
    def n_v(self) -> int:
        return self.mesh.n_v

    @property
    def n_u(self) -> int:
        return 2 * self.mesh.n_v

    @property
    def n_p(self) -> int:
        return self.mesh.n_pnodes

    def lifting_values(self) -> np.ndarray:
        """Dirichlet values at the Dirichlet nodes, shape (2, n_dirichlet): steady
        profile; the time factor is `tprofile` (Section 5.1 inflow)."""
        d = self.mesh.dnodes
        out = np.zeros((2, d.size))
        out[0] = self.mesh.inflow[d]
        return out


def time_profile(n_t: int, tau: float) -> np.ndarray:
    t = tau * np.arange(1, n_t + 1)
    return 1.0 - np.exp(-10.0 * t)


def make_problem(name: str, *, h, L=5.0, m, d, n_t, tau, nu0, sigma, b=1.0,
                 tol: Tolerances | None = None, kind="step") -> Problem:
    mesh = step_mesh(h, L) if kind == "step" else channel_mesh(h, L)
    nu, beta = viscosity_fields(mesh, nu0, sigma, b, m)
    return Problem(name=name, mesh=mesh, nu=nu, m=m, d=d, mi=gpc_multi_indices(m, d),
                   n_t=n_t, tau=tau, tprofile=time_profile(n_t, tau),
                   tol=tol or Tolerances(),
                   params=dict(h=h, L=L, nu0=nu0, sigma=sigma, b=b, kl_beta=beta, kind=kind))


def preset(name: str, **over) -> Problem:
    """Named workloads (sizes in the module docstring)."""
    if name == "tiny":
        kw = dict(h=0.5, L=1.0, m=1, d=2, n_t=4, tau=0.25, nu0=1 / 20, sigma=0.1, b=1.0,
                  tol=Tolerances(eps_gmres=1e-8, eps_soln=1e-10, eps_conv=1e-8))
    elif name == "small":
        kw = dict(h=0.25, L=5.0, m=2, d=2, n_t=20, tau=0.1, nu0=1 / 50, sigma=0.1, b=1.0,
                  tol=Tolerances(eps_gmres=1e-6))
    elif name == "medium":
        kw = dict(h=0.125, L=5.0, m=3, d=3, n_t=100, tau=0.05, nu0=1 / 100, sigma=0.2, b=1.0,
                  tol=Tolerances(eps_gmres=1e-5))
    elif name == "large":
        kw = dict(h=0.0625, L=5.0, m=5, d=3, n_t=400, tau=0.025, nu0=1 / 200, sigma=0.25, b=1.0,
                  tol=Tolerances(eps_gmres=1e-5))
    elif name == "paper":
        kw = dict(h=0.25, L=12.0, m=3, d=3, n_t=64, tau=1 / 64, nu0=1 / 50, sigma=0.01, b=4.0,
                  tol=Tolerances())
    else:
        raise KeyError(name)
    kw.update(over)
    return make_problem(name, **kw)


def batch(name: str, count: int, seed: int = 5, nu0_range=(1 / 200, 1 / 50), sigma_range=(0.05, 0.3),
          **over) -> list:
    """`count` independent problems of preset `name` with seeded draws of the
    viscosity: nu0 log-uniform in nu0_range, sigma uniform in sigma_range."""
    rng = np.random.default_rng(seed)
    lo, hi = np.log(nu0_range[0]), np.log(nu0_range[1])
    out = []
    for _ in range(count):
        nu0 = float(np.exp(rng.uniform(lo, hi)))
        sigma = float(rng.uniform(*sigma_range))
        out.append(preset(name, nu0=nu0, sigma=sigma, **over))
    return out


def random_tt(n_t, n_xi_, n_x, r1, r2, seed=0, decay=None):
    """Seeded random TT cores in the paper's shapes (n_t x r1, r1 x n_xi x r2, r2 x n_x).

    With `decay`, the cores are built so the two unfoldings have singular values
    10**(-decay * i / r): Gaussian cores are orthonormalised and the spectra are
    placed between them.
    """
    rng = np.random.default_rng(seed)
    z1 = rng.standard_normal((n_t, r1))
    z2 = rng.standard_normal((r1, n_xi_, r2))
    z3 = rng.standard_normal((r2, n_x))
    if decay is not None:
        if r1 > n_t or r2 > n_x or r2 > r1 * n_xi_:
            raise ValueError("a prescribed spectrum needs ranks no larger than the mode sizes")
        q1, _ = np.linalg.qr(z1)
        z1 = q1[:, :r1] * (10.0 ** (-decay * np.arange(r1) / max(r1, 1)))[None, :]
        q3, _ = np.linalg.qr(z3.T)
        z3 = (q3[:, :r2] * (10.0 ** (-decay * np.arange(r2) / max(r2, 1)))[None, :]).T
        q2, _ = np.linalg.qr(z2.reshape(r1 * n_xi_, r2))
        z2 = q2[:, :r2].reshape(r1, n_xi_, r2)
    return z1, z2, z3
