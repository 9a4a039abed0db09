"""The all-at-once stochastic Galerkin system of Section 3.3 and its pieces.

Oracle (test infrastructure only; see oracle/__init__.py).

`Discretisation` holds the spatial matrices restricted to free (f) and
Dirichlet (D) velocity degrees of freedom, the gPC matrices, the time shift
C_{n_t} and the Dirichlet lifting.  Velocity vectors order the x1-components
of the free nodes first, then the x2-components (the basis ordering of
Section 3.2); bold matrices are 2 x 2 block diagonal with identical scalar
blocks.

Unknowns are corrections on the free degrees of freedom.  The full velocity
is w = E u + u_D, where u_D (rank one: inflow ramp (x) psi_1 (x) boundary values)
carries the Dirichlet data; the convection field of N(.) is always the full
velocity on every node.

Operators (all as sums of Kronecker products, eq. (F), eq. (N_kron)):
  L(w)[u; p] = [ tau^-1 (I(x)I(x)M) u + sum_l (I(x)G_l(x)A_l) u + N(w) u
                 - tau^-1 (C(x)I(x)M) u + (I(x)I(x)B^T) p ;  (I(x)I(x)B) u ]
  mean:  (F_0 + C) u with N_0(w) = sum diag(w1_a) (x) w2(a,1,b) I (x) N(w3_b)  (Section 5.2)
Right-hand side (Dirichlet lifting): f = -[A_fD-type couplings] u_D, see `rhs`.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fem, gpc
from .tt import TT, add, kron_apply, round_tt


def shift_matrix(n_t):
    """C_{n_t}: ones on the first subdiagonal (Section 3.3)."""
    return sp.diags([np.ones(n_t - 1)], [-1], shape=(n_t, n_t), format="csr")


def bd2(A):
    """2 x 2 block diagonal matrix with identical scalar blocks."""
    return sp.block_diag([A, A], format="csr")


class Discretisation:
    def __init__(self, prob):
        mesh = prob.mesh
        self.prob = prob
        self.n_t, self.tau = prob.n_t, prob.tau
        self.m = prob.m
        self.free, self.dn = mesh.free, mesh.dnodes
        f, D = self.free, self.dn
        self.n_nodes = mesh.n_nodes
        self.n_v = f.size
        self.n_u = 2 * f.size
        self.n_p = mesh.n_pnodes
        self.n_xi = prob.n_xi
        Mfull = fem.mass(mesh)
        self.Mfull = Mfull
        Afull = [fem.stiffness(mesh, prob.nu[l]) for l in range(prob.m + 1)]
        Bx, By = fem.divergence(mesh)
        self.Bxfull, self.Byfull = Bx, By
        self.M = Mfull[f][:, f]
        self.MfD = Mfull[f][:, D]
        self.A = [A[f][:, f] for A in Afull]
        self.AfD = [A[f][:, D] for A in Afull]
        self.bM = bd2(self.M)
        self.bMfD = bd2(self.MfD)
        self.bA = [bd2(A) for A in self.A]
        self.bAfD = [bd2(A) for A in self.AfD]
        self.B = sp.hstack([Bx[:, f], By[:, f]], format="csr")          # n_p x n_u
        self.BD = sp.hstack([Bx[:, D], By[:, D]], format="csr")         # n_p x 2 n_D
        self.Bt = self.B.T.tocsr()
        self.G = gpc.g_matrices(prob.mi)
        self.H = gpc.h_matrices(prob.mi)
        self.C = shift_matrix(self.n_t)
        # diagonal of the consistent mass matrix (the "M_*" of Section 5.1)
        self.Mstar_diag = np.concatenate([self.M.diagonal(), self.M.diagonal()])
        # lifting u_D: ramp (x) psi_1 (x) boundary values (x1 comps then x2 comps)
        e0 = np.zeros(self.n_xi); e0[0] = 1.0
        self.uD = TT.rank1(prob.tprofile, e0, prob.lifting_values().reshape(-1))

    # ---- velocity embedding --------------------------------------------------------
    def full_velocity(self, u):
        """Full-node velocity TT w = E u + u_D (2 n_nodes spatial rows)."""
        f, D, n = self.free, self.dn, self.n_nodes
        E = sp.csr_matrix((np.ones(2 * f.size), (np.concatenate([f, f + n]), np.arange(2 * f.size))),
                          shape=(2 * n, 2 * f.size))
        ED = sp.csr_matrix((np.ones(2 * D.size), (np.concatenate([D, D + n]), np.arange(2 * D.size))),
                           shape=(2 * n, 2 * D.size))
        return add((1.0, kron_apply(None, None, E, u)), (1.0, kron_apply(None, None, ED, self.uD)))

    def conv_matrix(self, w3col, rows="f", cols="f"):
        """Bold N(w) for one full-node Q2 field (length 2 n_nodes), restricted."""
        n = self.n_nodes
        Nfull = fem.convection(self.prob.mesh, w3col[:n], w3col[n:])
        r = self.free if rows == "f" else np.arange(n)
        c = {"f": self.free, "D": self.dn, "all": np.arange(n)}[cols]
        return bd2(Nfull[r][:, c])

    def hmix(self, w2, a, b):
        """sum_l w2(a, l, b) H_l (eq. N_kron)."""
        return np.einsum("l,lrs->rs", w2[a, :, b], self.H)

    # ---- operators on TTs ----------------------------------------------------------
    def conv_terms(self, w, z, cols="f", mean=False):
        """N(w) z (eq. N_kron) or N_0(w) z (Section 5.2), one term per (a, b), as a list of TTs."""
        out = []
        k1, k2 = w.ranks
        Nb = [self.conv_matrix(w.z3[b], "f", cols) for b in range(k2)]
        for a in range(k1):
            Da = sp.diags(w.z1[:, a])
            for b in range(k2):
                S = w.z2[a, 0, b] * np.eye(self.n_xi) if mean else self.hmix(w.z2, a, b)
                out.append(kron_apply(Da, S, Nb[b], z))
        return out

    def conv_apply(self, w, z, cols="f", mean=False):
        """The same sum as one TT: the terms of eq. (N_kron) that share diag(w1_a) share
        a first-core block, those that share N(w3_b) share a last-core block, and the
        middle core holds (sum_l w2(a,l,b) H_l) z2 in block (a, b).  Identical tensor
        to adding the terms of conv_terms one by one, with far smaller ranks."""
        k1, k2 = w.ranks
        r1, r2 = z.ranks
        n_t, n_xi = self.n_t, self.n_xi
        z1 = np.hstack([w.z1[:, a:a + 1] * z.z1 for a in range(k1)])
        z3 = np.vstack([np.asarray((self.conv_matrix(w.z3[b], "f", cols) @ z.z3.T).T) for b in range(k2)])
        z2 = np.zeros((k1 * r1, n_xi, k2 * r2))
        for a in range(k1):
            for b in range(k2):
                S = w.z2[a, 0, b] * np.eye(n_xi) if mean else self.hmix(w.z2, a, b)
                z2[a * r1:(a + 1) * r1, :, b * r2:(b + 1) * r2] = np.einsum("rs,asb->arb", S, z.z2)
        return TT(z1, z2, z3)

    def apply(self, w, u, p, eps=0.0):
        """L(w)[u; p] with convection field w (None: Stokes, N = 0); rounded if eps > 0."""
        ti = 1.0 / self.tau
        terms = [(ti, kron_apply(None, None, self.bM, u)),
                 (-ti, kron_apply(self.C, None, self.bM, u))]
        terms += [(1.0, kron_apply(None, self.G[l], self.bA[l], u)) for l in range(self.m + 1)]
        if w is not None:
            terms += [(1.0, self.conv_apply(w, u))]
        terms += [(1.0, kron_apply(None, None, self.Bt, p))]
        uo = add(*terms)
        po = kron_apply(None, None, self.B, u)
        if eps > 0:
            uo, po = round_tt(uo, eps)[0], round_tt(po, eps)[0]
        return uo, po

    def apply_mean(self, w, u):
        """(F_0 + C) u for the mean matrix of Section 5.2 (w None: no convection)."""
        ti = 1.0 / self.tau
        terms = [(ti, kron_apply(None, None, self.bM, u)),
                 (-ti, kron_apply(self.C, None, self.bM, u)),
                 (1.0, kron_apply(None, None, self.bA[0], u))]
        if w is not None:
            terms += [(1.0, self.conv_apply(w, u, mean=True))]
        return add(*terms)

    # ---- pressure space (mean-based PCD, Section 5.2) ------------------------------
    def pressure_matrices(self):
        """M_p, A_p,0 (mean viscosity) and the diagonal of M_p (the M_p* of eq. mean_pcd),
        assembled on first use."""
        if not hasattr(self, "_pm"):
            mesh = self.prob.mesh
            Mp = fem.pressure_mass(mesh)
            Ap0 = fem.pressure_stiffness(mesh, self.prob.nu[0])
            self._pm = (Mp, Ap0, Mp.diagonal())
        return self._pm

    def pconv_matrix(self, w3col):
        """N_p(w) on the pressure space for one full-node Q2 field (length 2 n_nodes)."""
        n = self.n_nodes
        return fem.pressure_convection(self.prob.mesh, w3col[:n], w3col[n:])

    def apply_mean_p(self, w, p):
        """(F_p,0 + C_p) p (Section 5.2): tau^-1 (I (x) I (x) M_p) p + (I (x) I (x) A_p,0) p
        + N_p,0(w) p - tau^-1 (C (x) I (x) M_p) p, with N_p,0(w) = sum_a sum_b diag(w1_a)
        (x) w2(a,1,b) I (x) N_p(w3_b) (w None: no convection), one term at a time."""
        Mp, Ap0, _ = self.pressure_matrices()
        ti = 1.0 / self.tau
        terms = [(ti, kron_apply(None, None, Mp, p)),
                 (1.0, kron_apply(None, None, Ap0, p)),
                 (-ti, kron_apply(self.C, None, Mp, p))]
        if w is not None:
            k1, k2 = w.ranks
            for b in range(k2):
                Npb = self.pconv_matrix(w.z3[b])
                for a in range(k1):
                    terms.append((1.0, kron_apply(sp.diags(w.z1[:, a]), w.z2[a, 0, b] * np.eye(self.n_xi), Npb, p)))
        return add(*terms)

    def rhs(self):
        """f = (f^u; f^p): the Dirichlet data moved to the right-hand side (linear part).

        f^u = -[tau^-1 (I - C) (x) I (x) M_fD + sum_l I (x) G_l (x) A_l,fD] u_D,
        f^p = -(I (x) I (x) B_D) u_D.
        """
        ti = 1.0 / self.tau
        terms = [(-ti, kron_apply(None, None, self.bMfD, self.uD)),
                 (ti, kron_apply(self.C, None, self.bMfD, self.uD))]
        terms += [(-1.0, kron_apply(None, self.G[l], self.bAfD[l], self.uD)) for l in range(self.m + 1)]
        fu = add(*terms)
        fp = kron_apply(None, None, self.BD, self.uD).scale(-1.0)
        return fu, fp

    def residual(self, u, p, eps):
        """r = f - A(w)[u; p] with the untruncated full velocity w in N (Section 4.3),
        truncated with eps (Section 4.2).  Returns ((r_u, r_p), ||r||)."""
        fu, fp = self.rhs()
        w = self.full_velocity(u)
        lu, lp = self.apply(None, u, p)                 # linear part
        nw = self.conv_apply(w, w, cols="all")          # [N(w) w]_free
        ru = add((1.0, fu), (-1.0, lu), (-1.0, nw))
        rp = add((1.0, fp), (-1.0, lp))
        ru, _ = round_tt(ru, eps)
        rp, _ = round_tt(rp, eps)
        from .tt import norm
        return (ru, rp), float(np.hypot(norm(ru), norm(rp)))

    # ---- dense / sparse forms for tiny cases ---------------------------------------
    def full_matrix(self, wvec=None):
        """Uncompressed all-at-once matrix [[F(w) + C, B^T], [B, 0]] (eq. ns_sys_all_iter).

        wvec: full-node velocity vector of length n_t n_xi 2 n_nodes (None: Stokes).
        Returns (K, Nfd): K over the free unknowns and the free-row x Dirichlet-column
        convection block needed for the right-hand side.
        """
        n_t, n_xi = self.n_t, self.n_xi
        It, Ix = sp.identity(n_t), sp.identity(n_xi)
        ti = 1.0 / self.tau
        F = ti * sp.kron(sp.kron(It, Ix), self.bM) - ti * sp.kron(sp.kron(self.C, Ix), self.bM)
        for l in range(self.m + 1):
            F = F + sp.kron(sp.kron(It, sp.csr_matrix(self.G[l])), self.bA[l])
        NfD = None
        if wvec is not None:
            W = wvec.reshape(n_t, n_xi, -1)
            blocks, bfd = [], []
            for k in range(n_t):
                Nk = None; NkD = None
                for l in range(n_xi):
                    Hl = sp.csr_matrix(self.H[l])
                    t1 = sp.kron(Hl, self.conv_matrix(W[k, l], "f", "f"))
                    t2 = sp.kron(Hl, self.conv_matrix(W[k, l], "f", "D"))
                    Nk = t1 if Nk is None else Nk + t1
                    NkD = t2 if NkD is None else NkD + t2
                blocks.append(Nk); bfd.append(NkD)
            F = F + sp.block_diag(blocks)
            NfD = sp.block_diag(bfd).tocsr()
        Bb = sp.kron(sp.identity(n_t * n_xi), self.B)
        K = sp.bmat([[F, Bb.T], [Bb, None]], format="csc")
        return K, NfD
