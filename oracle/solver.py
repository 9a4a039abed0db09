"""Low-rank GMRES (Algorithm 4.2), mean-based preconditioning (Section 5) and
truncated inexact Picard (Algorithm 3.1 with eq. eps_soln, eq. eps_conv).

Oracle (test infrastructure only; see oracle/__init__.py).

Vectors are either single TTs (inner solve) or (velocity TT, pressure TT)
pairs (outer solve); the pair's TTs are truncated separately (Section 4.2).
Fixed choices where the paper leaves room (the GPU path makes the same ones):
z_0 = 0, no restarts, modified Gram-Schmidt without intermediate truncation,
h_{k+1,k} = ||x|| from the orthogonalised train and v_{k+1} = T(x)/h (T is
scale-equivariant), the stopping test on the norm of the truncated s_k, happy
breakdown when h_{k+1,k} <= 1e-14 beta.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .tt import (TT, add, dot, kron_apply, norm, pair_add, pair_dot, pair_scale,
                 round_tt, truncate)


# ---------------------------------------------------------------- vector spaces
class _Single:
    """Single TT vectors; round returns (T(v), ||v||, ||T(v)||)."""
    @staticmethod
    def add(*terms): return add(*terms)
    @staticmethod
    def round(v, eps):
        return truncate(v, eps)
    @staticmethod
    def dot(a, b): return dot(a, b)
    @staticmethod
    def scale(v, c): return v.scale(c)
    @staticmethod
    def zeros_like(v): return TT.zeros(*v.shape)


class _Pair:
    """(velocity, pressure) pairs, truncated separately (Section 4.2)."""
    @staticmethod
    def add(*terms): return pair_add(*terms)
    @staticmethod
    def round(v, eps):
        u, bu, au = truncate(v[0], eps)
        p, bp, ap = truncate(v[1], eps)
        return (u, p), float(np.hypot(bu, bp)), float(np.hypot(au, ap))
    @staticmethod
    def dot(a, b): return pair_dot(a, b)
    @staticmethod
    def scale(v, c): return pair_scale(v, c)
    @staticmethod
    def zeros_like(v): return (TT.zeros(*v[0].shape), TT.zeros(*v[1].shape))


def _lsq(Hbar, beta):
    """y = argmin ||beta e_1 - Hbar y|| (Algorithm 4.2): a dense least-squares solve."""
    rhs = np.zeros(Hbar.shape[0]); rhs[0] = beta
    y, *_ = np.linalg.lstsq(Hbar, rhs, rcond=None)
    return y


def gmres(apply_L, apply_P, b, *, tol, eps, maxit, space, bnorm=None, log=None):
    """Algorithm 4.2 with z_0 = 0 (flexible: v_hat_k = P^{-1} v_k stored).

    Returns (z, stats) with stats = dict(its, resnorms, ranks).
    """
    S = space
    s0, b_before, beta = S.round(b, eps)       # s_0 = T(b - L 0)
    if bnorm is None:
        bnorm = b_before
    stats = dict(its=0, res=[beta], bnorm=bnorm)
    if beta == 0.0 or beta <= tol * bnorm:
        return S.zeros_like(b), stats
    V = [S.scale(s0, 1.0 / beta)]
    Vh = []
    Hbar = np.zeros((maxit + 1, maxit))
    z = S.zeros_like(b)
    res = beta
    k = 0
    while res > tol * bnorm and k < maxit:
        k += 1
        vh = apply_P(V[k - 1])
        Vh.append(vh)
        x = S.round(apply_L(vh), eps)[0]
        for i in range(k):
            Hbar[i, k - 1] = S.dot(x, V[i])
            x = S.add((1.0, x), (-Hbar[i, k - 1], V[i]))
        xr, hk, _ = S.round(x, eps)            # h_{k+1,k} = ||x||, v_{k+1} = T(x) / h
        Hbar[k, k - 1] = hk
        breakdown = hk <= 1e-14 * beta
        if not breakdown:
            V.append(S.scale(xr, 1.0 / hk))
        y = _lsq(Hbar[:k + 1, :k], beta)
        z = S.round(S.add(*[(y[i], Vh[i]) for i in range(k)]), eps)[0]
        s, _, res = S.round(S.add((1.0, b), (-1.0, apply_L(z))), eps)
        stats["res"].append(res)
        if log is not None:
            log(k, res)
        if breakdown:
            break
    stats["its"] = k
    return z, stats



# ---------------------------------------------------------------- preconditioner
def mean_velocity_field(w):
    """Time average of the mean (psi_1) mode of the full-node convection TT w:
    the field w_avg of eq. (11_prec), as a (2 n_nodes,) vector."""
    c = w.z1.mean(axis=0) @ w.z2[:, 0, :]
    return c @ w.z3


def mean_oseen_matrix(disc, w):
    """K = tau^-1 M + A_0 + N(w_avg) over the free scalar velocity dofs, the
    spatial factor of eq. (11_prec) (w None: no convection)."""
    d = disc
    K = d.M / d.tau + d.A[0]
    if w is not None:
        wavg = mean_velocity_field(w)
        n = d.n_nodes
        from . import fem
        Nf = fem.convection(d.prob.mesh, wavg[:n], wavg[n:])
        K = K + Nf[d.free][:, d.free]
    return sp.csc_matrix(K)


class MeanLSC:
    """Mean-based block triangular preconditioner (eq. prec) with S^{-1} from
    eq. (mean_lsc) and the (1,1) solve by an inner low-rank GMRES preconditioned
    with M = (I - C) (x) I (x) (tau^-1 M + A_0 + N(w_avg)) (eq. 11_prec, Section 5.3).

    w: the (truncated) full-node convection TT, or None for the Stokes problem.
    """

    def __init__(self, disc, w, eps, tol_inner, maxit_inner, learned_minv=None):
        self.d, self.w, self.eps = disc, w, eps
        # optional replacement of M^{-1} in the inner solve (a learned K^{-1}); the
        # exact M^{-1} is the fallback when the inner solve misses its tolerance with it
        self.learned_minv = learned_minv
        self.fallbacks = 0
        self.tol_inner, self.maxit_inner = tol_inner, maxit_inner
        d = disc
        self.Minv = sp.diags(1.0 / d.Mstar_diag)
        Lp = (d.B @ self.Minv @ d.Bt).tocsc()                    # B M_*^{-1} B^T
        self.Lp = spla.splu(Lp)
        self.K = spla.splu(mean_oseen_matrix(d, w))
        n_t = d.n_t
        self.cum = np.tril(np.ones((n_t, n_t)))                  # (I - C)^{-1}
        self.inner_its = []

    def _space(self, Xop, z):
        return kron_apply(None, None, Xop, z)

    def _lp_solve(self, z):
        return TT(z.z1, z.z2, self.Lp.solve(z.z3.T).T)

    def apply_Minv(self, z):
        """M^{-1} z = ((I - C)^{-1} (x) I (x) K^{-1}) z, K^{-1} applied per component."""
        n = self.d.n_v
        Z = z.z3.T                                               # n_u x k2
        out = np.vstack([self.K.solve(Z[:n]), self.K.solve(Z[n:])])
        return TT(self.cum @ z.z1, z.z2, out.T)

    def schur(self, ap):
        """p = -S_LSC,0^{-1} a_p (eq. mean_lsc), truncated after the mean product."""
        d = self.d
        y = self._lp_solve(ap)
        y = self._space(self.Minv @ d.Bt, y)
        y, _ = round_tt(d.apply_mean(self.w, y), self.eps)
        y = self._space(d.B @ self.Minv, y)
        y = self._lp_solve(y)
        return y.scale(-1.0)

    def __call__(self, v):
        au, ap = v
        d = self.d
        p = self.schur(ap)
        rhs, _ = round_tt(add((1.0, au), (-1.0, kron_apply(None, None, d.Bt, p))), self.eps)
        A = lambda z: d.apply_mean(self.w, z)
        if self.learned_minv is not None:
            # the learned attempt gets a fifth of the inner budget (at least 4 iterations)
            u, st = gmres(A, self.learned_minv, rhs, tol=self.tol_inner, eps=self.eps,
                          maxit=min(self.maxit_inner, max(4, self.maxit_inner // 5)), space=_Single)
            if st["res"][-1] <= self.tol_inner * st["bnorm"]:
                self.inner_its.append(st["its"])
                return (u, p)
            self.fallbacks += 1
        u, st = gmres(A, self.apply_Minv, rhs, tol=self.tol_inner, eps=self.eps,
                      maxit=self.maxit_inner, space=_Single)
        self.inner_its.append(st["its"])
        return (u, p)


class MeanPCD(MeanLSC):
    """The same block triangular preconditioner with S^{-1} from the mean-based PCD
    approximation, eq. (mean_pcd): S_PCD,0^{-1} = (B M_*^{-1} B^T)^{-1} (F_p,0 + C_p) M_p*^{-1}."""

    def schur(self, ap):
        """p = -S_PCD,0^{-1} a_p, truncated after the pressure-space mean product."""
        d = self.d
        _, _, mpd = d.pressure_matrices()
        y = self._space(sp.diags(1.0 / mpd), ap)
        y, _ = round_tt(d.apply_mean_p(self.w, y), self.eps)
        y = self._lp_solve(y)
        return y.scale(-1.0)


# ---------------------------------------------------------------- Picard
def picard(disc, tol=None, log=None, schur="lsc"):
    """Truncated inexact Picard iteration (Algorithm 3.1, Sections 4.2, 4.3, 5.2).

    Returns (u, p, stats) with u, p TTs over the free velocity / pressure dofs.
    schur: "lsc" (eq. mean_lsc) or "pcd" (eq. mean_pcd) Schur complement approximation.
    """
    Prec = {"lsc": MeanLSC, "pcd": MeanPCD}[schur]
    t = tol or disc.prob.tol
    fu, fp = disc.rhs()
    f = (fu, fp)
    fnorm = float(np.hypot(norm(fu), norm(fp)))
    # Stokes problem for the initial iterate (N = 0), solved to tol_gmres ||f||
    P = Prec(disc, None, t.eps_gmres, t.tol_inner, t.maxit_inner)
    (u, p), st = gmres(lambda v: disc.apply(None, *v), P, f, tol=t.tol_gmres, eps=t.eps_gmres,
                       maxit=t.maxit_gmres, space=_Pair, bnorm=fnorm)
    stats = dict(fnorm=fnorm, stokes_its=st["its"], gmres_its=[], res=[], ranks=[], conv_ranks=[],
                 inner_its=[list(P.inner_its)])
    r, rn = disc.residual(u, p, t.eps_gmres)
    stats["res"].append(rn)
    i = 0
    while rn > t.tol_picard * fnorm and i < t.maxit_picard:
        i += 1
        wt, _ = round_tt(disc.full_velocity(u), t.eps_conv)           # eq. (eps_conv)
        P = Prec(disc, wt, t.eps_gmres, t.tol_inner, t.maxit_inner)
        (du, dp), st = gmres(lambda v: disc.apply(wt, *v), P, r, tol=t.tol_gmres, eps=t.eps_gmres,
                             maxit=t.maxit_gmres, space=_Pair, bnorm=rn)
        u, _ = round_tt(add((1.0, u), (1.0, du)), t.eps_soln)         # eq. (eps_soln)
        p, _ = round_tt(add((1.0, p), (1.0, dp)), t.eps_soln)
        r, rn = disc.residual(u, p, t.eps_gmres)
        stats["gmres_its"].append(st["its"]); stats["res"].append(rn)
        stats["ranks"].append((u.ranks, p.ranks, du.ranks, dp.ranks)); stats["conv_ranks"].append(wt.ranks)
        stats["inner_its"].append(list(P.inner_its))
        if log is not None:
            log(i, rn / fnorm, st["its"], u.ranks, p.ranks)
    stats["picard_its"] = i
    return u, p, stats


# ---------------------------------------------------------------- definition level
def direct_picard(disc, tol=1e-12, maxit=60):
    """Picard on the uncompressed all-at-once system (eq. ns_sys_all_iter) with a
    sparse direct solve per step, from the Stokes solution.  Returns full-tensor
    velocity (n_t, n_xi, n_u) and pressure (n_t, n_xi, n_p) and the step count."""
    fu, fp = disc.rhs()
    fuv, fpv = fu.vec(), fp.vec()
    uDv = disc.uD.vec()
    K, _ = disc.full_matrix(None)
    sol = spla.spsolve(K, np.concatenate([fuv, fpv]))
    nU = fuv.size
    n_t, n_xi = disc.n_t, disc.n_xi
    fnorm = np.linalg.norm(np.concatenate([fuv, fpv]))
    for it in range(maxit):
        uf = sol[:nU].reshape(n_t, n_xi, disc.n_u)
        wvec = _full_vec(disc, uf)
        K, NfD = disc.full_matrix(wvec)
        rhs_u = fuv - NfD @ uDv
        res = np.concatenate([rhs_u, fpv]) - K @ sol
        if np.linalg.norm(res) <= tol * fnorm:
            break
        sol = spla.spsolve(K, np.concatenate([rhs_u, fpv]))
    uf = sol[:nU].reshape(n_t, n_xi, disc.n_u)
    pf = sol[nU:].reshape(n_t, n_xi, disc.n_p)
    return uf, pf, it


def _full_vec(disc, uf):
    """Full-node velocity tensor from free-dof values plus the lifting (vectorised)."""
    n_t, n_xi = uf.shape[:2]
    n, f, D = disc.n_nodes, disc.free, disc.dn
    W = np.zeros((n_t, n_xi, 2 * n))
    W[:, :, f] = uf[:, :, :f.size]
    W[:, :, f + n] = uf[:, :, f.size:]
    W += disc.full_velocity(TT.zeros(n_t, n_xi, disc.n_u)).full()
    return W.reshape(-1)
