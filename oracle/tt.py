"""Three-core tensor trains of Section 4.1.

Oracle (test infrastructure only; see oracle/__init__.py).

A tensor z in R^{n_t x n_xi x n_x} is held as cores z1 (n_t x k1), z2 (k1 x n_xi x k2),
z3 (k2 x n_x) with z(i1,i2,i3) = sum z1(i1,a1) z2(a1,i2,a2) z3(a2,i3) (eq. z_tt);
vec(z) runs over i3 fastest, then i2, then i1 (the index map of Section 4.1).

Operations follow the text of Section 4.1: the Kronecker matrix-vector product
of eq. (Xz), addition by concatenating cores, inner products by contracting
cores, TT-SVD (Algorithm 4.1) for full tensors, and the truncation T_eps of an
existing tensor train, with delta_j = eps ||z||_F / sqrt(d - 1), d = 3.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class TT:
    __slots__ = ("z1", "z2", "z3")

    def __init__(self, z1, z2, z3):
        self.z1 = np.asarray(z1, dtype=np.float64)
        self.z2 = np.asarray(z2, dtype=np.float64)
        self.z3 = np.asarray(z3, dtype=np.float64)
        assert self.z1.shape[1] == self.z2.shape[0] and self.z2.shape[2] == self.z3.shape[0]

    @property
    def shape(self):
        return (self.z1.shape[0], self.z2.shape[1], self.z3.shape[1])

    @property
    def ranks(self):
        return (self.z1.shape[1], self.z3.shape[0])

    def full(self):
        """Dense n_t x n_xi x n_x array (eq. z_tt)."""
        n_t, n_xi, n_x = self.shape
        k1, k2 = self.ranks
        left = (self.z1 @ self.z2.reshape(k1, n_xi * k2)).reshape(n_t * n_xi, k2)
        return (left @ self.z3).reshape(n_t, n_xi, n_x)

    def vec(self):
        return self.full().reshape(-1)

    def copy(self):
        return TT(self.z1.copy(), self.z2.copy(), self.z3.copy())

    def scale(self, a):
        return TT(self.z1 * a, self.z2, self.z3)

    @staticmethod
    def zeros(n_t, n_xi, n_x):
        return TT(np.zeros((n_t, 1)), np.zeros((1, n_xi, 1)), np.zeros((1, n_x)))

    @staticmethod
    def rank1(a, b, c):
        return TT(np.asarray(a, float)[:, None], np.asarray(b, float)[None, :, None],
                  np.asarray(c, float)[None, :])


def add(*terms):
    """Sum of tensor trains (coefficient, TT) by concatenation (Section 4.1): ranks add."""
    terms = [(c, t) for c, t in terms]
    n_t, n_xi, n_x = terms[0][1].shape
    k1 = sum(t.ranks[0] for _, t in terms)
    k2 = sum(t.ranks[1] for _, t in terms)
    z1 = np.zeros((n_t, k1)); z2 = np.zeros((k1, n_xi, k2)); z3 = np.zeros((k2, n_x))
    a = b = 0
    for c, t in terms:
        r1, r2 = t.ranks
        z1[:, a:a + r1] = c * t.z1
        z2[a:a + r1, :, b:b + r2] = t.z2
        z3[b:b + r2, :] = t.z3
        a += r1; b += r2
    return TT(z1, z2, z3)


def dot(x, y):
    """<vec x, vec y> by contracting the cores from the first to the last."""
    W = x.z1.T @ y.z1                                        # k1x x k1y
    T = np.einsum("ab,bsd->asd", W, y.z2)                    # k1x x n_xi x k2y
    W = np.einsum("asc,asd->cd", x.z2, T)                    # k2x x k2y
    return float(np.sum((W @ y.z3) * x.z3))


def kron_apply(X1, X2, X3, z):
    """(X1 kron X2 kron X3) vec z as a TT with z's ranks (eq. Xz).

    X1 (n_t' x n_t), X2 (n_xi' x n_xi), X3 (n_x' x n_x), each dense or sparse;
    None means the identity.
    """
    z1 = z.z1 if X1 is None else np.asarray(X1 @ z.z1)
    z2 = z.z2 if X2 is None else np.einsum("rs,asb->arb", np.asarray(X2.todense() if sp.issparse(X2) else X2), z.z2)
    z3 = z.z3 if X3 is None else np.asarray((X3 @ z.z3.T).T)
    return TT(z1, z2, z3)


def _trunc_rank(s, delta):
    """Smallest r >= 1 with sum_{i > r} s_i^2 <= delta^2."""
    tail = np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]])   # tail[r] = sum_{i>=r} s_i^2
    for r in range(1, len(s) + 1):
        if tail[r] <= delta * delta:
            return r
    return len(s)


def round_tt(z, eps):
    """T_eps(z) for a TT (Section 4.1): right-to-left QR orthogonalisation, then
    left-to-right truncated SVDs with delta = eps ||z|| / sqrt(2).

    Returns (rounded TT, ||z||_F).  eps <= 0 keeps every nonzero singular value.
    """
    n_t, n_xi, n_x = z.shape
    k1, k2 = z.ranks
    # right-to-left orthogonalisation: z3^T = Q3 R3, z3 <- Q3^T, z2 <- z2 x3 R3
    Q3, R3 = np.linalg.qr(z.z3.T)                   # n_x x c3, c3 x k2
    c3 = Q3.shape[1]
    z2 = np.einsum("asb,cb->asc", z.z2, R3)          # k1 x n_xi x c3
    # z2 right unfolding (k1 x n_xi c3) = R2^T Q2^T
    Q2, R2 = np.linalg.qr(z2.reshape(k1, n_xi * c3).T)   # (n_xi c3) x c2, c2 x k1
    c2 = Q2.shape[1]
    core2 = Q2.T.reshape(c2, n_xi, c3)
    core1 = z.z1 @ R2.T                              # n_t x c2
    nrm = float(np.linalg.norm(core1))
    if nrm == 0.0:
        return TT.zeros(n_t, n_xi, n_x), 0.0
    delta = eps * nrm / np.sqrt(2.0) if eps > 0 else 0.0
    # left-to-right truncated SVDs (Algorithm 4.1 on the orthogonalised train)
    U, s, Vt = np.linalg.svd(core1, full_matrices=False)
    r1 = _trunc_rank(s, delta) if eps > 0 else max(1, int((s > 0).sum()))
    new1 = U[:, :r1]
    core2 = np.einsum("ab,bsc->asc", s[:r1, None] * Vt[:r1], core2)    # r1 x n_xi x c3
    U, s, Vt = np.linalg.svd(core2.reshape(r1 * n_xi, c3), full_matrices=False)
    r2 = _trunc_rank(s, delta) if eps > 0 else max(1, int((s > 0).sum()))
    new2 = U[:, :r2].reshape(r1, n_xi, r2)
    new3 = (s[:r2, None] * Vt[:r2]) @ Q3.T           # r2 x n_x
    return TT(new1, new2, new3), nrm


def truncate(z, eps):
    """(T_eps(z), ||z||, ||T_eps(z)||); the last is the 2-norm of the kept singular
    values of the second unfolding (the new first two cores are orthonormal)."""
    r, before = round_tt(z, eps)
    return r, before, float(np.linalg.norm(r.z3))


def norm(z):
    """||vec z|| from the orthogonalised train (no cancellation, unlike sqrt(dot(z, z)))."""
    return round_tt(z, 0.0)[1]


def tt_svd(Z, eps):
    """Algorithm 4.1 (TT-SVD) of a full n1 x n2 x n3 tensor with delta_j = eps ||Z|| / sqrt 2."""
    n1, n2, n3 = Z.shape
    delta = eps * np.linalg.norm(Z) / np.sqrt(2.0)
    cores = []
    r_prev = 1
    W = Z.copy()
    for (nj, rest) in ((n1, n2 * n3), (n2, n3)):
        W = W.reshape(r_prev * nj, -1)
        U, s, Vt = np.linalg.svd(W, full_matrices=False)
        r = _trunc_rank(s, delta)
        cores.append(U[:, :r].reshape(r_prev, nj, r))
        W = s[:r, None] * Vt[:r]
        r_prev = r
    z1 = cores[0].reshape(n1, -1)
    return TT(z1, cores[1], W)


def pair_add(*terms):
    """Sum of (coef, (u TT, p TT)) pairs, each block concatenated separately."""
    u = add(*[(c, v[0]) for c, v in terms])
    p = add(*[(c, v[1]) for c, v in terms])
    return (u, p)


def pair_round(v, eps):
    """Truncate the velocity and pressure trains separately (Section 4.2)."""
    u, nu = round_tt(v[0], eps)
    p, np_ = round_tt(v[1], eps)
    return (u, p), float(np.hypot(nu, np_))


def pair_dot(a, b):
    return dot(a[0], b[0]) + dot(a[1], b[1])


def pair_scale(v, c):
    return (v[0].scale(c), v[1].scale(c))
