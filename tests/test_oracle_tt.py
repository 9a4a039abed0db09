"""Pins of the oracle's tensor-train algebra (Section 4.1) against dense arithmetic."""
import numpy as np
import pytest

import synth
from oracle.tt import TT, add, dot, kron_apply, round_tt, truncate, tt_svd, norm


def _tt(n_t=5, n_xi=4, n_x=7, r1=3, r2=4, seed=0):
    return TT(*synth.random_tt(n_t, n_xi, n_x, r1, r2, seed=seed))


def test_full_tensor_index_map():
    """z(i1,i2,i3) = sum z1 z2 z3 (eq. z_tt) and vec runs i3 fastest (Section 4.1)."""
    z = _tt()
    Z = z.full()
    i1, i2, i3 = 3, 2, 5
    v = sum(z.z1[i1, a] * z.z2[a, i2, b] * z.z3[b, i3] for a in range(3) for b in range(4))
    assert abs(Z[i1, i2, i3] - v) < 1e-12
    n_x, n_xi = 7, 4
    assert z.vec()[i3 + i2 * n_x + i1 * n_xi * n_x] == Z[i1, i2, i3]


def test_kron_matvec_matches_dense_kron():
    """eq. (Xz): (X1 (x) X2 (x) X3) vec z equals the TT with each core multiplied."""
    rng = np.random.default_rng(1)
    z = _tt(seed=1)
    X1, X2, X3 = rng.standard_normal((6, 5)), rng.standard_normal((4, 4)), rng.standard_normal((3, 7))
    y = kron_apply(X1, X2, X3, z)
    assert y.ranks == z.ranks
    ref = np.kron(np.kron(X1, X2), X3) @ z.vec()
    assert np.abs(y.vec() - ref).max() < 1e-11


def test_add_dot_norm_match_dense():
    a, b = _tt(seed=2), _tt(r1=2, r2=5, seed=3)
    s = add((0.7, a), (-1.3, b))
    assert s.ranks == (5, 9)
    assert np.abs(s.vec() - (0.7 * a.vec() - 1.3 * b.vec())).max() < 1e-12
    assert abs(dot(a, b) - a.vec() @ b.vec()) < 1e-10
    assert abs(norm(s) - np.linalg.norm(s.vec())) < 1e-12


def test_norm_of_cancelled_sum_is_accurate():
    """||z - (z - e)|| via orthogonalisation is accurate where dot() would cancel."""
    z = _tt(seed=4)
    e = _tt(seed=5).scale(1e-9)
    d = add((1.0, z), (-1.0, add((1.0, z), (-1.0, e))))
    assert abs(norm(d) - np.linalg.norm(e.vec())) < 1e-6 * np.linalg.norm(e.vec())


@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-6, 1e-10])
def test_round_error_bound(eps):
    """||T_eps(z) - z|| <= eps ||z|| (Section 4.1) on a train with a decaying spectrum."""
    z = TT(*synth.random_tt(8, 5, 30, 6, 10, seed=7, decay=8))
    z = add((1.0, z), (0.5, TT(*synth.random_tt(8, 5, 30, 6, 10, seed=8, decay=8))))
    r, nz = round_tt(z, eps)
    err = np.linalg.norm(r.vec() - z.vec())
    assert abs(nz - np.linalg.norm(z.vec())) < 1e-12 * nz
    assert err <= eps * nz * (1 + 1e-10)
    # cores 1 and 2 of the result are orthonormal frames
    assert np.abs(r.z1.T @ r.z1 - np.eye(r.ranks[0])).max() < 1e-12
    G = r.z2.reshape(-1, r.ranks[1])
    assert np.abs(G.T @ G - np.eye(r.ranks[1])).max() < 1e-12


def test_round_of_doubled_train_keeps_its_rank():
    """T(z + z) has the ranks of z and equals 2z (ranks add before truncation)."""
    z = _tt(n_t=9, n_xi=6, n_x=20, r1=3, r2=4, seed=9)
    zz = add((1.0, z), (1.0, z))
    assert zz.ranks == (6, 8)
    r, _ = round_tt(zz, 1e-12)
    assert r.ranks == (3, 4)
    assert np.abs(r.vec() - 2 * z.vec()).max() < 1e-10


def test_round_equals_tt_svd_of_full_tensor():
    """Rounding a TT and TT-SVD (Algorithm 4.1) of its full tensor agree: same ranks,
    same tensor (the truncated SVDs depend only on the tensor)."""
    z = TT(*synth.random_tt(10, 6, 25, 7, 9, seed=11, decay=6))
    Z = z.full()
    for eps in (1e-2, 1e-4):
        a, _ = round_tt(z, eps)
        b = tt_svd(Z, eps)
        assert a.ranks == b.ranks
        assert np.abs(a.vec() - b.vec()).max() < 1e-10 * np.abs(Z).max()
        assert np.linalg.norm(b.vec() - Z.ravel()) <= eps * np.linalg.norm(Z) * (1 + 1e-10)


def test_truncation_rank_from_known_spectrum():
    """Orthonormal frames with singular values s_i on both unfoldings: the rank is
    the smallest r with sum_{i>r} s_i^2 <= (eps ||z|| / sqrt 2)^2."""
    n_t, n_xi, n_x, r = 12, 1, 40, 8
    rng = np.random.default_rng(3)
    s = 10.0 ** -np.arange(r)
    U, _ = np.linalg.qr(rng.standard_normal((n_t, r)))
    V, _ = np.linalg.qr(rng.standard_normal((n_x, r)))
    z = TT(U * s, np.eye(r).reshape(r, 1, r), V.T)
    nrm = np.linalg.norm(s)
    for eps in (2e-3, 2e-5):
        delta = eps * nrm / np.sqrt(2)
        tail = np.array([np.sqrt((s[k:] ** 2).sum()) for k in range(r + 1)])
        expect = int(np.argmax(tail <= delta))
        rr, _ = round_tt(z, eps)
        assert rr.ranks == (expect, expect)


def test_truncate_reports_norms():
    z = TT(*synth.random_tt(6, 4, 15, 4, 5, seed=13, decay=5))
    r, before, after = truncate(z, 1e-2)
    assert abs(before - np.linalg.norm(z.vec())) < 1e-12 * before
    assert abs(after - np.linalg.norm(r.vec())) < 1e-12 * before


def test_zero_train_rounds_to_rank_one_zero():
    z = TT(np.zeros((4, 2)), np.zeros((2, 3, 2)), np.zeros((2, 5)))
    r, n = round_tt(z, 1e-3)
    assert n == 0.0 and r.ranks == (1, 1) and not r.vec().any()
