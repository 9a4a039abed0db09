"""GPU parity: every step of the hot path through the C ABI against the CPU oracle.

Tolerances (FP64 on both sides, different summation orders):
  * assembled matrices, Kronecker products, dots, concatenation: 1e-12 relative
    (a handful of FP64 roundings per entry);
  * truncation: the truncated tensor is a function of the tensor alone, so the
    GPU and oracle results must agree to within the truncation tolerance of the
    discarded part plus roundoff; inputs are built with spectra that keep every
    singular value away from the cut, so ranks match exactly and tensors agree
    to 1e-10 relative;
  * end-to-end Picard solves: 1e-6 relative (the FP64 target of the method).
"""
import numpy as np
import pytest
import scipy.sparse as sp

from ttfull import full

import synth
from oracle import tt as otm
from oracle.system import Discretisation
from oracle.solver import MeanLSC, picard as oracle_picard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1906_06785_gb300 import binding
    return binding.Context()


@pytest.fixture(scope="module")
def tiny():
    prob = synth.preset("tiny")
    return prob, Discretisation(prob)


@pytest.fixture(scope="module")
def small():
    prob = synth.preset("small")
    return prob, Discretisation(prob)


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _oracle_tt(h):
    return otm.TT(*h.cores())


def _tt_diff(a, b):
    """||a - b|| / ||b|| for oracle trains via concatenation + orthogonalisation."""
    return otm.norm(otm.add((1.0, a), (-1.0, b))) / otm.norm(b)


# ------------------------------------------------------------------ trains
def test_create_and_read_back(ctx):
    z = synth.random_tt(7, 5, 33, 3, 4, seed=1)
    t = ctx.tt(*z)
    for a, b in zip(t.cores(), z):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("shape", [(4, 3, 10, 1, 1), (9, 6, 257, 5, 7), (20, 6, 1312, 12, 40)])
def test_dot_and_axpby(ctx, shape):
    n_t, n_xi, n_x, r1, r2 = shape
    za = synth.random_tt(n_t, n_xi, n_x, r1, r2, seed=2)
    zb = synth.random_tt(n_t, n_xi, n_x, r2 % 5 + 1, r1 + 2, seed=3)
    a, b = ctx.tt(*za), ctx.tt(*zb)
    oa, ob = otm.TT(*za), otm.TT(*zb)
    assert abs(ctx.dot(a, b) - otm.dot(oa, ob)) <= 1e-12 * otm.norm(oa) * otm.norm(ob)
    s = ctx.axpby(0.3, a, -1.7, b)
    ref = otm.add((0.3, oa), (-1.7, ob))
    assert s.ranks == ref.ranks
    assert _rel(full(s), ref.full()) < 1e-14


# ------------------------------------------------------------------ truncation
@pytest.mark.parametrize("shape,eps", [
    ((6, 4, 30, 5, 8), 1e-3),        # tiny, one CTA
    ((20, 6, 1312, 20, 60), 1e-6),   # several row blocks, ragged tail
    ((100, 20, 5440, 30, 90), 1e-5), # medium-sized velocity train
    ((11, 3, 40, 9, 120), 1e-8),     # wide: n_x < pre-rounding rank
    ((40, 6, 1500, 40, 240), 1e-6),  # first rank above n_t; 150-column SVDs
    ((24, 20, 1200, 24, 300), 1e-6), # 320 x 301 SVD: 16 lanes x 32 entries per pair
])
def test_round_matches_oracle(ctx, shape, eps):
    n_t, n_xi, n_x, r1, r2 = shape
    # sum of two trains with decaying spectra: ranks add, truncation has work to do;
    # when the pre-rounding rank exceeds n_x (wide case) plain Gaussian cores are used
    dec = 10 if r2 // 2 + 1 <= n_x else None
    z = otm.add((1.0, otm.TT(*synth.random_tt(n_t, n_xi, n_x, r1 // 2 + 1, r2 // 2 + 1, seed=5, decay=dec))),
                (0.5, otm.TT(*synth.random_tt(n_t, n_xi, n_x, r1 // 2, r2 // 2, seed=6, decay=dec))))
    t = ctx.tt(z.z1, z.z2, z.z3)
    g, nb, na = ctx.round(t, eps)
    ref, nref = otm.round_tt(z, eps)
    assert abs(nb - nref) <= 1e-12 * nref
    og = _oracle_tt(g)
    assert g.ranks == ref.ranks
    # the library's Jacobi stops at column orthogonality jtol = 1e-3 eps (clamped to
    # [1e-13, 1e-8]) on the R-factor route: frames and tensor agree to that level
    jtol = min(1e-8, max(1e-13, 1e-3 * eps))
    tol = max(1e-10, 10 * jtol)
    assert _tt_diff(og, ref) < tol
    assert otm.norm(otm.add((1.0, og), (-1.0, z))) <= eps * nref * (1 + 1e-6)
    assert abs(na - otm.norm(ref)) <= tol * nref
    # new first and second cores are orthonormal frames
    z1, z2, _ = g.cores()
    assert np.abs(z1.T @ z1 - np.eye(z1.shape[1])).max() < max(1e-12, 10 * jtol)
    G = z2.reshape(-1, z2.shape[2])
    assert np.abs(G.T @ G - np.eye(G.shape[1])).max() < max(1e-12, 10 * jtol)


def test_round_zero_and_rank_one(ctx):
    z = ctx.tt(np.zeros((5, 2)), np.zeros((2, 3, 2)), np.zeros((2, 9)))
    g, nb, na = ctx.round(z, 1e-3)
    assert nb == 0.0 and g.ranks == (1, 1) and not full(g).any()
    one = ctx.tt(*synth.random_tt(5, 3, 9, 1, 1, seed=9))
    g, nb, _ = ctx.round(one, 1e-12)
    assert g.ranks == (1, 1) and _rel(full(g), full(one)) < 1e-14


def test_round_keeps_everything_at_eps_zero(ctx):
    z = synth.random_tt(8, 3, 50, 4, 6, seed=11)
    g, nb, na = ctx.round(ctx.tt(*z), 0.0)
    assert _rel(full(g), otm.TT(*z).full()) < 1e-13
    assert abs(nb - na) < 1e-13 * nb


# ------------------------------------------------------------------ discretisation
@pytest.mark.parametrize("name", ["tiny", "small"])
def test_assembled_matrices_match(ctx, name, tiny, small):
    prob, d = {"tiny": tiny, "small": small}[name]
    P = ctx.problem(prob)
    sz = P.sizes()
    assert (sz["n_u"], sz["n_p"]) == (d.n_u, d.n_p)

    def csr(which, block):
        rp, cl, v, shape = P.matrix(which, block)
        return sp.csr_matrix((v, cl, rp), shape=shape)

    for which, ref_f, ref_d in [(0, d.M, d.MfD)] + [(1 + l, d.A[l], d.AfD[l]) for l in range(prob.m + 1)]:
        for block, ref in ((0, ref_f), (1, ref_d)):
            got = csr(which, block)
            assert abs(got - ref).max() <= 1e-13 * abs(ref).max()
    Bx = d.Bxfull[:, d.free]
    By = d.Byfull[:, d.free]
    assert abs(csr(100, 0) - Bx).max() < 1e-13
    assert abs(csr(101, 0) - By).max() < 1e-13
    assert abs(csr(100, 1) - d.Bxfull[:, d.dn]).max() < 1e-13


def _pair(ctx, d, seed, r=(2, 3)):
    u = otm.TT(*synth.random_tt(d.n_t, d.n_xi, d.n_u, r[0], r[1], seed=seed))
    p = otm.TT(*synth.random_tt(d.n_t, d.n_xi, d.n_p, 2, 2, seed=seed + 1))
    return u, p, ctx.tt(u.z1, u.z2, u.z3), ctx.tt(p.z1, p.z2, p.z3)


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_rhs_and_lifting(ctx, name, tiny, small):
    prob, d = {"tiny": tiny, "small": small}[name]
    P = ctx.problem(prob)
    fu, fp = P.rhs()
    rfu, rfp = d.rhs()
    assert _rel(full(fu), rfu.full()) < 1e-12
    assert _rel(full(fp), rfp.full()) < 1e-12
    u, _, gu, _ = _pair(ctx, d, 21)
    w = P.full_velocity(gu)
    assert _rel(full(w), d.full_velocity(u).full()) < 1e-14


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_full_operator_matches(ctx, name, tiny, small):
    prob, d = {"tiny": tiny, "small": small}[name]
    P = ctx.problem(prob)
    u, p, gu, gp = _pair(ctx, d, 31)
    wu = otm.TT(*synth.random_tt(d.n_t, d.n_xi, d.n_u, 2, 3, seed=41))
    w = d.full_velocity(wu)
    gw = ctx.tt(w.z1, w.z2, w.z3)
    for conv in (None, (w, gw)):
        op = P.op(conv[1] if conv else None)
        ou, op_ = op.matvec(gu, gp)
        ru, rp = d.apply(conv[0] if conv else None, u, p)
        assert _tt_diff(_oracle_tt(ou), ru) < 1e-12
        assert _tt_diff(_oracle_tt(op_), rp) < 1e-12


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_mean_operator_matches(ctx, name, tiny, small):
    from paper_1906_06785_gb300 import binding
    prob, d = {"tiny": tiny, "small": small}[name]
    P = ctx.problem(prob)
    u, p, gu, gp = _pair(ctx, d, 51)
    w = d.full_velocity(otm.TT(*synth.random_tt(d.n_t, d.n_xi, d.n_u, 2, 2, seed=61)))
    op = P.op(ctx.tt(w.z1, w.z2, w.z3), which=binding.OP_MEAN)
    got = op.matvec(gu)
    assert _tt_diff(_oracle_tt(got), d.apply_mean(w, u)) < 1e-12


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_residual_matches(ctx, name, tiny, small):
    prob, d = {"tiny": tiny, "small": small}[name]
    P = ctx.problem(prob)
    u, p, gu, gp = _pair(ctx, d, 71)
    ru, rp, rn = P.residual(gu, gp, 1e-10)
    (oru, orp), orn = d.residual(u, p, 1e-10)
    assert abs(rn - orn) <= 1e-9 * orn
    assert _tt_diff(_oracle_tt(ru), oru) < 1e-9
    assert _tt_diff(_oracle_tt(rp), orp) < 1e-9


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_preconditioner_matches(ctx, name, tiny, small):
    """LSC Schur part exactly; the inner solve with a tight inner tolerance so that
    both sides run the same number of inner iterations to the same answer."""
    prob, d = {"tiny": tiny, "small": small}[name]
    P = ctx.problem(prob)
    u, p, gu, gp = _pair(ctx, d, 81)
    w = d.full_velocity(otm.TT(*synth.random_tt(d.n_t, d.n_xi, d.n_u, 2, 2, seed=91)).scale(0.3))
    op = P.op(ctx.tt(w.z1, w.z2, w.z3))
    eps, tol_in = 1e-12, 1e-9
    gu2, gp2, its, fb = op.prec(gu, gp, eps, tol_in, 40)
    assert fb == 0
    pre = MeanLSC(d, w, eps, tol_in, 40)
    ou, opp = pre((u, p))
    assert _tt_diff(_oracle_tt(gp2), opp) < 1e-10
    assert _tt_diff(_oracle_tt(gu2), ou) < 1e-8


def test_gmres_matches(ctx, tiny):
    from paper_1906_06785_gb300 import binding
    prob, d = tiny
    P = ctx.problem(prob)
    fu, fp = P.rhs()
    op = P.op(None)
    o = binding.opts_from(prob.tol, tol_gmres=1e-8, eps_gmres=1e-12, tol_inner=1e-3)
    zu, zp, st, code = op.gmres(o, fu, fp)
    from oracle.solver import gmres, _Pair
    t = prob.tol
    pre = MeanLSC(d, None, 1e-12, 1e-3, t.maxit_inner)
    (ou, opp), ost = gmres(lambda v: d.apply(None, *v), pre, d.rhs(), tol=1e-8, eps=1e-12,
                           maxit=t.maxit_gmres, space=_Pair)
    assert code == binding.TT_OK
    assert st.its == ost["its"]
    assert _rel(full(zu), ou.full()) < 1e-8
    assert _rel(full(zp), opp.full()) < 1e-8


# ------------------------------------------------------------------ end to end
def _picard_pair(ctx, prob):
    from paper_1906_06785_gb300 import binding
    P = ctx.problem(prob)
    u, p, st, code = P.picard(binding.opts_from(prob.tol))
    ou, op_, ost = oracle_picard(Discretisation(prob))
    return u, p, st, code, ou, op_, ost


def test_picard_tiny_tight(ctx):
    prob = synth.preset("tiny")
    t = prob.tol
    t.tol_picard, t.tol_gmres, t.tol_inner = 1e-10, 1e-4, 1e-4
    t.eps_gmres, t.eps_soln, t.eps_conv = 1e-12, 1e-13, 1e-12
    u, p, st, code, ou, op_, ost = _picard_pair(ctx, prob)
    assert code == 0 and st.picard_its == ost["picard_its"]
    assert _rel(full(u), ou.full()) < 1e-8
    assert _rel(full(p), op_.full()) < 1e-8


def test_picard_tiny_default_tolerances(ctx):
    prob = synth.preset("tiny")
    prob.tol.eps_gmres, prob.tol.eps_soln, prob.tol.eps_conv = 1e-3, 1e-7, 1e-3
    u, p, st, code, ou, op_, ost = _picard_pair(ctx, prob)
    assert code == 0
    assert st.picard_its == ost["picard_its"]
    assert list(st.gmres_its[1:st.picard_its + 1]) == ost["gmres_its"]
    assert _rel(full(u), ou.full()) < 1e-6
    assert _rel(full(p), op_.full()) < 1e-6
    assert st.res[st.picard_its] <= prob.tol.tol_picard * st.fnorm


@pytest.mark.parametrize("eps", [1e-5, 1e-3])
def test_round_gram_route_and_first_core_compression(ctx, eps):
    """Tolerances >= 5e-6 take the Gram route; first ranks above n_t are compressed
    first.  Both give T_eps of the same tensor: equal ranks (spectra with gaps at
    the cut) and a TT difference far below the truncation tolerance."""
    n_t, n_xi, n_x = 12, 5, 700
    a = otm.TT(*synth.random_tt(n_t, n_xi, n_x, 10, 40, seed=31, decay=9))
    b = otm.TT(*synth.random_tt(n_t, n_xi, n_x, 10, 40, seed=32, decay=9))
    z = otm.add((1.0, a), (0.6, b))          # first rank 20 > n_t = 12
    g, nb, na = ctx.round(ctx.tt(z.z1, z.z2, z.z3), eps)
    ref, nref = otm.round_tt(z, eps)
    assert g.ranks == ref.ranks
    assert abs(nb - nref) < 1e-12 * nref
    assert _tt_diff(_oracle_tt(g), ref) < 1e-8
    assert otm.norm(otm.add((1.0, _oracle_tt(g)), (-1.0, z))) <= eps * nref * (1 + 1e-6)


@pytest.mark.parametrize("eps", [1e-5, 1e-3])
def test_round_gram_route_on_the_smaller_gram_side(ctx, eps):
    """Gram route with r1 n_xi far above R2 (2 R2^3 < (r1 n_xi)^3): the second unfolding's
    singular pairs come from the R2 x R2 Gram matrix B^T B.  Same T_eps as the oracle's."""
    n_t, n_xi, n_x = 12, 20, 700
    a = otm.TT(*synth.random_tt(n_t, n_xi, n_x, 10, 40, seed=33, decay=9))
    b = otm.TT(*synth.random_tt(n_t, n_xi, n_x, 10, 40, seed=34, decay=9))
    z = otm.add((1.0, a), (0.6, b))
    g, nb, na = ctx.round(ctx.tt(z.z1, z.z2, z.z3), eps)
    ref, nref = otm.round_tt(z, eps)
    assert g.ranks == ref.ranks
    assert 2 * 80 ** 3 < (g.ranks[0] * n_xi) ** 3
    assert abs(nb - nref) < 1e-12 * nref
    assert _tt_diff(_oracle_tt(g), ref) < 1e-8
    assert otm.norm(otm.add((1.0, _oracle_tt(g)), (-1.0, z))) <= eps * nref * (1 + 1e-6)
