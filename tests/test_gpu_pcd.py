"""The mean-based PCD preconditioner (eq. mean_pcd, Section 5.2) on the GPU against
the oracle: the Q1 pressure-space matrices, the preconditioner applied once (PCD
Schur part to rounding, the inner solve to its tight tolerance) and whole Picard
solves with the PCD Schur approximation."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import fem
from oracle import tt as otm
from oracle.solver import MeanPCD, picard as opicard
from oracle.system import Discretisation

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1906_06785_gb300 import binding
    return binding.Context()


@pytest.fixture(scope="module")
def small():
    prob = synth.preset("small")
    return prob, Discretisation(prob)


def _tt_diff(a, b):
    return otm.norm(otm.add((1.0, a), (-1.0, b))) / otm.norm(b)


def test_pressure_matrices_match(ctx, small):
    prob, d = small
    P = ctx.problem(prob)

    def csr(which):
        rp, cl, v, shape = P.matrix(which, 0)
        return sp.csr_matrix((v, cl, rp), shape=shape)

    Mp, Ap, _ = d.pressure_matrices()
    for which, ref in ((200, Mp), (201, Ap)):
        got = csr(which)
        assert got.shape == ref.shape
        assert abs(got - ref).max() <= 1e-13 * abs(ref).max()


def test_pcd_preconditioner_matches(ctx):
    """PCD Schur part to rounding; the inner solve, identical to the LSC one, to its
    tight inner tolerance (tiny problem: the oracle's inner solve at 1e-9 is slow)."""
    from paper_1906_06785_gb300 import binding
    prob = synth.preset("tiny")
    d = Discretisation(prob)
    P = ctx.problem(prob)
    u = otm.TT(*synth.random_tt(d.n_t, d.n_xi, d.n_u, 2, 3, seed=181))
    p = otm.TT(*synth.random_tt(d.n_t, d.n_xi, d.n_p, 2, 2, seed=182))
    gu, gp = ctx.tt(u.z1, u.z2, u.z3), ctx.tt(p.z1, p.z2, p.z3)
    w = d.full_velocity(otm.TT(*synth.random_tt(d.n_t, d.n_xi, d.n_u, 2, 2, seed=191)).scale(0.3))
    op = P.op(ctx.tt(w.z1, w.z2, w.z3))
    eps, tol_in = 1e-12, 1e-9
    gu2, gp2, its, fb = op.prec(gu, gp, eps, tol_in, 40, kind=binding.PREC_PCD)
    ou, opp = MeanPCD(d, w, eps, tol_in, 40)((u, p))
    assert _tt_diff(otm.TT(*gp2.cores()), opp) < 1e-10
    assert _tt_diff(otm.TT(*gu2.cores()), ou) < 1e-8


def test_picard_with_pcd_matches_the_oracle(ctx):
    """Algorithm 3.1 with the PCD Schur approximation on the tiny problem at tight
    tolerances: same Picard and GMRES counts as the oracle, same solution."""
    from paper_1906_06785_gb300 import binding
    prob = synth.preset("tiny")
    prob.tol.eps_gmres, prob.tol.eps_soln, prob.tol.eps_conv = 1e-8, 1e-10, 1e-8
    d = Discretisation(prob)
    P = ctx.problem(prob)
    u, p, st, code = P.picard(binding.opts_from(prob.tol, schur=binding.PREC_PCD))
    assert code == binding.TT_OK
    ou, op_, ost = opicard(d, schur="pcd")
    assert st.picard_its == ost["picard_its"]
    assert list(st.gmres_its[1:st.picard_its + 1]) == ost["gmres_its"]
    assert _tt_diff(otm.TT(*u.cores()), ou) < 1e-6
    assert _tt_diff(otm.TT(*p.cores()), op_) < 1e-6
