"""Randomized truncation (tt_round_randomized, and rounding=TT_ROUND_RANDOMIZED in the
solver) against the deterministic T_eps of the oracle: the error bound
||T(z) - z|| <= eps ||z|| measured exactly by the oracle (concatenation and
orthogonalisation), ranks within the rank-decision noise of the deterministic ones,
and whole solves within the mixed-precision tolerance 1e-4 of the oracle's."""
import os

import numpy as np
import pytest

import synth
from oracle import tt as otm

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ctx():
    from paper_1906_06785_gb300 import binding
    return binding.Context()


def _wide_sum(n_t, n_xi, n_x, parts, r1, r2, seed, decay=16):
    """A sum of `parts` trains with graded spectra: second rank parts * r2 (like a Krylov
    sum or a matvec output), numerical rank far lower."""
    z = None
    for k in range(parts):
        t = otm.TT(*synth.random_tt(n_t, n_xi, n_x, r1, r2, seed=seed + k, decay=decay))
        z = t if z is None else otm.add((1.0, z), (0.5 ** k, t))
    return z


def _err(g, z):
    return otm.norm(otm.add((1.0, otm.TT(*g.cores())), (-1.0, z)))


@pytest.mark.parametrize("eps", [1e-5, 1e-3])
def test_randomized_truncation_meets_the_bound(ctx, eps):
    z = _wide_sum(20, 20, 1500, 4, 5, 100, seed=61)
    assert z.ranks[1] == 400
    t = ctx.tt(z.z1, z.z2, z.z3)
    nz = otm.norm(z)
    g, nb, na, ell = ctx.round_randomized(t, eps, seed=7)
    assert ell < 400                                      # the sketch path was taken
    assert _err(g, z) <= eps * nz * (1 + 1e-6)
    assert abs(nb - nz) <= 1e-6 * nz
    ref, _ = otm.round_tt(z, eps)
    assert abs(g.ranks[0] - ref.ranks[0]) <= 2 and abs(g.ranks[1] - ref.ranks[1]) <= 3
    # deterministic in its seed
    g2, _, _, _ = ctx.round_randomized(t, eps, seed=7)
    assert _err(g2, otm.TT(*g.cores())) <= 1e-12 * nz


def test_small_second_rank_takes_the_deterministic_route(ctx):
    z = otm.TT(*synth.random_tt(10, 8, 300, 6, 40, seed=62, decay=6))
    t = ctx.tt(z.z1, z.z2, z.z3)
    g, nb, na, ell = ctx.round_randomized(t, 1e-4, seed=3)
    d, nb2, na2 = ctx.round(t, 1e-4)
    assert ell == 40 and g.ranks == d.ranks
    assert _err(g, otm.TT(*d.cores())) <= 1e-14 * otm.norm(z)


@pytest.mark.parametrize("precision", [0, 1])
def test_small_picard_with_randomized_truncation(ctx, precision):
    from paper_1906_06785_gb300 import binding
    prob = synth.preset("small")
    P = ctx.problem(prob)
    u, p, st, code = P.picard(binding.opts_from(prob.tol, precision=precision,
                                                rounding=binding.ROUND_RANDOMIZED))
    assert code == binding.TT_OK
    assert st.res[st.picard_its] <= prob.tol.tol_picard * st.fnorm
    c = np.load(os.path.join(GOLD, "picard_small_cores.npz"))
    for h, k in ((u, "u"), (p, "p")):
        ref = otm.TT(c[k + "1"], c[k + "2"], c[k + "3"])
        assert _err(h, ref) <= 1e-4 * otm.norm(ref)


def test_medium_stokes_with_randomized_truncation(ctx):
    from paper_1906_06785_gb300 import binding
    c = np.load(os.path.join(GOLD, "stokes_medium.npz"))
    prob = synth.preset("medium")
    P = ctx.problem(prob)
    fu, fp = P.rhs()
    o = binding.opts_from(prob.tol, precision=binding.MIXED, rounding=binding.ROUND_RANDOMIZED)
    u, p, st, code = P.op(None).gmres(o, fu, fp, float(c["fnorm"]))
    assert code == binding.TT_OK and st.its == int(c["its"])
    # the tolerance of the mixed-precision Stokes iterate (see test_gpu_solve.py)
    for h, k in ((u, "u"), (p, "p")):
        ref = otm.TT(c[k + "1"], c[k + "2"], c[k + "3"])
        assert _err(h, ref) <= 1e-3 * otm.norm(ref)
