"""Algorithm-level pins: the truncated TT-GMRES / Picard iteration against the
definition-level sparse direct Picard solve of the uncompressed system."""
import numpy as np
import pytest

import synth
from oracle.solver import direct_picard, picard
from oracle.system import Discretisation


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_tight_tt_picard_matches_direct_solve():
    """With truncation tolerances near roundoff and tight stopping tests the
    low-rank solver reproduces the sparse direct Picard solution."""
    prob = synth.preset("tiny")
    t = prob.tol
    t.tol_picard, t.tol_gmres, t.tol_inner = 1e-11, 1e-4, 1e-4
    t.eps_gmres, t.eps_soln, t.eps_conv = 1e-13, 1e-14, 1e-13
    d = Discretisation(prob)
    uf, pf, _ = direct_picard(d, tol=1e-13)
    u, p, st = picard(d)
    assert st["res"][-1] <= 1e-11 * st["fnorm"]
    assert _rel(u.full(), uf) < 1e-8
    assert _rel(p.full(), pf) < 1e-8


def test_default_tolerances_converge_like_the_paper():
    """Table 5.2 tolerances: inexact Picard reaches ||r|| <= 1e-5 ||f|| in a handful
    of steps with few GMRES iterations each (Section 5.3), and the result is
    within the stopping tolerance's reach of the direct solution."""
    prob = synth.preset("tiny")
    prob.tol.eps_gmres, prob.tol.eps_soln, prob.tol.eps_conv = 1e-3, 1e-7, 1e-3
    d = Discretisation(prob)
    uf, pf, _ = direct_picard(d, tol=1e-13)
    u, p, st = picard(d)
    assert st["res"][-1] <= 1e-5 * st["fnorm"]
    assert 2 <= st["picard_its"] <= 10
    assert max(st["gmres_its"]) <= 8
    # linear convergence of inexact Picard (Fig. 5.2b): residuals decrease
    assert all(b < a for a, b in zip(st["res"], st["res"][1:]))
    assert _rel(u.full(), uf) < 1e-3
