"""The allocation-free inner product (tt_dot_noalloc) against tt_dot, through the
C ABI.  Collected last so that it also runs after every other GPU test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _train(ctx, rng, n_t, n_xi, n_x, r1, r2):
    z1 = rng.standard_normal((n_t, r1))
    z2 = rng.standard_normal((r1, n_xi, r2)) / np.sqrt(r1)
    z3 = rng.standard_normal((r2, n_x)) / np.sqrt(r2)
    return ctx.tt(z1, z2, z3), (z1, z2, z3)


@pytest.fixture(scope="module")
def ctx():
    from paper_1906_06785_gb300 import binding
    return binding.Context()


@pytest.mark.parametrize("shape,ra,rb", [
    ((20, 6, 1521), (13, 49), (14, 57)),      # small-problem ranks
    ((100, 20, 6209), (40, 300), (26, 275)),  # medium-problem ranks, split-K in the scratch
    ((5, 3, 37), (1, 1), (4, 2)),             # ragged tiny case
])
def test_dot_noalloc_matches_dot_on_two_calls_in_a_row(ctx, shape, ra, rb):
    rng = np.random.default_rng(2024)
    a, _ = _train(ctx, rng, *shape, *ra)
    b, _ = _train(ctx, rng, *shape, *rb)
    ref_ab, ref_aa, ref_bb = ctx.dot(a, b), ctx.dot(a, a), ctx.dot(b, b)
    scale = np.sqrt(ref_aa * ref_bb)
    for _ in range(2):
        assert abs(ctx.dot_noalloc(a, b) - ref_ab) <= 1e-12 * scale
        assert abs(ctx.dot_noalloc(a, a) - ref_aa) <= 1e-12 * ref_aa
        assert abs(ctx.dot_noalloc(b, a) - ref_ab) <= 1e-12 * scale


def test_dot_noalloc_matches_the_full_contraction(ctx):
    rng = np.random.default_rng(7)
    a, ca = _train(ctx, rng, 6, 4, 50, 3, 5)
    b, cb = _train(ctx, rng, 6, 4, 50, 2, 7)
    full = lambda c: np.einsum("ia,ajb,bk->ijk", *c)
    want = float(np.sum(full(ca) * full(cb)))
    assert abs(ctx.dot_noalloc(a, b) - want) <= 1e-12 * np.linalg.norm(full(ca)) * np.linalg.norm(full(cb))


def test_dot_noalloc_rejects_ranks_beyond_the_static_scratch(ctx):
    from paper_1906_06785_gb300 import binding
    rng = np.random.default_rng(3)
    # r1a * n_xi * r2b = 100 * 20 * 1100 = 2.2e6 > 2^21 doubles
    a, _ = _train(ctx, rng, 100, 20, 64, 100, 8)
    b, _ = _train(ctx, rng, 100, 20, 64, 4, 1100)
    with pytest.raises(binding.LibraryError, match="static scratch"):
        ctx.dot_noalloc(a, b)
    # the context stays usable and the entry point still answers for fitting sizes
    assert abs(ctx.dot_noalloc(a, a) - ctx.dot(a, a)) <= 1e-12 * ctx.dot(a, a)
