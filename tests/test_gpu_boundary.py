"""The C-ABI boundary beyond the hot-path kernels: caller allocators, rank
capacities and TT_ERANK, tt_norm, truncating axpby, preconditioner objects and
resuming a Picard solve from a given iterate (Algorithm 3.1)."""
import numpy as np
import pytest

import synth
from oracle import tt as otm
from ttfull import full

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def binding():
    from paper_1906_06785_gb300 import binding as b
    return b


@pytest.fixture(scope="module")
def ctx(binding):
    return binding.Context()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _capped_tt_svd(Z, c1, c2):
    """Algorithm 4.1 with fixed ranks: project the first unfolding on its c1 leading
    left singular vectors, then the second unfolding of the result on its c2."""
    n_t, n_xi, n_x = Z.shape
    U, _, _ = np.linalg.svd(Z.reshape(n_t, -1), full_matrices=False)
    U1 = U[:, :c1]
    Z1 = (U1 @ (U1.T @ Z.reshape(n_t, -1))).reshape(n_t * n_xi, n_x)
    U, _, _ = np.linalg.svd(Z1, full_matrices=False)
    U2 = U[:, :c2]
    return (U2 @ (U2.T @ Z1)).reshape(n_t, n_xi, n_x)


def test_caller_allocator_serves_every_device_buffer(binding):
    import torch
    live, count = {}, [0]

    def alloc(nbytes, stream):
        p = torch.cuda.caching_allocator_alloc(nbytes, torch.cuda.current_device(), stream)
        live[p] = nbytes
        count[0] += 1
        return p

    def free(p, nbytes, stream):
        assert live.pop(p) == nbytes
        torch.cuda.caching_allocator_delete(p)

    c = binding.Context(alloc=alloc, free=free)
    z = otm.TT(*synth.random_tt(8, 4, 300, 6, 20, seed=5, decay=8))
    t = c.tt(z.z1, z.z2, z.z3)
    g, nb, na = c.round(t, 1e-6)
    ref, nref = otm.round_tt(z, 1e-6)
    assert g.ranks == ref.ranks and abs(nb - nref) < 1e-12 * nref
    assert otm.norm(otm.add((1.0, otm.TT(*g.cores())), (-1.0, ref))) < 1e-9 * nref
    assert count[0] > 5
    del t, g
    torch.cuda.synchronize()
    c.close()
    assert not live, f"{len(live)} buffers not returned"


def test_one_sided_allocator_is_refused(binding):
    with pytest.raises(ValueError):
        binding.Context(alloc=lambda n, s: 0)


def test_capacity_and_round_to(ctx, binding):
    z = otm.TT(*synth.random_tt(10, 5, 400, 8, 30, seed=7, decay=7))
    t = ctx.tt(z.z1, z.z2, z.z3, cap=(12, 40))
    assert t.ranks == (8, 30) and t.capacity == (12, 40)
    ref, nref = otm.round_tt(z, 1e-4)
    out = ctx.tt(np.zeros((10, 1)), np.zeros((1, 5, 1)), np.zeros((1, 400)), cap=(10, 30))
    code, nb, na = ctx.round_to(t, 1e-4, out)
    assert code == binding.TT_OK and out.ranks == ref.ranks and out.capacity == (10, 30)
    assert otm.norm(otm.add((1.0, otm.TT(*out.cores())), (-1.0, ref))) < 1e-9 * nref


def test_round_to_a_small_capacity_reports_erank(ctx, binding):
    z = otm.TT(*synth.random_tt(9, 4, 200, 7, 15, seed=11, decay=6))
    t = ctx.tt(z.z1, z.z2, z.z3)
    out = ctx.tt(np.zeros((9, 1)), np.zeros((1, 4, 1)), np.zeros((1, 200)), cap=(3, 5))
    code, nb, na = ctx.round_to(t, 1e-8, out)
    assert code == binding.TT_ERANK
    assert out.ranks == (3, 5)
    want = _capped_tt_svd(z.full(), 3, 5)
    assert _rel(full(out), want) < 1e-9
    # the context stays usable after the error
    code, _, _ = ctx.round_to(t, 1e-1, out)
    assert code == binding.TT_OK


def test_norm_and_truncating_axpby(ctx):
    za = otm.TT(*synth.random_tt(6, 4, 120, 3, 9, seed=21, decay=5))
    zb = otm.TT(*synth.random_tt(6, 4, 120, 2, 7, seed=22, decay=5))
    a, b = ctx.tt(za.z1, za.z2, za.z3), ctx.tt(zb.z1, zb.z2, zb.z3)
    assert abs(ctx.norm(a) - otm.norm(za)) < 1e-13 * otm.norm(za)
    s = ctx.axpby(0.5, a, -2.0, b, eps=1e-3)
    ref, _ = otm.round_tt(otm.add((0.5, za), (-2.0, zb)), 1e-3)
    assert s.ranks == ref.ranks
    assert otm.norm(otm.add((1.0, otm.TT(*s.cores())), (-1.0, ref))) < 1e-9 * otm.norm(ref)
    plain = ctx.axpby(0.5, a, -2.0, b)
    assert plain.ranks == (5, 16)


def test_preconditioner_kinds(ctx, binding):
    prob = synth.preset("tiny")
    P = ctx.problem(prob)
    op = P.op(None)
    with pytest.raises(binding.LibraryError, match="kind"):
        op.make_prec(7, 1e-8, 1e-1, 10)
    with pytest.raises(binding.LibraryError, match="network"):
        op.make_prec(binding.PREC_LEARNED, 1e-8, 1e-1, 10)
    fu, fp = P.rhs()
    pr = op.make_prec(binding.PREC_LSC, 1e-10, 1e-6, 30)
    u1, p1, its1, fb = pr.apply(fu, fp)
    u2, p2, its2, _ = op.prec(fu, fp, 1e-10, 1e-6, 30)
    assert its1 == its2 and fb == 0
    assert _rel(full(u1), full(u2)) < 1e-13 and _rel(full(p1), full(p2)) < 1e-13
    # GMRES with an explicit preconditioner object equals the default one
    o = binding.opts_from(prob.tol, tol_gmres=1e-6, eps_gmres=1e-10, tol_inner=1e-6)
    pr2 = op.make_prec(binding.PREC_LSC, o.eps_gmres, o.tol_inner, o.maxit_inner)
    za, pa, sa, _ = op.gmres(o, fu, fp, prec=pr2)
    zb, pb, sb, _ = op.gmres(o, fu, fp)
    assert sa.its == sb.its and _rel(full(za), full(zb)) < 1e-12


def test_picard_resumes_from_a_given_iterate(ctx, binding):
    prob = synth.preset("tiny")
    prob.tol.eps_gmres, prob.tol.eps_soln, prob.tol.eps_conv = 1e-8, 1e-10, 1e-8
    P = ctx.problem(prob)
    u, p, st, code = P.picard(binding.opts_from(prob.tol))
    assert code == binding.TT_OK and st.picard_its >= 3
    # stop after two steps, then resume from there
    u2, p2, st2, code2 = P.picard(binding.opts_from(prob.tol, maxit_picard=2))
    assert code2 == binding.TT_ENOCONV and st2.picard_its == 2
    u3, p3, st3, code3 = P.picard(binding.opts_from(prob.tol, init=(u2, p2)))
    assert code3 == binding.TT_OK
    assert st3.stokes_its == 0 and st3.picard_its == st.picard_its - 2
    assert abs(st3.res[0] - st.res[2]) <= 1e-12 * st.res[2]
    assert _rel(full(u3), full(u)) < 1e-12 and _rel(full(p3), full(p)) < 1e-12


def test_device_wait_limit_gives_timeout_and_recovers(ctx, binding):
    """A cooperative Householder R factor over many CTAs (n_x = 60000 rows of z3, more
    than one cluster's shared memory holds, spread over the whole GPU) with a wait limit
    of 0 polls: blocks that reach a grid barrier before the others give up, the call
    returns TT_ETIMEOUT, and with the default limit the same call succeeds on the same
    context."""
    z = otm.TT(*synth.random_tt(6, 3, 60000, 4, 12, seed=41, decay=4))
    t = ctx.tt(z.z1, z.z2, z.z3)
    ref, nref = otm.round_tt(z, 1e-8)
    ctx.set_wait_limit(0)
    try:
        with pytest.raises(binding.LibraryError) as e:
            ctx.round(t, 1e-8)
        assert e.value.code == binding.TT_ETIMEOUT
    finally:
        ctx.set_wait_limit(20000000)
    g, nb, na = ctx.round(t, 1e-8)
    assert g.ranks == ref.ranks and abs(nb - nref) <= 1e-12 * nref
