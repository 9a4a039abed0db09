"""Batched form: independent problems solved concurrently (one context and stream
per problem, picard_solve_batched) give the same solutions as one-by-one solves."""
import numpy as np

from ttfull import full
import pytest

pytestmark = pytest.mark.gpu


def test_batched_solves_match_sequential_solves():
    import torch
    import synth
    from paper_1906_06785_gb300 import binding
    probs = synth.batch("tiny", 3, seed=5, nu0_range=(1 / 50, 1 / 20))
    ref = []
    c0 = binding.Context()
    for pr in probs:
        u, p, st, code = c0.problem(pr).picard(binding.opts_from(pr.tol))
        assert code == binding.TT_OK
        ref.append((full(u), full(p), st.picard_its))
    streams = [torch.cuda.Stream() for _ in probs]
    ctxs = [binding.Context(stream=s.cuda_stream) for s in streams]
    handles = [c.problem(pr) for c, pr in zip(ctxs, probs)]
    out = binding.picard_batched(handles, [binding.opts_from(pr.tol) for pr in probs])
    assert len(out) == len(probs)
    for (u, p, st, code, sec), (ru, rp, rits) in zip(out, ref):
        assert code == binding.TT_OK
        assert sec > 0.0
        assert st.picard_its == rits
        assert np.linalg.norm(full(u) - ru) <= 1e-12 * np.linalg.norm(ru)
        assert np.linalg.norm(full(p) - rp) <= 1e-12 * np.linalg.norm(rp)


def test_batched_rejects_problems_sharing_a_context():
    import synth
    from paper_1906_06785_gb300 import binding
    probs = synth.batch("tiny", 2, seed=6, nu0_range=(1 / 50, 1 / 20))
    c = binding.Context()
    handles = [c.problem(pr) for pr in probs]
    with pytest.raises(binding.LibraryError, match="share a context"):
        binding.picard_batched(handles, binding.opts_from(probs[0].tol))
