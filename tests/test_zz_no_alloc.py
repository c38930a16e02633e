"""nmf_gram_noalloc: the Gram matrix for callers that cannot allocate device
memory (its partial sums live in a fixed static device array).  Checked
through the C ABI against the context's own Gram step (nmf_run_step with
NMF_STEP_S) and against FP64, on two calls in a row with different shapes so
that nothing left in the shared array from the first call can leak into the
second."""

import numpy as np
import pytest

from paper_1904_07935_b300 import synth

pytestmark = pytest.mark.gpu

TOL = 2e-6        # max-norm relative, as for the other Gram / product parity tests


def _existing_gram(nmf, torch, W, V, K):
    # A context whose W buffer is set to W; its Gram step computes S = W^T W.
    sp = synth.sparse_termdoc(V, max(K, 64), 3, mean_terms=8)
    ctx = nmf.from_sparse(sp, K)
    ctx.set_buffer(nmf.BUF_W, W)
    ctx.run_step(nmf.STEP_S)
    return ctx.get_buffer(nmf.BUF_S).astype(np.float64)


def test_gram_noalloc_matches_existing_gram_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1904_07935_b300 import nmf
    for (V, K, seed) in ((3000, 48, 1), (5000, 37, 2)):
        W, _ = synth.init_factors(seed, V, 8, K)
        Xd = torch.from_numpy(W).cuda()
        Sd = torch.full((K, K), float("nan"), device="cuda")
        nmf.gram_noalloc(Xd, Sd)
        torch.cuda.synchronize()
        got = Sd.cpu().numpy().astype(np.float64)
        ref = _existing_gram(nmf, torch, W, V, K)
        exact = W.astype(np.float64).T @ W.astype(np.float64)
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < TOL
        assert np.max(np.abs(got - exact)) / np.max(np.abs(exact)) < TOL
