"""nmf_gram_noalloc: the Gram matrix for callers that cannot allocate device
memory (its partial sums live in a fixed static device array).  Checked
through the C ABI against the context's own Gram step (nmf_run_step with
NMF_STEP_S) and against FP64, on calls in a row with different shapes, so
that nothing left in the shared array by one call can leak into the next.
The shapes reach each code path: the small-tile and 128-row-tile SIMT
kernels (K = 48, 37 and 128 with a row stride that is not a multiple of
four), the FP64 combination of more than 256 row chunks (K = 32, N = 100,000)
and the one-chunk limit of the array (K = 2048).  Free device memory is the
same before and after the calls, and K beyond the array is rejected."""

import numpy as np
import pytest

from paper_1904_07935_b300 import synth

pytestmark = pytest.mark.gpu

TOL = 2e-6        # max-norm relative, as for the other Gram / product parity tests


def _existing_gram(nmf, W, V, K):
    # A context whose W buffer is set to W; its Gram step computes S = W^T W.
    sp = synth.sparse_termdoc(V, max(K, 64), 3, mean_terms=8)
    ctx = nmf.from_sparse(sp, K)
    ctx.set_buffer(nmf.BUF_W, W)
    ctx.run_step(nmf.STEP_S)
    return ctx.get_buffer(nmf.BUF_S).astype(np.float64)


def _call(nmf, Xd, V, K, ldx, Sd):
    # Straight through the C ABI: X is V x K inside a V x ldx buffer.
    st = nmf.lib.nmf_gram_noalloc(Xd.data_ptr(), V, K, ldx, Sd.data_ptr(), None)
    assert st == nmf.NMF_OK, nmf.lib.nmf_status_str(st)


def _rel(got, ref):
    return np.max(np.abs(got - ref)) / np.max(np.abs(ref))


def test_gram_noalloc_matches_existing_gram_and_fp64():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1904_07935_b300 import nmf
    cases = ((3000, 48, 48, 1, True), (5000, 37, 37, 2, True), (4000, 128, 131, 4, True),
             (100000, 32, 32, 5, False), (300, 2048, 2048, 6, False))   # no context of those sizes
    data = []
    for V, K, ldx, seed, ctx_ref in cases:
        W, _ = synth.init_factors(seed, V, 8, K)
        Xh = np.zeros((V, ldx), dtype=np.float32)
        Xh[:, :K] = W
        data.append((V, K, ldx, W, torch.from_numpy(Xh).cuda(), torch.full((K, K), float("nan"), device="cuda"),
                     ctx_ref))
    # First round: the first call on the device looks up the array's address,
    # and the driver loads the library's kernels on their first use (lazy
    # module loading), both of which may take device memory once.
    for V, K, ldx, W, Xd, Sd, _ in data:
        _call(nmf, Xd, V, K, ldx, Sd)
        Sd.fill_(float("nan"))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for V, K, ldx, W, Xd, Sd, _ in data:          # second round, checked below
        _call(nmf, Xd, V, K, ldx, Sd)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0                          # no device allocation by the calls
    for V, K, ldx, W, Xd, Sd, ctx_ref in data:
        got = Sd.cpu().numpy().astype(np.float64)
        exact = W.astype(np.float64).T @ W.astype(np.float64)
        assert _rel(got, exact) < TOL, (V, K)
        if ctx_ref:
            assert _rel(got, _existing_gram(nmf, W, V, K)) < TOL, (V, K)


def test_gram_noalloc_rejects_k_beyond_the_array():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1904_07935_b300 import nmf
    X = torch.zeros((64, 2049), device="cuda")
    S = torch.zeros((2049, 2049), device="cuda")
    with pytest.raises(nmf.NmfError) as e:
        nmf.gram_noalloc(X, S)
    assert e.value.status == nmf.NMF_EUNSUPPORTED
